"""The FP32-predictor forms: Picard in FP32, then FP64 sweeps (precision "fp32")
or float-float sweeps and epilogue (precision "fp32ff"), corrector and CFL in
FP64.  It is compared with the FP64 oracle and with the exact advected
solution; the target is an L1 error within 2x of the FP64 form's at N <= 5."""
import numpy as np
import pytest

import workloads as W
from conftest import rel_linf

pytestmark = pytest.mark.gpu


def to_dev(a, cuda):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=cuda)


@pytest.mark.parametrize("prec", ["fp32", "fp32ff"])
@pytest.mark.parametrize("N,nc", [(2, 40), (3, 20), (5, 10)])
def test_fp32_predictor_error_vs_exact(cuda, oracle_mod, N, nc, prec):
    import torch
    from paper_2409_12483_gb300 import Context
    o = oracle_mod.Oracle(N)
    f = W.sine()
    u = W.nodal_state(f, o.node_x(nc))
    exact = lambda x: f.rho(x, 1.0)
    ref, steps_ref, _, _ = o.solve("dg", u, 1.0 / nc, t_end=1.0)
    e64 = oracle_mod.dg_density_errors(o, ref, exact)[0]
    ctx = Context(nc, N, "dg", precision=prec, fp64_sweeps=2)
    ud = to_dev(u, cuda)
    steps, t, rc = ctx.ader_solve(ud, t_end=1.0)
    torch.cuda.synchronize()
    got = ud.cpu().numpy()
    e32 = oracle_mod.dg_density_errors(o, got, exact)[0]
    assert steps == steps_ref
    assert e32 <= 2.0 * e64, (e32, e64)


def test_fp32_predictor_one_step_n7_sampled(cuda, oracle_mod):
    """DG N = 7, 10^6 cells: one step of the FP32-predictor form against the FP64
    oracle on sampled cells.  The FP32 stage stops at its own tolerance (1e-6);
    each FP64 sweep then contracts the predictor error, so two sweeps must beat one."""
    import torch
    from paper_2409_12483_gb300 import Context
    N, nc = 7, 1_000_000
    o = oracle_mod.Oracle(N)
    u = W.nodal_state(W.modes4(), o.node_x(nc))
    dx = 1.0 / nc
    ud = to_dev(u, cuda)
    dt = o.dg_dt(u, dx)
    cells = np.random.default_rng(2).integers(0, nc, 24)
    sel, _ = o.dg_step_cells(u, dx, dt, cells)
    errs = []
    for sweeps in (1, 2, 3):
        ctx = Context(nc, N, "dg", precision="fp32", fp64_sweeps=sweeps)
        out = torch.empty_like(ud)
        ctx.ader_step(ud, out, 0.0)
        torch.cuda.synchronize()
        errs.append(rel_linf(out.cpu().numpy().reshape(nc, N + 1, 3)[cells], sel))
        del ctx
    print("FP32 predictor, N = 7: rel Linf vs FP64 oracle after 1/2/3 FP64 sweeps:", errs)
    assert errs[0] < 1e-7
    assert errs[1] < errs[0] and errs[2] < errs[1]


def test_fp32_ff_sweeps_one_step_n7_sampled(cuda, oracle_mod):
    """DG N = 7, 10^6 cells: the FP32 stage followed by float-float sweeps
    contracts the predictor error like FP64 sweeps do (each sweep by the same
    factor, to within 3x of the FP64-sweep form's error at every sweep count)."""
    import torch
    from paper_2409_12483_gb300 import Context
    N, nc = 7, 1_000_000
    o = oracle_mod.Oracle(N)
    u = W.nodal_state(W.modes4(), o.node_x(nc))
    dx = 1.0 / nc
    ud = to_dev(u, cuda)
    dt = o.dg_dt(u, dx)
    cells = np.random.default_rng(3).integers(0, nc, 24)
    sel, _ = o.dg_step_cells(u, dx, dt, cells)
    errs = {}
    for prec in ("fp32", "fp32ff"):
        for sweeps in (1, 2, 3):
            ctx = Context(nc, N, "dg", precision=prec, fp64_sweeps=sweeps)
            out = torch.empty_like(ud)
            ctx.ader_step(ud, out, 0.0)
            torch.cuda.synchronize()
            errs[prec, sweeps] = rel_linf(out.cpu().numpy().reshape(nc, N + 1, 3)[cells], sel)
            del ctx
    print("N = 7 rel Linf vs FP64 oracle per sweep count:", errs)
    for sweeps in (1, 2, 3):
        a, b = errs["fp32ff", sweeps], errs["fp32", sweeps]
        assert a < 3.0 * b and b < 3.0 * a
    assert errs["fp32ff", 1] < 1e-7
    assert errs["fp32ff", 3] < errs["fp32ff", 2] < errs["fp32ff", 1]


@pytest.mark.parametrize("N", [1, 4, 7])
def test_fp32_ff_predictor_against_oracle(cuda, oracle_mod, N):
    """The predictor q of the fp32ff form against the FP64 oracle's converged q:
    within the FP32 stage's tolerance, and closer with more sweeps."""
    import torch
    from paper_2409_12483_gb300 import Context
    from test_gpu_dg import NCELLS, field_nonlinear
    o = oracle_mod.Oracle(N)
    u = W.nodal_state(field_nonlinear(50 + N), o.node_x(NCELLS))
    dx = 1.0 / NCELLS
    dt = o.dg_dt(u, dx)
    q_ref, _ = o.predict(u, dt / dx)
    e = []
    for sweeps in (1, 4):
        ctx = Context(NCELLS, N, "dg", precision="fp32ff", fp64_sweeps=sweeps)
        q = torch.empty(ctx.predictor_count, dtype=torch.float64, device=cuda)
        ctx.ader_predict(to_dev(u, cuda), dt, q)
        torch.cuda.synchronize()
        e.append(rel_linf(q.cpu().numpy(), q_ref))
        assert ctx.ader_get_stats()["status"] == 0
    assert e[0] < 1e-5 and e[1] < e[0]
