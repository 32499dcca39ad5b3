"""FP64-accurate float-float predictor (precision "ff"): the Picard iteration runs
in float-float arithmetic on the FP32 pipes, the epilogue, corrector and CFL in
FP64.  It must meet the same parity bar as the FP64 path: 1e-12 relative L-inf
against the FP64 oracle per step and 1e-10 at t_end."""
import numpy as np
import pytest

import workloads as W
from conftest import rel_linf
from test_gpu_dg import NCELLS, field_nonlinear, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N", range(1, 8))
@pytest.mark.parametrize("fixed", [True, False])
def test_ff_predictor_parity(cuda, oracle_mod, N, fixed):
    import torch
    from paper_2409_12483_gb300 import Context
    o = oracle_mod.Oracle(N)
    u = W.nodal_state(field_nonlinear(N), o.node_x(NCELLS))
    dx = 1.0 / NCELLS
    dt = o.dg_dt(u, dx)
    it = N + 3 if fixed else 0
    o.set(fixed_iter=it)
    q_ref, iters = o.predict(u, dt / dx)
    ctx = Context(NCELLS, N, "dg", precision="ff", picard_fixed_iter=it)
    q = torch.empty(ctx.predictor_count, dtype=torch.float64, device=cuda)
    ctx.ader_predict(to_dev(u, cuda), dt, q)
    torch.cuda.synchronize()
    assert rel_linf(q.cpu().numpy(), q_ref) < 1e-12
    st = ctx.ader_get_stats()
    assert st["status"] == 0
    if not fixed:
        assert abs(st["max_iters"] - iters.max()) <= 1


@pytest.mark.parametrize("N", range(0, 8))
def test_ff_step_parity(cuda, oracle_mod, N):
    import torch
    from paper_2409_12483_gb300 import Context
    o = oracle_mod.Oracle(N)
    u = W.nodal_state(field_nonlinear(30 + N), o.node_x(NCELLS))
    dx = 1.0 / NCELLS
    dt = o.dg_dt(u, dx)
    ref, _, _, rc = o.dg_step(u, dx, dt)
    ctx = Context(NCELLS, N, "dg", precision="ff")
    ud = to_dev(u, cuda)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, 0.0)
    torch.cuda.synchronize()
    assert rel_linf(out.cpu().numpy(), ref) < 1e-12


def test_ff_sine_wave_one_period(cuda, oracle_mod):
    import torch
    from paper_2409_12483_gb300 import Context
    N, nc = 2, 100
    o = oracle_mod.Oracle(N)
    f = W.sine()
    u = W.nodal_state(f, o.node_x(nc))
    ref, steps_ref, _, _ = o.solve("dg", u, 1.0 / nc, t_end=1.0)
    ctx = Context(nc, N, "dg", precision="ff")
    ud = to_dev(u, cuda)
    steps, t, rc = ctx.ader_solve(ud, t_end=1.0)
    torch.cuda.synchronize()
    assert steps == steps_ref and t == 1.0
    assert rel_linf(ud.cpu().numpy(), ref) < 1e-10


@pytest.mark.parametrize("N", [2, 4])
def test_ff_weno_fv_step(cuda, oracle_mod, N):
    import torch
    from paper_2409_12483_gb300 import Context
    o = oracle_mod.Oracle(N)
    v = W.cell_average_state(field_nonlinear(40 + N), NCELLS)
    dx = 1.0 / NCELLS
    dt = o.fv_dt(v, dx)
    ref, _, _ = o.fv_step(v, dx, dt)
    ctx = Context(NCELLS, N, "fv", precision="ff")
    vd = to_dev(v, cuda)
    out = torch.empty_like(vd)
    ctx.ader_step(vd, out, dt)
    torch.cuda.synchronize()
    assert rel_linf(out.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("N,nc", [(5, 100_000), (7, 1_000_000)])
def test_ff_full_size_sampled(cuda, oracle_mod, N, nc):
    import torch
    from paper_2409_12483_gb300 import Context
    o = oracle_mod.Oracle(N)
    u = W.nodal_state(W.modes4(), o.node_x(nc))
    dx = 1.0 / nc
    ctx = Context(nc, N, "dg", precision="ff")
    ud = to_dev(u, cuda)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, 0.0)
    torch.cuda.synchronize()
    dt = o.dg_dt(u, dx)
    cells = np.unique(np.concatenate([[0, nc - 1], np.random.default_rng(5).integers(0, nc, 30)]))
    sel, _ = o.dg_step_cells(u, dx, dt, cells)
    assert rel_linf(out.cpu().numpy().reshape(nc, N + 1, 3)[cells], sel) < 1e-12


def test_ff_predictor_weno_fv_many_steps(cuda):
    """The float-float predictor fed by WENO5 (the FV time step has no 1/(2N+1)
    factor, so the Picard map contracts more weakly): 100 steps on 10^5 cells
    without hitting the iteration cap, within 1e-11 of the FP64 path."""
    import torch
    from paper_2409_12483_gb300 import Context
    nc = 100_000
    v0 = torch.tensor(W.cell_average_state(W.modes4(), nc), device=cuda).reshape(-1)
    a = Context(nc, 4, "fv")
    b = Context(nc, 4, "fv", precision="ff")
    va, vb = v0.clone(), v0.clone()
    a.ader_solve(va, max_steps=100)
    steps, t, rc = b.ader_solve(vb, max_steps=100)
    torch.cuda.synchronize()
    assert rc == 0 and steps == 100
    assert rel_linf(vb.cpu().numpy(), va.cpu().numpy()) < 1e-11
