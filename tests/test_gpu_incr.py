"""The increment form of the predictor (precision "incr"): the tau-independent
first Picard iteration and the terms of u in float-float, the later iterations
on the correction in FP32 with F(u + d) - F(u) as exact differences.  Its FP32
rounding is relative to the size of the correction, so its distance from the
FP64 oracle shrinks with the step: FP64-grade (the 1e-12 per-step bar) on the
fine meshes of the throughput configurations, within 1e-10 per step on coarse
meshes of ~100 cells, and within 2x of the FP64 form's L1 error against the exact
solution wherever the discretisation error is above that level."""
import numpy as np
import pytest

import workloads as W
from conftest import rel_linf
from test_gpu_dg import NCELLS, field_nonlinear, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N", range(1, 8))
def test_incr_step_coarse_mesh(cuda, oracle_mod, N):
    """103 cells (several predictor tiles and a ragged tail), device CFL step"""
    import torch
    from paper_2409_12483_gb300 import Context
    o = oracle_mod.Oracle(N)
    u = W.nodal_state(field_nonlinear(N), o.node_x(NCELLS))
    dx = 1.0 / NCELLS
    dt = o.dg_dt(u, dx)
    ref, _, _, rc = o.dg_step(u, dx, dt)
    ctx = Context(NCELLS, N, "dg", precision="incr")
    ud = to_dev(u, cuda)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, 0.0)
    torch.cuda.synchronize()
    assert rc == 0 and ctx.ader_get_stats()["status"] == 0
    assert rel_linf(out.cpu().numpy(), ref) < 1e-10


@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_incr_step_fine_mesh_meets_fp64_bar(cuda, oracle_mod, N):
    """10^5 cells: one step against the oracle's per-cell step on sampled cells
    at the FP64 bar (1e-12 relative L-inf)"""
    import torch
    from paper_2409_12483_gb300 import Context
    nc = 100_000
    o = oracle_mod.Oracle(N)
    u = W.nodal_state(W.modes4(), o.node_x(nc))
    dx = 1.0 / nc
    dt = o.dg_dt(u, dx)
    cells = np.unique(np.concatenate([[0, 1, nc - 1], np.random.default_rng(N).integers(0, nc, 30)]))
    sel, rc = o.dg_step_cells(u, dx, dt, cells)
    ctx = Context(nc, N, "dg", precision="incr")
    ud = to_dev(u, cuda)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, dt)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(nc, N + 1, 3)[cells]
    assert rc == 0 and rel_linf(got, sel) < 1e-12


@pytest.mark.parametrize("N,nc", [(2, 40), (3, 20), (5, 10)])
def test_incr_error_vs_exact_within_2x_of_fp64(cuda, oracle_mod, N, nc):
    import torch
    from paper_2409_12483_gb300 import Context
    o = oracle_mod.Oracle(N)
    f = W.sine()
    u = W.nodal_state(f, o.node_x(nc))
    exact = lambda x: f.rho(x, 1.0)
    ref, steps_ref, _, _ = o.solve("dg", u, 1.0 / nc, t_end=1.0)
    e64 = oracle_mod.dg_density_errors(o, ref, exact)[0]
    ctx = Context(nc, N, "dg", precision="incr")
    ud = to_dev(u, cuda)
    steps, t, rc = ctx.ader_solve(ud, t_end=1.0)
    torch.cuda.synchronize()
    e = oracle_mod.dg_density_errors(o, ud.cpu().numpy(), exact)[0]
    assert rc == 0 and steps == steps_ref
    assert e <= 2.0 * e64, (e, e64)


@pytest.mark.parametrize("N", [2, 5])
def test_incr_predictor_against_oracle(cuda, oracle_mod, N):
    """q itself (ader_predict) against the oracle's converged q on 10^4 cells"""
    import torch
    from paper_2409_12483_gb300 import Context
    nc = 10_000
    o = oracle_mod.Oracle(N)
    u = W.nodal_state(field_nonlinear(60 + N), o.node_x(nc))
    dx = 1.0 / nc
    dt = o.dg_dt(u, dx)
    cells = np.random.default_rng(5).integers(0, nc, 40)
    q_ref, _ = o.predict(u.reshape(nc, N + 1, 3)[cells], dt / dx)
    ctx = Context(nc, N, "dg", precision="incr")
    q = torch.empty(ctx.predictor_count, dtype=torch.float64, device=cuda)
    ctx.ader_predict(to_dev(u, cuda), dt, q)
    torch.cuda.synchronize()
    got = q.cpu().numpy().reshape(nc, N + 1, N + 1, 3)[cells]
    assert rel_linf(got, q_ref) < 1e-12
    assert ctx.ader_get_stats()["status"] == 0


def test_incr_hundred_steps_against_fp64_path(cuda):
    """the headline workload (N = 5, 10^5 cells, 100 CFL steps): the increment
    form stays within 1e-11 relative L-inf of the FP64 path"""
    import torch
    from paper_2409_12483_gb300 import Context
    nc, N = 100_000, 5
    a = Context(nc, N, "dg")
    b = Context(nc, N, "dg", precision="incr")
    u0 = torch.tensor(W.nodal_state(W.modes4(12483), a.node_coords()), device=cuda).reshape(-1)
    ua, ub = u0.clone(), u0.clone()
    sa, ta, _ = a.ader_solve(ua, max_steps=100)
    sb, tb, rc = b.ader_solve(ub, max_steps=100)
    torch.cuda.synchronize()
    assert sa == sb == 100 and rc == 0
    assert abs(ta - tb) <= 1e-12 * ta
    assert rel_linf(ub.cpu().numpy(), ua.cpu().numpy()) < 1e-11


def test_incr_weno_step(cuda, oracle_mod):
    """the same predictor fed by the WENO5 reconstruction (FV scheme)"""
    import torch
    from paper_2409_12483_gb300 import Context
    N, nc = 4, 1000
    o = oracle_mod.Oracle(N)
    v = W.cell_average_state(field_nonlinear(77), nc)
    dt = o.fv_dt(v, 1.0 / nc)
    ref, _, rc = o.fv_step(v, 1.0 / nc, dt)
    ctx = Context(nc, N, "fv", precision="incr")
    vd = to_dev(v, cuda)
    out = torch.empty_like(vd)
    ctx.ader_step(vd, out, dt)
    torch.cuda.synchronize()
    assert rc == 0 and rel_linf(out.cpu().numpy(), ref) < 1e-10
