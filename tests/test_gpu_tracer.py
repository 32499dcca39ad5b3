"""GPU parity of the non-conservative product (system ADER_SYSTEM_TRACER: 1D
Euler with a passive tracer in non-conservative form; nested Picard predictor
with the b term, B volume term, path-conservative Rusanov face) against the
oracle's ob_nc_* family.  Bar: 1e-12 relative L-inf per step, 1e-10 after a
solve; the uniform-flow invariant (tracer = rho) through the GPU path."""
import numpy as np
import pytest

from conftest import rel_linf
from test_oracle_nc import state

pytestmark = pytest.mark.gpu

GAMMA = 1.4


def make(nc, N, **kw):
    from paper_2409_12483_gb300 import Context
    return Context(nc, N, "dg", system="tracer", **kw)


def to_dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("N", range(0, 8))
def test_step_parity(cuda, oracle_mod, N):
    import torch
    nc = 37  # two interface tiles, a ragged tail
    o = oracle_mod.NCOracle(N)
    u = state(o, nc, seed=N)
    dt = o.dt(u, 1.0 / nc)
    ref, rc, _ = o.step(u, 1.0 / nc, dt)
    assert rc == 0
    ctx = make(nc, N)
    ud = to_dev(u)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, dt)
    torch.cuda.synchronize()
    assert rel_linf(out.cpu().numpy(), ref) < 1e-12
    assert abs(ctx.ader_compute_dt(ud) - dt) < 1e-14 * dt


@pytest.mark.parametrize("N", [2, 5])
def test_fixed_iteration_step_parity(cuda, oracle_mod, N):
    import torch
    nc = 24
    o = oracle_mod.NCOracle(N, fixed_iter=2)
    u = state(o, nc, seed=11)
    dt = o.dt(u, 1.0 / nc)
    ref, rc, _ = o.step(u, 1.0 / nc, dt)
    ctx = make(nc, N, picard_fixed_iter=2)
    ud = to_dev(u)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, dt)
    torch.cuda.synchronize()
    assert rel_linf(out.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("N", [1, 3, 6])
def test_solve_parity(cuda, oracle_mod, N):
    import torch
    nc = 20
    o = oracle_mod.NCOracle(N)
    u = state(o, nc, seed=4)
    ref, steps_ref, t_ref, rc = o.solve(u, 1.0 / nc, t_end=0.3)
    assert rc == 0
    ctx = make(nc, N)
    ud = to_dev(u)
    steps, t, rc = ctx.ader_solve(ud, t_end=0.3)
    torch.cuda.synchronize()
    assert rc == 0 and steps == steps_ref and t == 0.3
    assert rel_linf(ud.cpu().numpy(), ref) < 1e-10


def test_tracer_equal_to_rho_in_uniform_flow(cuda, oracle_mod):
    import torch
    N, nc = 4, 16
    o = oracle_mod.NCOracle(N)
    U = state(o, nc, phi_fn=lambda x, rho: rho, u_fn=lambda x: np.ones_like(x))
    U[..., 2] = 1 / (GAMMA - 1) + 0.5 * U[..., 0]
    ctx = make(nc, N)
    ud = to_dev(U)
    steps, t, rc = ctx.ader_solve(ud, max_steps=40)
    torch.cuda.synchronize()
    out = ud.cpu().numpy().reshape(nc, N + 1, 4)
    assert rc == 0 and steps == 40
    assert np.abs(out[..., 3] - out[..., 0]).max() < 1e-12


@pytest.mark.parametrize("nc,N", [(1, 3), (2, 0), (33, 7)])
def test_degenerate_and_tile_edge_meshes(cuda, oracle_mod, nc, N):
    """one cell (its own neighbour), two cells, and one cell past a full tile"""
    import torch
    o = oracle_mod.NCOracle(N)
    u = state(o, nc, seed=nc)
    dt = o.dt(u, 1.0 / nc)
    ref, rc, _ = o.step(u, 1.0 / nc, dt)
    ctx = make(nc, N)
    ud = to_dev(u)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, dt)
    torch.cuda.synchronize()
    assert rc == 0 and rel_linf(out.cpu().numpy(), ref) < 1e-12
