"""GPU parity of the 2D Euler ADER-DG path (ader_init_2d: tensor-product
predictor of Sec. 1.1, x/y faces of Sec. 1.2, d = 2 time step of Sec. 1.5)
against the oracle's ob2_* family.  Bar: 1e-12 relative L-inf per step, 1e-10
after a solve; the sine-wave errors of Sec. 2.1 through the GPU path equal the
oracle's."""
import numpy as np
import pytest

from conftest import rel_linf

pytestmark = pytest.mark.gpu

GAMMA = 1.4


def conserved2(rho, u, v, p, g=GAMMA):
    return np.stack([rho, rho * u, rho * v, p / (g - 1) + 0.5 * rho * (u * u + v * v)], -1)


def smooth_state(o, nx, ny, seed=0, x1=1.0, y1=1.0):
    X, Y = o.node_xy(nx, ny, 0.0, x1, 0.0, y1)
    X, Y = X / x1, Y / y1
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.05, 0.15, 4)
    rho = 1 + a[0] * np.sin(2 * np.pi * (X + 2 * Y)) + a[1] * np.cos(2 * np.pi * X)
    u = 0.6 + a[2] * np.sin(2 * np.pi * Y)
    v = -0.4 + a[3] * np.cos(2 * np.pi * (X - Y))
    p = 1 + 0.1 * np.sin(2 * np.pi * (2 * X + Y))
    return conserved2(rho, u, v, p)


def make(nx, ny, N, **kw):
    from paper_2409_12483_gb300 import Context2D
    return Context2D(nx, ny, N, **kw)


def to_dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("N", range(0, 8))
def test_step_parity(cuda, oracle_mod, N):
    """one step on smooth data, a ragged number of cells (several blocks, a
    partial last block), dx != dy"""
    import torch
    nx, ny = 7, 5
    o = oracle_mod.Oracle2D(N)
    u = smooth_state(o, nx, ny, seed=N, x1=1.0, y1=0.8)
    dx, dy = 1.0 / nx, 0.8 / ny
    dt = o.dt(u, nx, ny, dx, dy)
    ref, rc, _ = o.step(u, nx, ny, dx, dy, dt)
    assert rc == 0
    ctx = make(nx, ny, N, y1=0.8)
    ud = to_dev(u)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, dt)
    torch.cuda.synchronize()
    assert rel_linf(out.cpu().numpy(), ref) < 1e-12
    assert abs(ctx.ader_compute_dt(ud) - dt) < 1e-14 * dt


@pytest.mark.parametrize("N", [1, 3, 5])
def test_fixed_iteration_step_parity(cuda, oracle_mod, N):
    import torch
    nx, ny = 6, 6
    o = oracle_mod.Oracle2D(N, fixed_iter=2)
    u = smooth_state(o, nx, ny, seed=3)
    dt = o.dt(u, nx, ny, 1 / nx, 1 / ny)
    ref, rc, _ = o.step(u, nx, ny, 1 / nx, 1 / ny, dt)
    ctx = make(nx, ny, N, picard_fixed_iter=2)
    ud = to_dev(u)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, dt)
    torch.cuda.synchronize()
    assert rel_linf(out.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("N", [1, 2, 4])
def test_solve_parity_and_conservation(cuda, oracle_mod, N):
    import torch
    nx, ny = 9, 8
    o = oracle_mod.Oracle2D(N)
    u = smooth_state(o, nx, ny, seed=7)
    ref, steps_ref, t_ref, rc = o.solve(u, nx, ny, 1 / nx, 1 / ny, t_end=0.15)
    assert rc == 0
    ctx = make(nx, ny, N)
    ud = to_dev(u)
    steps, t, rc = ctx.ader_solve(ud, t_end=0.15)
    torch.cuda.synchronize()
    got = ud.cpu().numpy()
    assert rc == 0 and steps == steps_ref and t == 0.15
    assert rel_linf(got, ref) < 1e-10
    w = o.table("w")
    tot = lambda V: np.einsum("yxklr,k,l->r", V.reshape(ny, nx, N + 1, N + 1, 4), w, w)
    np.testing.assert_allclose(tot(got), tot(u), rtol=1e-13, atol=1e-13)


def test_sine_wave_errors_equal_the_oracle(cuda, oracle_mod):
    """Sec. 2.1 2D sine wave, DG N = 3, 10^2 cells, t = 1 (936 steps): the GPU
    path's density errors equal the oracle's"""
    import torch
    N, nc = 3, 10
    o = oracle_mod.Oracle2D(N)
    X, Y = o.node_xy(nc, nc)
    one = np.ones(X.shape)
    u = conserved2(1 + 0.5 * np.sin(2 * np.pi * (X + Y)), one, one, one)
    ref, steps_ref, _, rc = o.solve(u, nc, nc, 1 / nc, 1 / nc, t_end=1.0)
    ctx = make(nc, nc, N)
    ud = to_dev(u)
    steps, t, rc = ctx.ader_solve(ud, t_end=1.0)
    torch.cuda.synchronize()
    assert rc == 0 and steps == steps_ref and t == 1.0
    exact = lambda X, Y: 1 + 0.5 * np.sin(2 * np.pi * (X + Y))
    e_gpu = oracle_mod.dg2_density_errors(o, ud.cpu().numpy(), nc, nc, exact)
    e_ref = oracle_mod.dg2_density_errors(o, ref, nc, nc, exact)
    np.testing.assert_allclose(e_gpu, e_ref, rtol=1e-8)
    assert rel_linf(ud.cpu().numpy(), ref) < 1e-10


def test_host_solve_and_stats(cuda, oracle_mod):
    N, nx, ny = 2, 5, 4
    o = oracle_mod.Oracle2D(N)
    u = smooth_state(o, nx, ny, seed=11)
    ref, steps_ref, _, _ = o.solve(u, nx, ny, 1 / nx, 1 / ny, max_steps=12)
    ctx = make(nx, ny, N)
    host = np.ascontiguousarray(u.ravel())
    steps, t, rc = ctx.ader_solve_host(host, max_steps=12)
    assert rc == 0 and steps == 12
    assert rel_linf(host, ref) < 1e-11
    st = ctx.ader_get_stats()
    assert st["steps"] == 12 and st["cells"] == 12 * nx * ny and st["max_iters"] >= 1


@pytest.mark.parametrize("nx,ny,N", [(1, 1, 3), (1, 4, 2), (6, 1, 5)])
def test_degenerate_meshes(cuda, oracle_mod, nx, ny, N):
    """one cell (its own periodic neighbour in both directions) and single rows /
    columns"""
    import torch
    o = oracle_mod.Oracle2D(N)
    u = smooth_state(o, nx, ny, seed=nx + ny)
    dx, dy = 1.0 / nx, 1.0 / ny
    dt = o.dt(u, nx, ny, dx, dy)
    ref, rc, _ = o.step(u, nx, ny, dx, dy, dt)
    ctx = make(nx, ny, N)
    ud = to_dev(u)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, dt)
    torch.cuda.synchronize()
    assert rc == 0 and rel_linf(out.cpu().numpy(), ref) < 1e-12


def test_full_size_n5_320x320_sampled(cuda, oracle_mod):
    """DG N = 5 on 320 x 320 cells (the size the 2D throughput line times), one
    step with the time step taken on the device: the CFL step equals the
    oracle's and sampled cells (the four corners, wrap-around edges, random
    interior) equal the oracle's per-cell step."""
    import torch
    N, nc = 5, 320
    o = oracle_mod.Oracle2D(N)
    u = smooth_state(o, nc, nc, seed=21)
    h = 1.0 / nc
    ctx = make(nc, nc, N)
    ud = to_dev(u)
    out = torch.empty_like(ud)
    dt_dev = ctx.ader_compute_dt(ud)
    ctx.ader_step(ud, out, 0.0)  # CFL step on the device
    torch.cuda.synchronize()
    dt = o.dt(u, nc, nc, h, h)
    assert abs(dt_dev - dt) <= 1e-14 * dt
    last = nc * nc - 1
    cells = np.unique(np.concatenate([[0, nc - 1, last - nc + 1, last, nc, 2 * nc - 1],
                                      np.random.default_rng(2).integers(0, nc * nc, 40)]))
    sel, rc = o.step_cells(u, nc, nc, h, h, dt, cells)
    assert rc == 0
    got = out.cpu().numpy().reshape(nc * nc, N + 1, N + 1, 4)[cells]
    assert rel_linf(got, sel) < 1e-12


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_large_block_shapes_sampled(cuda, oracle_mod, N):
    """100 x 100 cells: enough for the launchers to take the large block shapes of
    the predictor and the update (the ragged meshes above take the small ones);
    one device-CFL step checked on sampled cells against the oracle's per-cell
    step."""
    import torch
    nc = 100
    o = oracle_mod.Oracle2D(N)
    u = smooth_state(o, nc, nc, seed=40 + N)
    h = 1.0 / nc
    ctx = make(nc, nc, N)
    ud = to_dev(u)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, 0.0)
    torch.cuda.synchronize()
    dt = o.dt(u, nc, nc, h, h)
    cells = np.unique(np.concatenate([[0, nc - 1, nc * nc - nc, nc * nc - 1],
                                      np.random.default_rng(N).integers(0, nc * nc, 40)]))
    sel, rc = o.step_cells(u, nc, nc, h, h, dt, cells)
    assert rc == 0
    got = out.cpu().numpy().reshape(nc * nc, N + 1, N + 1, 4)[cells]
    assert rel_linf(got, sel) < 1e-12
