"""GPU parity of the 3D Euler ADER-DG path (ader_init_3d, degrees 0..7 (N = 7:
the two-CTA cluster predictor):
tensor-product predictor along xi, eta, zeta of Sec. 1.1, x/y/z faces of Sec.
1.2, d = 3 time step of Sec. 1.5) against the oracle's ob3_* family.  Bar:
1e-12 relative L-inf per step, 1e-10 after a solve."""
import numpy as np
import pytest

from conftest import rel_linf

pytestmark = pytest.mark.gpu

GAMMA = 1.4


def conserved3(rho, u, v, w, p, g=GAMMA):
    return np.stack([rho, rho * u, rho * v, rho * w,
                     p / (g - 1) + 0.5 * rho * (u * u + v * v + w * w)], -1)


def smooth_state(o, dims, box, seed=0):
    X, Y, Z = o.node_xyz(*dims, box=box)
    X, Y, Z = X / box[0], Y / box[1], Z / box[2]
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.05, 0.15, 5)
    rho = 1 + a[0] * np.sin(2 * np.pi * (X + 2 * Y - Z)) + a[1] * np.cos(2 * np.pi * Z)
    u = 0.5 + a[2] * np.sin(2 * np.pi * Y)
    v = -0.3 + a[3] * np.cos(2 * np.pi * (X - Z))
    w = 0.2 + a[4] * np.sin(2 * np.pi * X)
    p = 1 + 0.1 * np.sin(2 * np.pi * (X + Y + Z))
    return conserved3(rho, u, v, w, p)


def make(dims, N, box=(1.0, 1.0, 1.0), **kw):
    from paper_2409_12483_gb300 import Context3D
    return Context3D(*dims, N, box=box, **kw)


def to_dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("N", range(0, 8))
def test_step_parity(cuda, oracle_mod, N):
    """one step on smooth data, a ragged mesh (partial blocks), unequal spacings"""
    import torch
    dims, box = (5, 3, 2), (1.0, 0.9, 0.7)
    h = tuple(b / d for b, d in zip(box, dims))
    o = oracle_mod.Oracle3D(N)
    u = smooth_state(o, dims, box, seed=N)
    dt = o.dt(u, dims, h)
    ref, rc, _ = o.step(u, dims, h, dt)
    assert rc == 0
    ctx = make(dims, N, box)
    ud = to_dev(u)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, dt)
    torch.cuda.synchronize()
    assert rel_linf(out.cpu().numpy(), ref) < 1e-12
    assert abs(ctx.ader_compute_dt(ud) - dt) < 1e-14 * dt


@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_fixed_iteration_step_parity(cuda, oracle_mod, N):
    import torch
    dims, box = (3, 3, 3), (1.0, 1.0, 1.0)
    h = (1 / 3,) * 3
    o = oracle_mod.Oracle3D(N, fixed_iter=2)
    u = smooth_state(o, dims, box, seed=5)
    dt = o.dt(u, dims, h)
    ref, rc, _ = o.step(u, dims, h, dt)
    ctx = make(dims, N, picard_fixed_iter=2)
    ud = to_dev(u)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, dt)
    torch.cuda.synchronize()
    assert rel_linf(out.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("N", [1, 2, 3])
def test_solve_parity_and_conservation(cuda, oracle_mod, N):
    import torch
    dims, box = (4, 3, 3), (1.0, 1.0, 1.0)
    h = tuple(b / d for b, d in zip(box, dims))
    o = oracle_mod.Oracle3D(N)
    u = smooth_state(o, dims, box, seed=9)
    ref, steps_ref, t_ref, rc = o.solve(u, dims, h, t_end=0.05)
    assert rc == 0
    ctx = make(dims, N)
    ud = to_dev(u)
    steps, t, rc = ctx.ader_solve(ud, t_end=0.05)
    torch.cuda.synchronize()
    got = ud.cpu().numpy()
    assert rc == 0 and steps == steps_ref and t == 0.05
    assert rel_linf(got, ref) < 1e-10
    wq = o.table("w")
    n = N + 1
    tot = lambda V: np.einsum("zyxabcr,a,b,c->r", V.reshape(dims[::-1] + (n, n, n, 5)), wq, wq, wq)
    np.testing.assert_allclose(tot(got), tot(u), rtol=1e-13, atol=1e-13)


def test_sine_wave_errors_equal_the_oracle(cuda, oracle_mod):
    """Sec. 2.1 3D sine wave (velocity (1, 1, 1)), DG N = 2, 5^3 cells, t = 1"""
    import torch
    N, nc = 2, 5
    o = oracle_mod.Oracle3D(N)
    X, Y, Z = o.node_xyz(nc, nc, nc)
    one = np.ones(X.shape)
    u = conserved3(1 + 0.5 * np.sin(2 * np.pi * (X + Y + Z)), one, one, one, one)
    ref, steps_ref, _, rc = o.solve(u, (nc,) * 3, (1 / nc,) * 3, t_end=1.0)
    ctx = make((nc,) * 3, N)
    ud = to_dev(u)
    steps, t, rc = ctx.ader_solve(ud, t_end=1.0)
    torch.cuda.synchronize()
    assert rc == 0 and steps == steps_ref and t == 1.0
    exact = lambda X, Y, Z: 1 + 0.5 * np.sin(2 * np.pi * (X + Y + Z))
    e_gpu = oracle_mod.dg3_density_errors(o, ud.cpu().numpy(), (nc,) * 3, exact)
    e_ref = oracle_mod.dg3_density_errors(o, ref, (nc,) * 3, exact)
    np.testing.assert_allclose(e_gpu, e_ref, rtol=1e-8)


@pytest.mark.parametrize("dims,N", [((1, 1, 1), 2), ((1, 2, 3), 1), ((4, 1, 1), 4), ((2, 1, 2), 6),
                                    ((1, 1, 1), 7), ((3, 1, 2), 7)])
def test_degenerate_meshes(cuda, oracle_mod, dims, N):
    """one cell (its own periodic neighbour in every direction) and single lines"""
    import torch
    box = (1.0, 1.0, 1.0)
    h = tuple(b / d for b, d in zip(box, dims))
    o = oracle_mod.Oracle3D(N)
    u = smooth_state(o, dims, box, seed=sum(dims))
    dt = o.dt(u, dims, h)
    ref, rc, _ = o.step(u, dims, h, dt)
    ctx = make(dims, N)
    ud = to_dev(u)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, dt)
    torch.cuda.synchronize()
    assert rc == 0 and rel_linf(out.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("N,nc", [(3, 64), (6, 16), (7, 12)])
def test_full_size_sampled(cuda, oracle_mod, N, nc):
    """DG N = 3 on 64^3, N = 6 on 16^3 and N = 7 on 12^3 cells (sizes the 3D throughput lines
    time), one step with the time step taken on the device: the CFL step equals
    the oracle's and sampled cells (corners, wrap-around faces, random interior)
    equal the oracle's per-cell step."""
    import torch
    dims, box = (nc,) * 3, (1.0, 1.0, 1.0)
    h = (1.0 / nc,) * 3
    o = oracle_mod.Oracle3D(N)
    u = smooth_state(o, dims, box, seed=N + nc)
    ctx = make(dims, N)
    ud = to_dev(u)
    out = torch.empty_like(ud)
    dt_dev = ctx.ader_compute_dt(ud)
    ctx.ader_step(ud, out, 0.0)  # CFL step on the device
    torch.cuda.synchronize()
    dt = o.dt(u, dims, h)
    assert abs(dt_dev - dt) <= 1e-14 * dt
    total = nc ** 3
    corners = [0, nc - 1, nc * (nc - 1), nc * nc - 1, total - nc * nc, total - 1]
    cells = np.unique(np.concatenate([corners,
                                      np.random.default_rng(3).integers(0, total, 24)]))
    sel, rc = o.step_cells(u, dims, h, dt, cells)
    assert rc == 0
    got = out.cpu().numpy().reshape(total, N + 1, N + 1, N + 1, 5)[cells]
    assert rel_linf(got, sel) < 1e-12


@pytest.mark.parametrize("N", [1, 2, 3])
def test_large_block_shapes_sampled(cuda, oracle_mod, N):
    """18^3 cells: enough for the launchers to take the large block shapes of the
    predictor and the update (the ragged meshes above take the small ones); one
    device-CFL step checked on sampled cells against the oracle's per-cell step."""
    import torch
    nc = 18
    dims, box, h = (nc,) * 3, (1.0, 1.0, 1.0), (1.0 / nc,) * 3
    o = oracle_mod.Oracle3D(N)
    u = smooth_state(o, dims, box, seed=50 + N)
    ctx = make(dims, N)
    ud = to_dev(u)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, 0.0)
    torch.cuda.synchronize()
    dt = o.dt(u, dims, h)
    total = nc ** 3
    cells = np.unique(np.concatenate([[0, total - 1, nc * nc - 1, total - nc * nc],
                                      np.random.default_rng(N).integers(0, total, 24)]))
    sel, rc = o.step_cells(u, dims, h, dt, cells)
    assert rc == 0
    got = out.cpu().numpy().reshape(total, N + 1, N + 1, N + 1, 5)[cells]
    assert rel_linf(got, sel) < 1e-12


def test_n7_solve_parity_and_conservation(cuda, oracle_mod):
    """DG N = 7 (the cluster predictor) through the device time loop: a short
    solve against the oracle's, and the conserved totals to round-off."""
    import torch
    N, dims, box = 7, (2, 2, 2), (1.0, 1.0, 1.0)
    h = (0.5,) * 3
    o = oracle_mod.Oracle3D(N)
    u = smooth_state(o, dims, box, seed=77)
    ref, steps_ref, t_ref, rc = o.solve(u, dims, h, t_end=0.01)
    assert rc == 0
    ctx = make(dims, N)
    ud = to_dev(u)
    steps, t, rc = ctx.ader_solve(ud, t_end=0.01)
    torch.cuda.synchronize()
    got = ud.cpu().numpy()
    assert rc == 0 and steps == steps_ref and t == 0.01
    assert rel_linf(got, ref) < 1e-10
    wq = o.table("w")
    n = N + 1
    tot = lambda V: np.einsum("zyxabcr,a,b,c->r", V.reshape(dims[::-1] + (n, n, n, 5)), wq, wq, wq)
    np.testing.assert_allclose(tot(got), tot(u), rtol=1e-13, atol=1e-13)
