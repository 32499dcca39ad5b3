"""The CFL maximum lambda_max of the time step (Sec. 1.5) taken inside the time
loop -- the interface / update kernels bound every subcell's wave speed in FP32
and re-evaluate in FP64 only the subcells that can hold the maximum -- equals
the oracle's FP64 maximum over every subcell, on states built to stress that
screen: speeds equal to within the FP32 error (amplitude 1e-7), a little above
it (1e-5), well above it (1e-3), and a high-Mach region whose FP32 pressure
cannot be trusted (p / E ~ 1e-4).

The time loop's second step size is t2 - t1 (two solves from the same state,
one and two steps); the oracle computes the step size of the GPU's state after
one step.  A subcell wrongly left out shifts lambda_max by about the FP32
error, 1e-7 .. 1e-5 relative, far above the 1e-14 bar."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

GAMMA = 1.4
CASES = ["1e-7", "1e-5", "1e-3", "high-mach"]


def prim_1d(x, case, seed):
    g = np.random.default_rng(seed)
    ph = g.uniform(0, 2 * np.pi, 3)
    if case == "high-mach":
        rho = 1 + 0.1 * np.sin(2 * np.pi * x + ph[0])
        u = 0.3 + 20.0 * np.exp(-((x - 0.5) / 0.05) ** 2)
        p = 1e-2 * (1 + 0.1 * np.cos(2 * np.pi * x + ph[1]))
    else:
        eps = float(case)
        rho = 1 + eps * np.sin(2 * np.pi * x + ph[0])
        u = 0.3 + eps * np.cos(2 * np.pi * x + ph[1])
        p = 1 + eps * np.sin(4 * np.pi * x + ph[2])
    return rho, u, p


def to_dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda")


def second_step_dt(ctx, u0):
    """(state after one step, the loop's second step size)"""
    a, b = u0.clone(), u0.clone()
    s1, t1, rc1 = ctx.ader_solve(a, max_steps=1)
    s2, t2, rc2 = ctx.ader_solve(b, max_steps=2)
    assert (s1, s2, rc1, rc2) == (1, 2, 0, 0)
    return a.cpu().numpy(), t2 - t1


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_dg_1d(cuda, oracle_mod, N, case):
    from paper_2409_12483_gb300 import Context
    nc = 1000
    o = oracle_mod.Oracle(N)
    u = W.conserved(*prim_1d(o.node_x(nc), case, N))
    ctx = Context(nc, N, "dg")
    u1, dt2 = second_step_dt(ctx, to_dev(u))
    ref = o.dg_dt(u1, 1.0 / nc)
    assert abs(dt2 - ref) <= 1e-14 * ref


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("N", [1, 5])
def test_dg_1d_nodal_mode(cuda, oracle_mod, N, case):
    """the same screens over the nodal values (cfl_mode 1)"""
    from paper_2409_12483_gb300 import Context
    nc = 1000
    o = oracle_mod.Oracle(N)
    o.set(cfl_mode=1)
    u = W.conserved(*prim_1d(o.node_x(nc), case, N + 3))
    ctx = Context(nc, N, "dg", cfl_mode="nodal")
    u1, dt2 = second_step_dt(ctx, to_dev(u))
    ref = o.dg_dt(u1, 1.0 / nc)
    assert abs(dt2 - ref) <= 1e-14 * ref


@pytest.mark.parametrize("case", CASES)
def test_weno_1d(cuda, oracle_mod, case):
    from paper_2409_12483_gb300 import Context
    nc, N = 1000, 4
    o = oracle_mod.Oracle(N)
    xc = (np.arange(nc) + 0.5) / nc
    v = W.conserved(*prim_1d(xc, case, 11))
    ctx = Context(nc, N, "fv")
    v1, dt2 = second_step_dt(ctx, to_dev(v))
    ref = o.fv_dt(v1, 1.0 / nc)
    assert abs(dt2 - ref) <= 1e-14 * ref


@pytest.mark.parametrize("case", CASES)
def test_dg_1d_limiter(cuda, oracle_mod, case):
    from paper_2409_12483_gb300 import Context
    nc, N = 1000, 3
    o = oracle_mod.Oracle(N)
    u = W.conserved(*prim_1d(o.node_x(nc), case, 12))
    ctx = Context(nc, N, "dg", limiter=1)
    u1, dt2 = second_step_dt(ctx, to_dev(u))
    ref = o.dg_dt(u1, 1.0 / nc)
    assert abs(dt2 - ref) <= 1e-14 * ref


def cons2(rho, u, v, p):
    return np.stack([rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)], -1)


def cons3(rho, u, v, w, p):
    return np.stack([rho, rho * u, rho * v, rho * w,
                     p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v + w * w)], -1)


@pytest.mark.parametrize("case", CASES[:3])  # a Mach-170 region needs the 1D mesh's resolution
@pytest.mark.parametrize("N", [1, 3])
def test_dg_2d(cuda, oracle_mod, N, case):
    from paper_2409_12483_gb300 import Context2D
    nx, ny = 24, 20
    o = oracle_mod.Oracle2D(N)
    X, Y = o.node_xy(nx, ny)
    rho, u, p = prim_1d(X, case, N)
    _, v, _ = prim_1d(Y, case, N + 7)
    u0 = cons2(rho, u, v - 0.5, p)
    ctx = Context2D(nx, ny, N)
    ud = to_dev(u0)
    ref0 = o.dt(u0, nx, ny, 1.0 / nx, 1.0 / ny)
    assert abs(ctx.ader_compute_dt(ud) - ref0) <= 1e-14 * ref0  # the first step's kernel
    u1, dt2 = second_step_dt(ctx, ud)
    ref = o.dt(u1, nx, ny, 1.0 / nx, 1.0 / ny)
    assert abs(dt2 - ref) <= 1e-14 * ref


@pytest.mark.parametrize("case", CASES[:3])
@pytest.mark.parametrize("N", [1, 2])
def test_dg_3d(cuda, oracle_mod, N, case):
    """N = 1 projects in FP32 through all three passes, N = 2 only the last"""
    from paper_2409_12483_gb300 import Context3D
    dims, box = (8, 6, 5), (1.0, 1.0, 1.0)
    h = tuple(b / d for b, d in zip(box, dims))
    o = oracle_mod.Oracle3D(N)
    X, Y, Z = o.node_xyz(*dims, box=box)
    rho, u, p = prim_1d(X, case, N)
    _, v, _ = prim_1d(Y, case, N + 7)
    _, w, _ = prim_1d(Z, case, N + 9)
    u0 = cons3(rho, u, v - 0.2, w - 0.1, p)
    ctx = Context3D(*dims, N, box=box)
    ud = to_dev(u0)
    ref0 = o.dt(u0, dims, h)
    assert abs(ctx.ader_compute_dt(ud) - ref0) <= 1e-14 * ref0  # the first step's kernel
    u1, dt2 = second_step_dt(ctx, ud)
    ref = o.dt(u1, dims, h)
    assert abs(dt2 - ref) <= 1e-14 * ref
