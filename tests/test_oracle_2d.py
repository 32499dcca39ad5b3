"""Pins of the oracle's 2D Euler ADER-DG scheme (Sec. 1.1 tensor-product
predictor, Sec. 1.2 corrector with x- and y-faces, Sec. 1.5 time step with
d = 2) and of the 2D sine-wave advection problem of Sec. 2.1.

Independent pins: data uniform along y with v = 0 (or along x with u = 0) give
the 1D oracle's step row by row (column by column), which the 2D code reaches
through its own loops; the converged predictor solves the Kronecker-assembled
system K^tau q + K^xi f + K^eta g = F^0 u built from Upsilon, Lambda, Xi (which
fixes which index each contraction runs over); constant states are fixed
points; periodic steps conserve; the time step follows the d = 2 rule; the sine
wave converges at order N+1, with errors within a factor 3 of the paper's Table
conv_orders_pde_2d (tests/golden/conv_orders_pde_2d.txt: the paper does not
name its Riemann solver; with Rusanov the low-degree errors are larger)."""
import os

import numpy as np
import pytest

GAMMA = 1.4
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "conv_orders_pde_2d.txt")


def conserved2(rho, u, v, p, g=GAMMA):
    return np.stack([rho, rho * u, rho * v, p / (g - 1) + 0.5 * rho * (u * u + v * v)], -1)


def sine_state(o, nc):
    X, Y = o.node_xy(nc, nc)
    one = np.ones(X.shape)
    return conserved2(1 + 0.5 * np.sin(2 * np.pi * (X + Y)), one, one, one)


def paper_table():
    rows = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            N, nc, l1, l2, li = line.split()
            rows[(int(N), int(nc))] = (float(l1), float(l2), float(li))
    return rows


def test_flux_closed_forms(oracle_mod):
    o = oracle_mod.Oracle2D(1)
    U = conserved2(np.array(1.3), np.array(0.4), np.array(-0.7), np.array(2.0))
    F, G = o.flux(U)
    rho, u, v, p, E = 1.3, 0.4, -0.7, 2.0, U[3]
    np.testing.assert_allclose(F, [rho * u, rho * u * u + p, rho * u * v, (E + p) * u], rtol=1e-15)
    np.testing.assert_allclose(G, [rho * v, rho * u * v, rho * v * v + p, (E + p) * v], rtol=1e-15)
    np.testing.assert_allclose(o.rusanov(0, U, U), F, rtol=1e-15)
    np.testing.assert_allclose(o.rusanov(1, U, U), G, rtol=1e-15)


def _row_state(o1, nx, seed):
    rng = np.random.default_rng(seed)
    x = o1.node_x(nx)
    a = rng.uniform(0.05, 0.2, 3)
    rho = 1 + a[0] * np.sin(2 * np.pi * x + 0.3)
    u = 0.5 + a[1] * np.cos(2 * np.pi * x)
    p = 1 + a[2] * np.sin(4 * np.pi * x)
    return rho, u, p


@pytest.mark.parametrize("N", range(0, 5))
def test_uniform_along_one_direction_is_the_1d_scheme(oracle_mod, N):
    """y-uniform data with v = 0 (and x-uniform data with u = 0) step exactly as
    the 1D scheme does along the other direction"""
    o1 = oracle_mod.Oracle(N)
    o2 = oracle_mod.Oracle2D(N)
    n, nx, ny = N + 1, 7, 3
    rho, u, p = _row_state(o1, nx, N)
    u1 = np.stack([rho, rho * u, p / (GAMMA - 1) + 0.5 * rho * u * u], -1)  # [nx][n][3]
    dx, dy = 1.0 / nx, 0.37
    dt = 0.3 * o1.dg_dt(u1, dx)
    ref = o1.dg_step(u1, dx, dt)[0].reshape(nx, n, 3)
    # along x: U[iy][ix][k1][k2] = state(ix, k1)
    U = np.zeros((ny, nx, n, n, 4))
    U[..., 0] = rho[None, :, :, None]
    U[..., 1] = (rho * u)[None, :, :, None]
    U[..., 3] = u1[None, :, :, None, 2]
    out, rc, _ = o2.step(U, nx, ny, dx, dy, dt)
    out = out.reshape(ny, nx, n, n, 4)
    assert rc == 0
    got = out[..., [0, 1, 3]]
    scale = np.abs(ref).max()
    assert np.abs(got - ref[None, :, :, None, :]).max() < 1e-13 * scale
    assert np.abs(out[..., 2]).max() < 1e-13 * scale
    # along y: U[iy][ix][k1][k2] = state(iy, k2), momentum in m_y
    V = np.zeros((nx, 2, n, n, 4))
    V[..., 0] = rho[:, None, None, :]
    V[..., 2] = (rho * u)[:, None, None, :]
    V[..., 3] = u1[:, None, None, :, 2]
    out, rc, _ = o2.step(V, 2, nx, 0.37, dx, dt)
    out = out.reshape(nx, 2, n, n, 4)
    assert rc == 0
    got = out[..., [0, 2, 3]]
    assert np.abs(got - ref[:, None, None, :, :]).max() < 1e-13 * scale
    assert np.abs(out[..., 1]).max() < 1e-13 * scale


@pytest.mark.parametrize("N", [1, 2, 3])
def test_predictor_solves_the_kronecker_system(oracle_mod, N):
    """K^tau q + K^xi (dt/dx) F(q) + K^eta (dt/dy) G(q) = F^0 u with K^tau =
    Upsilon (x) Lambda (x) Lambda, K^xi = Lambda (x) Xi (x) Lambda, K^eta = Lambda
    (x) Lambda (x) Xi, F^0 = psi (x) Lambda (x) Lambda (Sec. 1.1)"""
    o = oracle_mod.Oracle2D(N, tol=1e-15, max_iter=200)
    n = N + 1
    rng = np.random.default_rng(10 + N)
    rho = 1 + 0.2 * rng.uniform(-1, 1, (n, n))
    u = 0.6 + 0.2 * rng.uniform(-1, 1, (n, n))
    v = -0.4 + 0.2 * rng.uniform(-1, 1, (n, n))
    p = 1 + 0.2 * rng.uniform(-1, 1, (n, n))
    U = conserved2(rho, u, v, p)
    lx, ly = 0.06, 0.045
    q, it, rc = o.predict_cell(U, lx, ly)
    assert rc == 0
    Ups, Lam, Xi, psi0 = (o.table(t) for t in ("ups", "lam", "xi_m", "psi0"))
    F = np.array([o.flux(x)[0] for x in q.reshape(-1, 4)]) * lx
    G = np.array([o.flux(x)[1] for x in q.reshape(-1, 4)]) * ly
    K = lambda a, b, c: np.kron(np.kron(a, b), c)
    res = (K(Ups, Lam, Lam) @ q.reshape(-1, 4) + K(Lam, Xi, Lam) @ F + K(Lam, Lam, Xi) @ G
           - K(psi0[:, None], Lam, Lam) @ U.reshape(-1, 4))
    assert np.abs(res).max() < 1e-13


def test_constant_state_and_conservation(oracle_mod):
    o = oracle_mod.Oracle2D(3)
    nx, ny = 5, 4
    X, Y = o.node_xy(nx, ny)
    one = np.ones(X.shape)
    U = conserved2(0.8 * one, 0.3 * one, -0.2 * one, 1.1 * one)
    out, rc, _ = o.step(U, nx, ny, 0.2, 0.25, 0.004)
    assert rc == 0
    np.testing.assert_allclose(out.reshape(U.shape), U, rtol=0, atol=1e-14)
    U = conserved2(1 + 0.3 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y), 0.5 + 0 * X,
                   0.2 * np.sin(2 * np.pi * Y), 1 + 0.1 * np.cos(2 * np.pi * (X - Y)))
    dt = o.dt(U, nx, ny, 0.2, 0.25)
    out, rc, _ = o.step(U, nx, ny, 0.2, 0.25, dt)
    w = o.table("w")
    tot = lambda V: np.einsum("yxklr,k,l->r", V.reshape(U.shape), w, w)
    assert rc == 0
    np.testing.assert_allclose(tot(out), tot(U), rtol=1e-14, atol=1e-14)


def test_time_step_rule(oracle_mod):
    """dt = CFL / (2 (2N+1)) min(dx / (|u| + c), dy / (|v| + c)) on a uniform state"""
    N = 2
    o = oracle_mod.Oracle2D(N, cfl=0.4)
    X, Y = o.node_xy(3, 2)
    one = np.ones(X.shape)
    rho, u, v, p = 1.2, 0.5, -1.5, 0.9
    U = conserved2(rho * one, u * one, v * one, p * one)
    c = np.sqrt(GAMMA * p / rho)
    dx, dy = 0.1, 0.3
    exact = 0.4 / (2 * (2 * N + 1)) * min(dx / (abs(u) + c), dy / (abs(v) + c))
    assert abs(o.dt(U, 3, 2, dx, dy) - exact) < 1e-15 * exact


@pytest.mark.parametrize("N,cells,lo,hi", [(1, (20, 25), 1.85, 2.3), (2, (15, 20), 2.6, 3.3),
                                           (3, (10, 15), 3.7, 4.4)])
def test_sine_wave_orders_and_paper_magnitudes(oracle_mod, N, cells, lo, hi):
    o = oracle_mod.Oracle2D(N)
    table = paper_table()
    exact = lambda X, Y: 1 + 0.5 * np.sin(2 * np.pi * (X + Y))
    errs = []
    for nc in cells:
        out, steps, t, rc = o.solve(sine_state(o, nc), nc, nc, 1.0 / nc, 1.0 / nc, t_end=1.0)
        assert rc == 0 and t == 1.0
        e = oracle_mod.dg2_density_errors(o, out, nc, nc, exact)
        errs.append(e)
        ratio = np.array(e) / np.array(table[(N, nc)])
        assert (ratio > 0.8).all() and (ratio < 3.0).all(), (N, nc, e, table[(N, nc)])
    orders = np.log(np.array(errs[0]) / np.array(errs[1])) / np.log(cells[1] / cells[0])
    assert (orders > lo).all() and (orders < hi).all(), orders


def test_step_cells_equals_the_full_step(oracle_mod):
    N, nx, ny = 3, 5, 4
    o = oracle_mod.Oracle2D(N)
    X, Y = o.node_xy(nx, ny)
    one = np.ones(X.shape)
    u = conserved2(1 + 0.2 * np.sin(2 * np.pi * (X + 2 * Y)), 0.5 * one, -0.3 * one, one)
    dt = o.dt(u, nx, ny, 0.2, 0.25)
    full, rc, _ = o.step(u, nx, ny, 0.2, 0.25, dt)
    cells = [0, 4, 7, 19]
    sel, rc2 = o.step_cells(u, nx, ny, 0.2, 0.25, dt, cells)
    assert rc == 0 and rc2 == 0
    np.testing.assert_array_equal(sel, full.reshape(ny * nx, N + 1, N + 1, 4)[cells])
