"""Pins of the oracle's 3D Euler ADER-DG scheme (Sec. 1.1 tensor-product
predictor with L^xi, L^eta, L^zeta; Sec. 1.2 corrector with x-, y- and
z-faces; Sec. 1.5 time step with d = 3).

Independent pins: data uniform along z with w = 0, along y with v = 0 and along
x with u = 0 step as the 2D oracle does on the remaining plane (so each of the
three directions is checked against the pinned 2D scheme, through the 3D code's
own loops); the converged predictor solves the Kronecker-assembled system
K^tau q + K^xi f + K^eta g + K^zeta h = F^0 u (Upsilon, Lambda, Xi); constant
states are fixed points; periodic steps conserve; the time step follows the
d = 3 rule."""
import numpy as np
import pytest

GAMMA = 1.4


def conserved3(rho, u, v, w, p, g=GAMMA):
    return np.stack([rho, rho * u, rho * v, rho * w,
                     p / (g - 1) + 0.5 * rho * (u * u + v * v + w * w)], -1)


def test_flux_closed_forms(oracle_mod):
    o = oracle_mod.Oracle3D(1)
    rho, u, v, w, p = 1.3, 0.4, -0.7, 0.2, 2.0
    U = conserved3(*map(np.array, (rho, u, v, w, p)))
    E = U[4]
    F = o.flux(U)
    vel = (u, v, w)
    for d in range(3):
        expect = [rho * vel[d]] + [rho * vel[c] * vel[d] + (p if c == d else 0) for c in range(3)]
        expect.append((E + p) * vel[d])
        np.testing.assert_allclose(F[d], expect, rtol=1e-15, atol=1e-15)
        np.testing.assert_allclose(o.rusanov(d, U, U), F[d], rtol=1e-15, atol=1e-15)


def _plane_state(o2, nx, ny, seed):
    """a smooth 2D state [ny][nx][n][n][4] with u, v != 0"""
    X, Y = o2.node_xy(nx, ny)
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.05, 0.15, 4)
    rho = 1 + a[0] * np.sin(2 * np.pi * (X + 2 * Y))
    u = 0.5 + a[1] * np.cos(2 * np.pi * X)
    v = -0.3 + a[2] * np.sin(2 * np.pi * Y)
    p = 1 + a[3] * np.cos(2 * np.pi * (X - Y))
    return np.stack([rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)], -1)


@pytest.mark.parametrize("N", range(0, 4))
def test_uniform_along_one_direction_is_the_2d_scheme(oracle_mod, N):
    o2 = oracle_mod.Oracle2D(N)
    o3 = oracle_mod.Oracle3D(N)
    n = N + 1
    a, b, c = 4, 3, 2  # cells along the two plane directions and the uniform one
    U2 = _plane_state(o2, a, b, N)  # [b][a][n][n][4]
    ha, hb, hc = 0.25, 0.31, 0.7
    dt = 0.3 * o2.dt(U2, a, b, ha, hb)
    ref, rc, _ = o2.step(U2, a, b, ha, hb, dt)
    ref = ref.reshape(b, a, n, n, 4)
    scale = np.abs(ref).max()
    rho, m1, m2, E = (U2[..., i] for i in range(4))
    zero = np.zeros_like(rho)
    # (plane axes, uniform axis) -> 3D arrays [nz][ny][nx][k1][k2][k3]
    cases = {
        "z": (lambda A: np.broadcast_to(A[None, :, :, :, :, None], (c, b, a, n, n, n)),
              (a, b, c), (ha, hb, hc), (0, 1, 2, 3, 4), (m1, m2, zero)),
        "y": (lambda A: np.broadcast_to(A[:, None, :, :, None, :], (b, c, a, n, n, n)),
              (a, c, b), (ha, hc, hb), (0, 1, 3, 2, 4), (m1, zero, m2)),
        "x": (lambda A: np.broadcast_to(A[:, :, None, None, :, :], (b, a, c, n, n, n)),
              (c, a, b), (hc, ha, hb), (0, 2, 3, 1, 4), (zero, m1, m2)),
    }
    for axis, (ext, dims, h, order, moms) in cases.items():
        U3 = np.stack([ext(rho), ext(moms[0]), ext(moms[1]), ext(moms[2]), ext(E)], -1)
        out, rc3, _ = o3.step(U3, dims, h, dt)
        assert rc3 == 0
        out = out.reshape(U3.shape)
        # map the 2D variables (rho, m_plane1, m_plane2, E) to their 3D slots
        slots = {"z": (0, 1, 2, 4), "y": (0, 1, 3, 4), "x": (0, 2, 3, 4)}[axis]
        normal = ({0, 1, 2, 3, 4} - set(slots)).pop()
        for i, s3 in enumerate(slots):
            assert np.abs(out[..., s3] - ext(ref[..., i])).max() < 1e-13 * scale, (axis, i)
        assert np.abs(out[..., normal]).max() < 1e-13 * scale, axis


@pytest.mark.parametrize("N", [1, 2])
def test_predictor_solves_the_kronecker_system(oracle_mod, N):
    o = oracle_mod.Oracle3D(N, tol=1e-15, max_iter=200)
    n = N + 1
    rng = np.random.default_rng(20 + N)
    sh = (n, n, n)
    U = conserved3(1 + 0.2 * rng.uniform(-1, 1, sh), 0.5 + 0.2 * rng.uniform(-1, 1, sh),
                   -0.3 + 0.2 * rng.uniform(-1, 1, sh), 0.2 + 0.2 * rng.uniform(-1, 1, sh),
                   1 + 0.2 * rng.uniform(-1, 1, sh))
    lam = (0.05, 0.04, 0.035)
    q, it, rc = o.predict_cell(U, *lam)
    assert rc == 0
    Ups, Lam, Xi, psi0 = (o.table(t) for t in ("ups", "lam", "xi_m", "psi0"))
    F = np.array([o.flux(x) for x in q.reshape(-1, 5)])  # [node][d][5]
    K = lambda *m: np.kron(np.kron(np.kron(m[0], m[1]), m[2]), m[3])
    res = (K(Ups, Lam, Lam, Lam) @ q.reshape(-1, 5)
           + K(Lam, Xi, Lam, Lam) @ (lam[0] * F[:, 0]) + K(Lam, Lam, Xi, Lam) @ (lam[1] * F[:, 1])
           + K(Lam, Lam, Lam, Xi) @ (lam[2] * F[:, 2])
           - K(psi0[:, None], Lam, Lam, Lam) @ U.reshape(-1, 5))
    assert np.abs(res).max() < 1e-13


def test_constant_state_conservation_and_time_step(oracle_mod):
    N = 2
    o = oracle_mod.Oracle3D(N, cfl=0.4)
    dims, h = (3, 2, 2), (1 / 3, 0.5, 0.5)
    X, Y, Z = o.node_xyz(*dims)
    one = np.ones(X.shape)
    rho, u, v, w, p = 0.9, 0.3, -0.6, 0.1, 1.2
    U = conserved3(rho * one, u * one, v * one, w * one, p * one)
    out, rc, _ = o.step(U, dims, h, 0.003)
    assert rc == 0
    np.testing.assert_allclose(out.reshape(U.shape), U, rtol=0, atol=1e-14)
    c = np.sqrt(GAMMA * p / rho)
    exact = 0.4 / (3 * (2 * N + 1)) * min(h[0] / (abs(u) + c), h[1] / (abs(v) + c), h[2] / (abs(w) + c))
    assert abs(o.dt(U, dims, h) - exact) < 1e-15 * exact
    U = conserved3(1 + 0.3 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Z), 0.5 * one,
                   0.2 * np.sin(2 * np.pi * Y), -0.1 * one, 1 + 0.1 * np.cos(2 * np.pi * (X - Y)))
    out, rc, _ = o.step(U, dims, h, o.dt(U, dims, h))
    wq = o.table("w")
    tot = lambda V: np.einsum("zyxabcr,a,b,c->r", V.reshape(U.shape), wq, wq, wq)
    assert rc == 0
    np.testing.assert_allclose(tot(out), tot(U), rtol=1e-14, atol=1e-14)


def test_step_cells_equals_the_full_step(oracle_mod):
    N, dims, h = 2, (3, 4, 2), (1 / 3, 0.25, 0.5)
    o = oracle_mod.Oracle3D(N)
    X, Y, Z = o.node_xyz(*dims)
    one = np.ones(X.shape)
    u = conserved3(1 + 0.2 * np.sin(2 * np.pi * (X + Y - Z)), 0.4 * one, -0.2 * one, 0.1 * one, one)
    dt = o.dt(u, dims, h)
    full, rc, _ = o.step(u, dims, h, dt)
    cells = [0, 5, 11, 23]
    sel, rc2 = o.step_cells(u, dims, h, dt, cells)
    assert rc == 0 and rc2 == 0
    np.testing.assert_array_equal(sel, full.reshape(24, N + 1, N + 1, N + 1, 5)[cells])
