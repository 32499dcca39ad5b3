"""Pins of the oracle's outflow boundaries, a posteriori subcell limiter
(Sec. 1.4 eq. p_operator / eq. r_operator, PAD and NAD eq. nad_ineq) and of the
exact Riemann solver used as the reference for the classical tests of Sec. 2
(Table classical_tests_1d).

Independent pins: the exact Riemann solution conserves mass, momentum and energy
(its integral changes by the boundary fluxes); R is a left inverse of P and P R
an orthogonal projector; with the limiter off (or on smooth data, where no cell
is troubled) the step is the plain DG step; the limited step is conservative
(periodic) and changes the totals by exactly the boundary fluxes (outflow);
the limited solutions of the four Riemann problems stay physical and converge
to the exact ones.  The subcell ADER-WENO2 scheme: its degree-1 WENO
reconstruction keeps the subcell average, is exact on linear data and takes the
flat side of a jump; with every cell recomputed on its subcells the step keeps
a uniform state, conserves, and converges at second order on a smooth wave."""
import numpy as np
import pytest

import workloads as W

TESTS = W.RIEMANN_TESTS
GAMMA = 1.4


def conserved(rho, u, p, g=GAMMA):
    return np.stack([rho, rho * u, p / (g - 1) + 0.5 * rho * u * u], -1)


def euler_flux(U, g=GAMMA):
    rho, m, E = U[..., 0], U[..., 1], U[..., 2]
    u = m / rho
    p = (g - 1) * (E - 0.5 * m * u)
    return np.stack([m, m * u + p, (E + p) * u], -1)


def riemann_state(o, nc, test):
    return W.riemann_initial(o.node_x(nc), test)


@pytest.mark.parametrize("test", [1, 2, 3, 4])
def test_exact_riemann_solution_is_conservative(test):
    """int_0^1 U(x, t) dx - int_0^1 U(x, 0) dx = -t (F(U_R) - F(U_L)) while the
    waves stay inside [0, 1] (trapezoid rule on 4e5 points)."""
    L, R = TESTS[test]
    t = 0.15
    x = np.linspace(0.0, 1.0, 400_001)
    rho, u, p = W.riemann_solution(L, R, x, t)
    Ut = conserved(rho, u, p)
    UL, UR = conserved(*map(np.array, L)), conserved(*map(np.array, R))
    integ = np.trapezoid(Ut, x, axis=0)
    init = 0.5 * (UL + UR)
    np.testing.assert_allclose(integ - init, -t * (euler_flux(UR) - euler_flux(UL)), atol=5e-5)
    # symmetric data (tests 3, 4) give u* = 0 and a symmetric density
    if test in (3, 4):
        assert abs(W.riemann_star_state(L, R)[1]) < 1e-14
        np.testing.assert_allclose(rho, rho[::-1], atol=1e-12)


@pytest.mark.parametrize("N", range(0, 8))
def test_reconstruction_is_pseudo_inverse_of_projection(oracle_mod, N):
    o = oracle_mod.Oracle(N)
    P, R = o.table("P"), o.r_matrix()
    np.testing.assert_allclose(R @ P, np.eye(N + 1), atol=1e-13)
    Pr = P @ R
    np.testing.assert_allclose(Pr, Pr.T, atol=1e-13)
    np.testing.assert_allclose(Pr @ Pr, Pr, atol=1e-13)


@pytest.mark.parametrize("N", [2, 5])
def test_limiter_off_periodic_is_the_dg_step(oracle_mod, N):
    o = oracle_mod.Oracle(N)
    nc = 40
    u = W.nodal_state(W.modes4(), o.node_x(nc))
    dt = o.dg_dt(u, 1.0 / nc)
    ref, _, _, _ = o.dg_step(u, 1.0 / nc, dt)
    got, tr, rc = o.dgl_step(u, 1.0 / nc, dt, bc="periodic", limiter=False)
    assert rc == 0 and not tr.any()
    np.testing.assert_array_equal(got, ref)


def test_smooth_data_is_never_troubled(oracle_mod):
    N, nc = 3, 50
    o = oracle_mod.Oracle(N)
    u = W.nodal_state(W.sine(), o.node_x(nc))
    a, steps, t, rc, ttot = o.dgl_solve(u, 1.0 / nc, max_steps=30, limiter=True)
    b, _, _, _, _ = o.dgl_solve(u, 1.0 / nc, max_steps=30, limiter=False)
    assert rc == 0 and ttot == 0
    np.testing.assert_array_equal(a, b)


def test_outflow_step_changes_totals_by_boundary_fluxes(oracle_mod):
    """Sod data: the boundary cells hold the constant left / right states, so the
    time-integrated boundary fluxes are dt F(U_L) and dt F(U_R) exactly."""
    N, nc = 3, 100
    o = oracle_mod.Oracle(N)
    u = riemann_state(o, nc, 1)
    dx = 1.0 / nc
    dt = o.dg_dt(u, dx)
    new, tr, rc = o.dgl_step(u, dx, dt, bc="outflow", limiter=True)
    assert rc == 0 and tr.any()
    w = o.table("w")
    tot = lambda U: dx * np.einsum("ckr,k->r", U.reshape(nc, N + 1, 3), w)
    UL, UR = conserved(*map(np.array, TESTS[1][0])), conserved(*map(np.array, TESTS[1][1]))
    np.testing.assert_allclose(tot(new) - tot(u), -dt * (euler_flux(UR) - euler_flux(UL)),
                               rtol=0, atol=1e-15)


@pytest.mark.parametrize("N", [3, 5])
def test_outflow_boundary_keeps_a_uniform_state_stable(oracle_mod, N):
    """A uniform state with 1e-10 noise stays within rounding of the uniform state
    over 1500 outflow steps: the ghost is the boundary cell's mean, so the Rusanov
    dissipation damps boundary trace modes (an interior-trace ghost lets the noise
    grow without bound at N = 5)."""
    nc = 16
    o = oracle_mod.Oracle(N)
    U = np.tile(np.array([0.125, 0.0, 0.25]), (nc, N + 1, 1))
    rng = np.random.default_rng(7)
    u = (U + 1e-10 * rng.standard_normal(U.shape)).ravel()
    dev0 = np.abs(u.reshape(U.shape) - U).max()
    u, steps, t, rc, _ = o.dgl_solve(u, 1e-3, max_steps=1500, bc="outflow", limiter=False)
    assert rc == 0 and steps == 1500
    assert np.abs(u.reshape(U.shape) - U).max() < 10 * dev0


def test_limited_periodic_step_is_conservative(oracle_mod):
    """Two jumps on a periodic mesh (a Sod tube and its mirror): the limiter
    acts and the totals stay fixed."""
    N, nc = 4, 80
    o = oracle_mod.Oracle(N)
    x = o.node_x(nc)
    inside = (x > 0.25) & (x < 0.75)
    rho = np.where(inside, 1.0, 0.125)
    p = np.where(inside, 1.0, 0.1)
    u = conserved(rho, np.zeros_like(rho), p)
    dx = 1.0 / nc
    w = o.table("w")
    tot = lambda U: dx * np.einsum("ckr,k->r", U.reshape(nc, N + 1, 3), w)
    out, steps, t, rc, ttot = o.dgl_solve(u, dx, max_steps=40, bc="periodic", limiter=True)
    assert rc == 0 and ttot > 0
    np.testing.assert_allclose(tot(out), tot(u), rtol=2e-14, atol=2e-15)


def density_l1(o, U, nc, test, t):
    L, R = TESTS[test]
    gx, gw = np.polynomial.legendre.leggauss(25)
    gx, gw = 0.5 * (gx + 1), 0.5 * gw
    phi = np.stack([o.phi(x) for x in gx])
    rho_h = U.reshape(nc, o.n, 3)[:, :, 0] @ phi.T
    xs = (np.arange(nc)[:, None] + gx[None, :]) / nc
    re, _, _ = W.riemann_solution(L, R, xs, t)
    return float((np.abs(rho_h - re) @ gw).sum() / nc)


@pytest.mark.parametrize("test", [1, 2, 3, 4])
def test_riemann_problems_with_limiter(oracle_mod, test):
    """Sec. 2 classical tests, DG N = 3, outflow, CFL 0.4, t_final = 0.15: every
    step stays physical, the L1 density error against the exact solution halves
    (first order, as for any scheme at discontinuities) when the mesh doubles,
    and only a few cells per step are limited (none or almost none for the two
    rarefactions)."""
    N = 3
    o = oracle_mod.Oracle(N)
    errs, per_step = [], []
    for nc in (100, 200):
        u = riemann_state(o, nc, test)
        out, steps, t, rc, ttot = o.dgl_solve(u, 1.0 / nc, t_end=0.15, bc="outflow", limiter=True)
        assert rc == 0 and t == 0.15
        v = np.einsum("jk,ckr->cjr", o.table("P"), out.reshape(nc, N + 1, 3))
        e_int = v[..., 2] - 0.5 * v[..., 1] ** 2 / v[..., 0]
        assert (v[..., 0] > 0).all() and (e_int > 0).all()
        errs.append(density_l1(o, out, nc, test, 0.15))
        per_step.append(ttot / steps)
    assert errs[1] < 0.6 * errs[0] and errs[1] < 0.005, errs
    assert max(per_step) < (2.0 if test == 4 else 15.0), per_step


def test_weno2_reconstruction(oracle_mod):
    """degree-1 WENO on a subcell: the Gauss-node values average to v0 (the
    subcell mean is kept); linear data give the common slope exactly; a
    symmetric extremum gives slope 0; at a jump the flat stencil wins."""
    o = oracle_mod.Oracle(1)
    xi = o.table("xi")
    rng = np.random.default_rng(3)
    for _ in range(20):
        vm, v0, vp = rng.uniform(0.1, 2.0, (3, 3))
        w = o.weno2(vm, v0, vp)
        np.testing.assert_allclose(0.5 * (w[0] + w[1]), v0, rtol=0, atol=4e-16)
    v0, s = np.array([1.0, -0.5, 2.5]), np.array([0.3, -0.2, 0.7])
    w = o.weno2(v0 - s, v0, v0 + s)
    np.testing.assert_allclose(w, v0 + np.outer(xi - 0.5, s), rtol=0, atol=1e-15)
    w = o.weno2(v0 + s, v0, v0 + s)
    np.testing.assert_allclose(w, np.tile(v0, (2, 1)), rtol=0, atol=1e-15)
    flat = np.array([1.0, 0.0, 2.5])
    w = o.weno2(flat, flat, flat + np.array([9.0, 3.0, 20.0]))
    np.testing.assert_allclose(w, np.tile(flat, (2, 1)), rtol=0, atol=1e-12)


def test_all_troubled_keeps_uniform_state_and_conserves(oracle_mod):
    """limiter 2 (every cell recomputed on its subcells): a uniform state is a
    fixed point (to rounding) and a periodic step with a jump conserves."""
    N, nc = 3, 24
    o = oracle_mod.Oracle(N)
    U = np.tile(np.array([0.7, 0.2, 1.9]), (nc, N + 1, 1))
    out, tr, rc = o.dgl_step(U.ravel(), 1.0 / nc, 1e-3, limiter=2)
    assert rc == 0 and tr.all()
    np.testing.assert_allclose(out.reshape(U.shape), U, rtol=0, atol=1e-14)
    x = o.node_x(nc)
    inside = (x > 0.25) & (x < 0.625)  # jumps on cell faces
    u = conserved(np.where(inside, 1.0, 0.125), np.where(inside, 0.4, 0.0),
                  np.where(inside, 1.0, 0.1))
    dt = o.dg_dt(u, 1.0 / nc)
    out, tr, rc = o.dgl_step(u, 1.0 / nc, dt, limiter=2)
    w = o.table("w")
    tot = lambda V: np.einsum("ckr,k->r", V.reshape(nc, N + 1, 3), w) / nc
    assert rc == 0
    np.testing.assert_allclose(tot(out), tot(u), rtol=2e-15, atol=2e-16)


def test_all_troubled_is_second_order(oracle_mod):
    """limiter 2 on the density wave rho = 1 + 0.2 sin(2 pi (x - t)), u = p = 1
    (an exact Euler solution), DG N = 2, t = 0.25: the L1 error of the density
    cell means falls at the second order of the ADER-WENO2 subcell scheme."""
    N = 2
    o = oracle_mod.Oracle(N)
    w = o.table("w")
    errs = []
    for nc in (16, 32, 64):
        x = o.node_x(nc)
        u = conserved(1 + 0.2 * np.sin(2 * np.pi * x), np.ones(x.shape), np.ones(x.shape))
        out, steps, t, rc, _ = o.dgl_solve(u, 1.0 / nc, t_end=0.25, limiter=2)
        assert rc == 0 and t == 0.25
        a = np.arange(nc) / nc - 0.25
        exact = 1 + 0.2 * nc * (np.cos(2 * np.pi * a) - np.cos(2 * np.pi * (a + 1.0 / nc))) / (2 * np.pi)
        errs.append(np.abs(np.einsum("ck,k->c", out.reshape(nc, N + 1, 3)[..., 0], w) - exact).mean())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 1.85 and orders.max() < 2.5, (errs, orders)


def test_rusanov_with_a_nonphysical_state_is_nan(oracle_mod):
    """the reading for a non-physical trace state (rho <= 0 or p <= 0, which the
    paper's PAD is there to catch): the Rusanov flux is NaN whichever side the
    state is on, so the cells of the face fail PAD and are recomputed"""
    import ctypes as C
    L = oracle_mod.lib()
    good = conserved(np.array(1.0), np.array(0.3), np.array(1.0))
    for bad in (conserved(np.array(1.0), np.array(0.0), np.array(-0.1)),
                np.array([-0.2, 0.0, -0.5])):
        for a, b in ((good, bad), (bad, good)):
            G = np.zeros(3)
            L.ob_rusanov(1.4, np.ascontiguousarray(a, dtype=np.float64),
                         np.ascontiguousarray(b, dtype=np.float64), G)
            assert np.isnan(G).all()
    G = np.zeros(3)
    L.ob_rusanov(1.4, good, good, G)
    np.testing.assert_allclose(G, euler_flux(good), rtol=1e-15)
