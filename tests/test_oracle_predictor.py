"""Pins of the oracle's pointwise physics and LST-DG predictor.

Sources: Sec. 2 eq. system_of_equations (Euler), Sec. 1.1 eq.
lst_dg_predictor_picard / eq. ind_prop / the zero eigenvalues of L^xi, and
Algorithm lst_dg_predictor (nested form).  The brute-force pin solves the
unpreconditioned predictor system K^tau q + K^xi f(q) = F^0 u, assembled with
Kronecker products, by Newton's method with a finite-difference Jacobian.
"""
import numpy as np
import pytest

import workloads as W

GAMMA = 1.4


def np_flux(U):
    rho, m, E = U[..., 0], U[..., 1], U[..., 2]
    u = m / rho
    p = (GAMMA - 1) * (E - 0.5 * rho * u * u)
    return np.stack([rho * u, rho * u * u + p, u * (E + p)], axis=-1)


def test_flux_and_wave_speed_closed_forms(oracle_mod):
    L = oracle_mod.lib()
    # rho = 1, u = 1, p = 1: E = 1/0.4 + 1/2 = 3; F = (1, 2, 4); c = sqrt(1.4)
    U = np.array([1.0, 1.0, 3.0])
    F = np.zeros(3)
    L.ob_euler_flux(GAMMA, U, F)
    np.testing.assert_allclose(F, [1.0, 2.0, 4.0], rtol=1e-15)
    assert abs(L.ob_wave_speed(GAMMA, U) - (1 + np.sqrt(1.4))) < 1e-15
    # rho = 2, u = -0.5, p = 0.8
    U = W.conserved(2.0, -0.5, 0.8)
    L.ob_euler_flux(GAMMA, U, F)
    np.testing.assert_allclose(F, [-1.0, 2 * 0.25 + 0.8, -0.5 * (0.8 / 0.4 + 0.25 + 0.8)],
                               rtol=1e-14)
    assert abs(L.ob_wave_speed(GAMMA, U) - (0.5 + np.sqrt(1.4 * 0.8 / 2.0))) < 1e-15
    # non-physical states are flagged
    assert np.isnan(L.ob_wave_speed(GAMMA, np.array([-1.0, 0.0, 1.0])))


def test_rusanov_consistency_and_closed_form(oracle_mod):
    L = oracle_mod.lib()
    rng = np.random.default_rng(0)
    a = W.random_state(rng, ())
    G = np.zeros(3)
    F = np.zeros(3)
    L.ob_rusanov(GAMMA, a, a, G)
    L.ob_euler_flux(GAMMA, a, F)
    np.testing.assert_allclose(G, F, rtol=1e-15)
    # two states with known speeds: s = max(|u|+c)
    a = W.conserved(1.0, 1.0, 1.0)
    b = W.conserved(0.5, -2.0, 0.5)
    sa, sb = 1 + np.sqrt(1.4), 2 + np.sqrt(1.4)
    s = max(sa, sb)
    expect = 0.5 * (np_flux(a) + np_flux(b)) - 0.5 * s * (b - a)
    L.ob_rusanov(GAMMA, a, b, G)
    np.testing.assert_allclose(G, expect, rtol=1e-14)


@pytest.mark.parametrize("N", [0, 1, 2, 3, 5, 7])
def test_constant_state_is_a_fixed_point(oracle_mod, N):
    o = oracle_mod.Oracle(N)
    u = np.tile(W.conserved(1.3, 0.7, 0.9), (o.n, 1))
    q, it, rc = o.predict_cell(u, lam=0.05)
    assert rc == 0
    # k~ 1 = 0 up to rounding of the operator entries
    np.testing.assert_allclose(q, np.broadcast_to(u, q.shape), rtol=0, atol=1e-14)
    assert it <= 2


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_advected_polynomial_is_exact_within_N_iterations(oracle_mod, N):
    """u = 1, p = 1 keeps the iterates on an affine manifold where the flux is
    affine; the exact space-time solution rho(xi - lam tau) is a polynomial of
    degree <= N in each variable.  The initial error rho(xi - lam tau) - rho(xi)
    has xi-degree N-1 and every sweep of the nilpotent L^xi = kappa~ (x) k~
    lowers it by one, so Picard is exact after N iterations."""
    o = oracle_mod.Oracle(N)
    rng = np.random.default_rng(N)
    coeff = rng.uniform(-0.1, 0.1, size=N + 1)
    coeff[0] = 1.0
    coeff[-1] = 0.3  # a full-degree polynomial
    rho = lambda x: np.polyval(coeff[::-1], x)
    xi = o.table("xi")
    lam = 0.4 / (2 * N + 1)
    u = W.conserved(rho(xi), 1.0, 1.0)
    exact = W.conserved(rho(xi[None, :] - lam * xi[:, None]), 1.0, 1.0)
    o.set(fixed_iter=N)
    q, it, rc = o.predict_cell(u, lam)
    np.testing.assert_allclose(q, exact, rtol=0, atol=2e-14)
    if N >= 2:
        o.set(fixed_iter=N - 1)  # one iteration short is measurably wrong
        q_short, _, _ = o.predict_cell(u, lam)
        assert np.abs(q_short - exact).max() > 1e-12
    o.set(fixed_iter=0)
    q, it, rc = o.predict_cell(u, lam)
    assert rc == 0 and it <= N + 1
    np.testing.assert_allclose(q, exact, rtol=0, atol=2e-14)


def _newton_predictor(o, u, lam):
    """Solve K^tau q + K^xi lam F(q) - F^0 u = 0 with Kronecker-assembled matrices."""
    n = o.n
    w = o.table("w")
    dphi = o.table("dphi")
    psi0, psi1 = o.table("psi0"), o.table("psi1")
    Lam = np.diag(w)
    Xi = Lam @ dphi.T  # Xi_kl = int phi_k phi_l' = w_k phi_l'(xi_k)
    Ups = np.outer(psi1, psi1) - Xi.T
    Kt = np.kron(Ups, Lam)
    Kx = np.kron(Lam, Xi)
    F0 = np.kron(psi0[:, None], Lam)
    rhs = F0 @ u.reshape(n, 3)

    def resid(qv):
        q = qv.reshape(n * n, 3)
        return (Kt @ q + Kx @ (lam * np_flux(q)) - rhs).ravel()

    qv = np.tile(u.reshape(n, 3), (n, 1)).ravel()
    for _ in range(30):
        r = resid(qv)
        J = np.zeros((qv.size, qv.size))
        for j in range(qv.size):
            h = 1e-7 * max(1.0, abs(qv[j]))
            e = np.zeros_like(qv)
            e[j] = h
            J[:, j] = (resid(qv + e) - resid(qv - e)) / (2 * h)
        dq = np.linalg.solve(J, -r)
        qv = qv + dq
        if np.abs(dq).max() < 1e-15:
            break
    return qv.reshape(n, n, 3), np.abs(resid(qv)).max()


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_picard_matches_newton_on_full_system(oracle_mod, N):
    o = oracle_mod.Oracle(N, tol=1e-15)
    rng = np.random.default_rng(100 + N)
    u = W.random_state(rng, (o.n,), rho=(0.8, 1.2), u=(-0.5, 0.5), p=(0.8, 1.2))
    lam = 0.4 / (2 * N + 1) / 2.5  # Courant-scaled dt/dx for |u|+c < 2.5
    q, it, rc = o.predict_cell(u, lam)
    qn, res = _newton_predictor(o, u, lam)
    assert res < 1e-13
    np.testing.assert_allclose(q, qn, rtol=0, atol=1e-13)


@pytest.mark.parametrize("N", [1, 3, 5])
def test_nested_algorithm_matches_direct_iteration(oracle_mod, N):
    o = oracle_mod.Oracle(N)
    rng = np.random.default_rng(7 + N)
    u = W.random_state(rng, (o.n,))
    lam = 0.4 / (2 * N + 1) / 3.0
    q1, it1, rc1 = o.predict_cell(u, lam)
    q2, it2, rc2 = o.predict_cell(u, lam, nested=True)
    assert rc1 == 0 and rc2 == 0 and it1 == it2
    np.testing.assert_allclose(q1, q2, rtol=0, atol=1e-15)


def test_iteration_cap_reports_not_converged(oracle_mod):
    o = oracle_mod.Oracle(3, max_iter=2)
    rng = np.random.default_rng(3)
    u = W.random_state(rng, (o.n,))
    _, it, rc = o.predict_cell(u, 0.02)
    assert it == 2 and rc == oracle_mod.OB_ERR_NOT_CONVERGED
