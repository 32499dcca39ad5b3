"""Pins of the oracle's basis and operator tables against facts fixed outside it.

Sources: Sec. 1.1 of the paper (eq. gl_rule, eq. m_and_kappa_matrices, the
Kronecker forms of K^tau and K^xi, the zero eigenvalues of L^xi, eq. ind_prop),
Sec. 1.4 (subcell projection P), and textbook Gauss-Legendre nodes.
"""
import numpy as np
import pytest

DEGREES = list(range(0, 10))


@pytest.fixture(scope="module", params=DEGREES)
def orc(request, oracle_mod):
    return oracle_mod.Oracle(request.param)


def test_textbook_nodes(oracle_mod):
    # closed forms of the Gauss-Legendre rule on [-1, 1], mapped to [0, 1]
    s35 = np.sqrt(3.0 / 5.0)
    a = np.sqrt(3.0 / 7.0 - 2.0 / 7.0 * np.sqrt(6.0 / 5.0))
    b = np.sqrt(3.0 / 7.0 + 2.0 / 7.0 * np.sqrt(6.0 / 5.0))
    wa = (18.0 + np.sqrt(30.0)) / 36.0
    wb = (18.0 - np.sqrt(30.0)) / 36.0
    cases = {
        0: ([0.0], [2.0]),
        1: ([-1 / np.sqrt(3.0), 1 / np.sqrt(3.0)], [1.0, 1.0]),
        2: ([-s35, 0.0, s35], [5 / 9, 8 / 9, 5 / 9]),
        3: ([-b, -a, a, b], [wb, wa, wa, wb]),
    }
    for N, (x, W) in cases.items():
        o = oracle_mod.Oracle(N)
        np.testing.assert_allclose(o.table("xi"), (1 + np.array(x)) / 2, rtol=0, atol=1e-15)
        np.testing.assert_allclose(o.table("w"), np.array(W) / 2, rtol=0, atol=1e-15)


def test_gl_exactness_degree_2N_plus_1(orc):
    xi, w = orc.table("xi"), orc.table("w")
    assert abs(w.sum() - 1.0) < 1e-14
    N = orc.N
    for j in range(0, 2 * N + 2):
        assert abs((w * xi**j).sum() - 1.0 / (j + 1)) < 2e-14, j
    # one degree higher the rule misses by the textbook remainder
    # E = (n!)^4 / ((2n+1) ((2n)!)^2) for f = xi^(2n) on [0, 1], n = N + 1
    from math import factorial
    n = N + 1
    j = 2 * n
    remainder = factorial(n) ** 4 / ((2 * n + 1) * factorial(2 * n) ** 2)
    got = 1.0 / (j + 1) - (w * xi**j).sum()
    assert abs(got - remainder) <= 1e-6 * remainder + 2e-15, (got, remainder)


def test_nodes_symmetric_and_sorted(orc):
    xi, w = orc.table("xi"), orc.table("w")
    assert np.all(np.diff(xi) > 0)
    np.testing.assert_allclose(xi + xi[::-1], 1.0, atol=1e-15)
    np.testing.assert_allclose(w, w[::-1], atol=1e-15)


def test_weights_are_basis_norms_and_mass_is_diagonal(orc):
    # w_k = int phi_k^2 (eq. gl_rule) and Lambda_kl = w_k delta_kl (eq. m_and_kappa_matrices)
    lam = orc.table("lam")
    np.testing.assert_allclose(np.diag(lam), orc.table("w"), rtol=1e-13, atol=1e-15)
    off = lam - np.diag(np.diag(lam))
    assert np.abs(off).max() < 1e-13


def test_lagrange_property_and_traces(orc):
    xi = orc.table("xi")
    for k in range(orc.n):
        np.testing.assert_allclose(orc.phi(xi[k]), np.eye(orc.n)[k], atol=1e-13)
    np.testing.assert_allclose(orc.table("psi0"), orc.phi(0.0), atol=1e-12)
    np.testing.assert_allclose(orc.table("psi1"), orc.phi(1.0), atol=1e-12)
    # partition of unity
    assert abs(orc.table("psi0").sum() - 1) < 1e-12 and abs(orc.table("psi1").sum() - 1) < 1e-12


def test_dphi_matches_finite_differences(orc):
    # Dphi_kl = phi_k'(xi_l), checked against central differences of the product form
    xi, D = orc.table("xi"), orc.table("dphi")
    h = 1e-6
    for l in range(orc.n):
        fd = (orc.phi(xi[l] + h) - orc.phi(xi[l] - h)) / (2 * h)
        np.testing.assert_allclose(D[:, l], fd, rtol=0, atol=1e-6 * max(1.0, np.abs(fd).max()))


def test_k_tilde_is_dphi_transposed(orc):
    # two constructions: k~ = Lambda^-1 Xi from exact integrals, Dphi from derivatives at nodes
    np.testing.assert_allclose(orc.table("kt"), orc.table("dphi").T, rtol=0,
                               atol=1e-12 * max(1.0, np.abs(orc.table("kt")).max()))


def test_k_tilde_differentiates_polynomials(orc):
    xi, kt = orc.table("xi"), orc.table("kt")
    np.testing.assert_allclose(kt @ np.ones(orc.n), 0.0, atol=1e-11 * (orc.N + 1) ** 2)
    for j in range(1, orc.N + 1):
        np.testing.assert_allclose(kt @ xi**j, j * xi ** (j - 1), rtol=0, atol=1e-10)


def test_k_tilde_and_L_xi_nilpotent(orc):
    # the eigenvalues of L^xi = kappa~ (x) k~ are zero (Sec. 1.1): k~^(N+1) = 0
    kt, kap = orc.table("kt"), orc.table("kap")
    P = np.linalg.matrix_power(kt, orc.n)
    assert np.abs(P).max() < 1e-8 * max(1.0, np.abs(kt).max()) ** orc.n
    L = np.kron(kap, kt)
    Ln = np.linalg.matrix_power(L, orc.n)
    assert np.abs(Ln).max() < 1e-8 * max(1.0, np.abs(L).max()) ** orc.n


def test_integration_by_parts(orc):
    # Xi + Xi^T = psi~ psi~^T - psi psi^T
    X, p0, p1 = orc.table("xi_m"), orc.table("psi0"), orc.table("psi1")
    np.testing.assert_allclose(X + X.T, np.outer(p1, p1) - np.outer(p0, p0), atol=1e-12)


def test_L0_is_identity_in_space(orc):
    # eq. ind_prop: L^0 = (Upsilon^-1 psi) (x) I = 1 (x) I, i.e. Upsilon 1 = psi
    U, p0 = orc.table("ups"), orc.table("psi0")
    np.testing.assert_allclose(U @ np.ones(orc.n), p0, atol=1e-12)
    # and kappa~ Lambda^-1 psi = 1
    np.testing.assert_allclose(orc.table("kap") @ (p0 / orc.table("w")), 1.0, atol=1e-11)


def test_kappa_tilde_integrates_in_time(orc):
    # upwind DG in time: q = u0 + kappa~ g solves dq/dtau = g exactly for g of degree <= N-1
    xi, kap = orc.table("xi"), orc.table("kap")
    for j in range(0, orc.N):
        np.testing.assert_allclose(kap @ xi**j, xi ** (j + 1) / (j + 1), rtol=0, atol=1e-12)


def test_d_tilde_columns_sum_to_zero(orc):
    np.testing.assert_allclose(orc.table("dt_m").sum(axis=0), 0.0, atol=1e-10 * orc.n**2)
    np.testing.assert_allclose(orc.table("dt_m"), orc.table("dphi") * orc.table("w")[None, :],
                               atol=1e-13 * orc.n**2)


def test_subcell_projection(orc):
    # P_jk = Ns int phi_k over subcell j: exact subcell averages of any polynomial of degree <= N
    P, xi = orc.table("P"), orc.table("xi")
    Ns = 2 * orc.N + 1
    assert P.shape == (Ns, orc.n)
    np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-12)
    edges = np.arange(Ns + 1) / Ns
    for j in range(0, orc.N + 1):
        exact = Ns * (edges[1:] ** (j + 1) - edges[:-1] ** (j + 1)) / (j + 1)
        np.testing.assert_allclose(P @ xi**j, exact, atol=1e-11)
