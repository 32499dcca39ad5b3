"""Pins of the oracle's source-term family (1D two-component reacting flow,
Sec. 2 eq. pdes_2_comps reduced to 1D; nested Picard predictor of eq.
lst_dg_predictor_nested_picards; source term of eq. ader_dg_method_full).

Pins that do not come from the oracle's own formulas:
* the ODE initial-value problem of Sec. 2.1 (eq. harm_osc) on one uniform cell
  is DG in time of degree N, whose values at the time nodes are the (N, N+1)
  Pade approximant of exp(dt A) (Lesaint-Raviart): textbook coefficients;
* global order 2N+1 at the time nodes and local order N+1 (Sec. 2.1);
* the predictor's fixed point solves the Kronecker-assembled system
  K^tau q + K^xi f(q) - M s(q) = F^0 u built from Upsilon, Lambda, Xi;
* with omega = 0 the species are passive: rho c1 = rho is advected exactly like
  the density, and the Euler part equals the (separately pinned) Euler oracle.
"""
from math import factorial

import numpy as np
import pytest

import workloads as W

MRS = 5


def pade_stability(N, Z):
    """(N, N+1) Pade approximant of exp at the matrix Z: Q(Z)^-1 P(Z)."""
    def coef(j, a, b):
        return factorial(a + b - j) * factorial(a) / (factorial(a + b) * factorial(j) * factorial(a - j))
    I = np.eye(Z.shape[0])
    P = sum(coef(j, N, N + 1) * np.linalg.matrix_power(Z, j) for j in range(N + 1))
    Q = sum(coef(j, N + 1, N) * np.linalg.matrix_power(-Z, j) for j in range(N + 2))
    return np.linalg.solve(Q, P)


def ode_state(n):
    return W.ode_state(n)[None]


# The data are uniform, so the cell width does not enter the exact solution;
# a wide cell keeps the (inactive) spatial DG operator far inside its stability
# limit (with dx = 1 the large ODE time steps give a Courant number ~2 and
# round-off perturbations of the uniform state grow ~100x per step).
ODE_DX = 1.0e3


def run_ode(orc, K, T=2 * np.pi):
    """K uniform steps of the one-cell ODE problem; returns node values and the
    predictor's time coefficients of every step."""
    n = orc.n
    dt = T / K
    u = ode_state(n).ravel()
    nodes, locs = [], []
    for _ in range(K):
        new, q, st, rc = orc.dg_step(u, ODE_DX, dt, want_q=True)
        assert rc == 0
        q = q.reshape(n, n, MRS)
        locs.append(q[:, 0, 3:5])
        nodes.append(new.reshape(n, MRS)[0, 3:5])
        u = new
    return dt, np.array(nodes), np.array(locs), u


@pytest.mark.parametrize("N", range(1, 8))
def test_ode_nodes_equal_pade_approximant(oracle_mod, N):
    orc = oracle_mod.ReactingOracle(N, omega=1.0, tol=1e-14, max_iter=200)
    K = 7
    dt, nodes, _, u = run_ode(orc, K)
    R = pade_stability(N, dt * np.array([[0.0, 1.0], [-1.0, 0.0]]))
    v = np.array([1.0, 0.0])
    ref = []
    for _ in range(K):
        v = R @ v
        ref.append(v)
    np.testing.assert_allclose(nodes, np.array(ref), rtol=0, atol=5e-14)
    # the state stays uniform in the cell and the Euler part does not move
    un = u.reshape(orc.n, MRS)
    np.testing.assert_allclose(un - un[0], 0.0, atol=1e-14)
    np.testing.assert_allclose(un[0, :3], ode_state(orc.n)[0, 0, :3], atol=1e-14)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_ode_orders_global_2n1_local_n1(oracle_mod, N):
    orc = oracle_mod.ReactingOracle(N, omega=1.0, tol=1e-14, max_iter=200)
    Ks = {1: (20, 40), 2: (20, 40), 3: (10, 20), 4: (8, 16)}[N]
    res = []
    for K in Ks:
        dt, nodes, locs, _ = run_ode(orc, K)
        res.append(oracle_mod.ode_errors(orc, dt, nodes, locs, 2 * np.pi))
    for i in range(3):
        pg = np.log(res[0][0][i] / res[1][0][i]) / np.log(2.0)
        pl = np.log(res[0][1][i] / res[1][1][i]) / np.log(2.0)
        assert abs(pg - (2 * N + 1)) < 0.35, (i, pg)
        assert abs(pl - (N + 1)) < 0.35, (i, pl)


def reacting_state(orc, nc, seed=1):
    return W.reacting_state(orc.node_x(nc), seed)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_predictor_solves_assembled_system(oracle_mod, N):
    """Fixed point of the nested loops = solution of
    (Upsilon (x) Lambda) q + (Lambda (x) Xi) f(q) - (Lambda (x) Lambda) s(q) = (phi(0) (x) Lambda) u
    (the paper's K^tau, K^xi, M, F^0 in 1D), assembled from the stored Upsilon,
    Lambda, Xi and checked to round-off; the single-loop form reaches it too."""
    orc = oracle_mod.ReactingOracle(N, omega=3.0, tol=1e-15)
    n = orc.n
    u = reacting_state(orc, 4, seed=N)[2]
    lam, dt = 0.05, 0.08
    q, it, inner, rc = orc.predict_cell(u, lam, dt)
    assert rc == 0 and inner >= it
    Ups, Lam, Xi = (orc.table(t) for t in ("ups", "lam", "xi_m"))
    phi0 = orc.table("psi0")
    f = np.array([[lam * orc.flux(q[a, b]) for b in range(n)] for a in range(n)])
    s = np.array([[dt * orc.source(q[a, b]) for b in range(n)] for a in range(n)])
    qv, fv, sv = q.reshape(n * n, MRS), f.reshape(n * n, MRS), s.reshape(n * n, MRS)
    res = (np.kron(Ups, Lam) @ qv + np.kron(Lam, Xi) @ fv - np.kron(Lam, Lam) @ sv
           - np.kron(phi0[:, None], Lam) @ u)
    assert np.abs(res).max() < 1e-13
    qd, itd, rcd = orc.predict_cell(u, lam, dt, direct=True)[0], None, None
    np.testing.assert_allclose(qd, q, rtol=0, atol=1e-13)


def test_omega_zero_species_are_passive(oracle_mod):
    """omega = 0, rho = 1 + 0.2 sin 2 pi x, u = p = 1, c1 = 1, c2 = 0: rho c1 is
    advected exactly like rho, and (rho, m, E) equal the Euler oracle's."""
    N, nc = 3, 24
    orc = oracle_mod.ReactingOracle(N, omega=0.0)
    eul = oracle_mod.Oracle(N)
    u3 = W.nodal_state(W.sine(), eul.node_x(nc))
    U = np.concatenate([u3, u3[..., :1], np.zeros_like(u3[..., :1])], -1)
    out, steps, t, rc = orc.solve(U, 1.0 / nc, max_steps=20)
    ref, steps_e, t_e, rc_e = eul.solve("dg", u3, 1.0 / nc, max_steps=20)
    out = out.reshape(nc, N + 1, MRS)
    assert rc == 0 and steps == steps_e == 20 and abs(t - t_e) < 1e-15
    np.testing.assert_allclose(out[..., :3], ref.reshape(nc, N + 1, 3), rtol=0, atol=2e-14)
    np.testing.assert_allclose(out[..., 3], out[..., 0], rtol=0, atol=2e-14)
    np.testing.assert_allclose(out[..., 4], 0.0, atol=0)


def test_step_balance_and_conservation(oracle_mod):
    """Periodic mesh: mass, momentum, energy conserved; each species changes by
    exactly the space-time integral of its source (the fluxes telescope)."""
    N, nc = 3, 16
    orc = oracle_mod.ReactingOracle(N, omega=2.0)
    U = reacting_state(orc, nc, seed=5)
    dx = 1.0 / nc
    dt = orc.dg_dt(U, dx)
    new, q, st, rc = orc.dg_step(U, dx, dt, want_q=True)
    assert rc == 0
    w = orc.table("w")
    q = q.reshape(nc, N + 1, N + 1, MRS)
    tot0 = dx * np.einsum("ckr,k->r", U, w)
    tot1 = dx * np.einsum("ckr,k->r", new.reshape(nc, N + 1, MRS), w)
    np.testing.assert_allclose(tot1[:3], tot0[:3], rtol=1e-14)
    src = np.zeros(MRS)
    for c in range(nc):
        for l0 in range(N + 1):
            for k in range(N + 1):
                src += dx * w[k] * w[l0] * dt * orc.source(q[c, l0, k])
    np.testing.assert_allclose(tot1[3:] - tot0[3:], src[3:], rtol=0, atol=1e-15)


def test_sampled_cells_equal_full_step(oracle_mod):
    N, nc = 2, 12
    orc = oracle_mod.ReactingOracle(N, omega=1.5)
    U = reacting_state(orc, nc, seed=9)
    dx = 1.0 / nc
    dt = orc.dg_dt(U, dx)
    full, _, _, _ = orc.dg_step(U, dx, dt)
    cells = np.array([0, 5, nc - 1])
    sel, rc = orc.dg_step_cells(U, dx, dt, cells)
    np.testing.assert_array_equal(sel, full.reshape(nc, N + 1, MRS)[cells])
