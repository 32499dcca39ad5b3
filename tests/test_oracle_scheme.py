"""Pins of the oracle's CFL rule, DG corrector, WENO reconstruction, FV update and
time loop against facts fixed outside the oracle.

Sources: Sec. 1.5 (time step constraint), Sec. 1.4 (subcell averages), eq.
ader_dg_method_full and eq. ader_weno_fv_method_full reduced to 1D, eq.
weno_reconstr, Sec. 2.1 (sine-wave advection, eq. epsilons, expected orders
N+1 of Table conv_orders_pde_2d).  Independent references used here: a numpy
brute-force corrector that integrates the interpolated fluxes with a 30-point
rule, the textbook first-order Rusanov scheme (the N = 0 case), exact
polynomial reproduction, conservation and free-stream preservation.
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


def np_speed(U):
    rho, m, E = U[..., 0], U[..., 1], U[..., 2]
    u = m / rho
    p = (GAMMA - 1) * (E - 0.5 * rho * u * u)
    return np.abs(u) + np.sqrt(GAMMA * p / rho)


def np_rusanov(a, b):
    s = np.maximum(np_speed(a), np_speed(b))[..., None]
    return 0.5 * (np_flux(a) + np_flux(b)) - 0.5 * s * (b - a)


def lagrange(xi, x):
    """Lagrange basis on nodes xi at points x, product form -> [n, len(x)]."""
    x = np.atleast_1d(np.asarray(x, dtype=float))
    n = len(xi)
    out = np.ones((n, x.size))
    for k in range(n):
        for m in range(n):
            if m != k:
                out[k] *= (x - xi[m]) / (xi[k] - xi[m])
    return out


def lagrange_deriv(xi, x):
    """Derivatives of the Lagrange basis by the product rule -> [n, len(x)]."""
    x = np.atleast_1d(np.asarray(x, dtype=float))
    n = len(xi)
    out = np.zeros((n, x.size))
    for k in range(n):
        for j in range(n):
            if j == k:
                continue
            term = np.full(x.size, 1.0 / (xi[k] - xi[j]))
            for m in range(n):
                if m != k and m != j:
                    term *= (x - xi[m]) / (xi[k] - xi[m])
            out[k] += term
    return out


# ---------------------------------------------------------------------------
# CFL
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N", [0, 1, 3, 5, 7])
def test_dt_constant_state(oracle_mod, N):
    o = oracle_mod.Oracle(N, cfl=0.4)
    U = W.conserved(1.2, -0.3, 0.7)
    u = np.tile(U, (10, o.n, 1))
    lam = 0.3 + np.sqrt(1.4 * 0.7 / 1.2)
    assert abs(o.dg_lambda_max(u) - lam) < 1e-14
    assert abs(o.dg_dt(u, 0.1) - 0.4 / (2 * N + 1) * 0.1 / lam) < 1e-16
    v = np.tile(U, (10, 1))
    assert abs(o.fv_dt(v, 0.1) - 0.4 * 0.1 / lam) < 1e-16


@pytest.mark.parametrize("N", [1, 2, 4])
def test_lambda_over_subcell_averages(oracle_mod, N):
    # linear rho, m, E in a cell: subcell averages = values at subcell midpoints
    o = oracle_mod.Oracle(N)
    xi = o.table("xi")
    Ns = 2 * N + 1
    mids = (np.arange(Ns) + 0.5) / Ns
    rho = lambda x: 1.0 + 0.5 * x
    m = lambda x: -0.2 + 1.5 * x
    E = lambda x: 2.0 + 0.1 * x
    u = np.stack([rho(xi), m(xi), E(xi)], axis=-1)[None]
    expect = np_speed(np.stack([rho(mids), m(mids), E(mids)], axis=-1)).max()
    assert abs(o.dg_lambda_max(u) - expect) < 1e-14
    # the nodal maximum would differ: the subcell rule is what is pinned
    assert abs(np_speed(u[0]).max() - expect) > 1e-6


@pytest.mark.parametrize("N", [0, 2, 5, 7])
def test_lambda_nodal_mode(oracle_mod, N):
    """cfl_mode 1: lambda over the nodal values themselves.  Pinned by the
    primitive fields (|u| + sqrt(gamma p / rho) from u and p as given, not from
    the conserved variables), the constant state's closed form, and a single
    fast node among slow ones that only the nodal rule sees (the subcell
    averages blur it)."""
    o = oracle_mod.Oracle(N, cfl=0.4)
    nc = 7
    x = o.node_x(nc)
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * x)
    vel = 0.4 * np.cos(2 * np.pi * x) - 0.1
    p = 0.8 + 0.2 * np.sin(4 * np.pi * x + 0.3)
    u = W.conserved(rho, vel, p)
    expect = (np.abs(vel) + np.sqrt(1.4 * p / rho)).max()
    assert abs(o.dg_lambda_max(u, nodal=True) - expect) <= 1e-14 * expect
    o.set(cfl_mode=1)
    assert abs(o.dg_dt(u, 1.0 / nc) - 0.4 / (2 * N + 1) / nc / expect) <= 1e-15 / nc
    o.set(cfl_mode=0)
    assert abs(o.dg_dt(u, 1.0 / nc) - 0.4 / (2 * N + 1) / nc / o.dg_lambda_max(u)) <= 1e-15 / nc
    U = W.conserved(1.2, -0.3, 0.7)
    c = np.tile(U, (3, o.n, 1))
    assert abs(o.dg_lambda_max(c, nodal=True) - (0.3 + np.sqrt(1.4 * 0.7 / 1.2))) < 1e-14
    if N >= 1:
        c[1, N // 2] = W.conserved(1.2, 2.0, 0.7)  # one fast node
        assert abs(o.dg_lambda_max(c, nodal=True) - (2.0 + np.sqrt(1.4 * 0.7 / 1.2))) < 1e-14
        assert o.dg_lambda_max(c) < 2.0 + np.sqrt(1.4 * 0.7 / 1.2) - 1e-3


# ---------------------------------------------------------------------------
# DG corrector
# ---------------------------------------------------------------------------

def _brute_force_correct(o, u, q, lam):
    """Corrector of eq. ader_dg_method_full from its integrals: numpy Lagrange
    polynomials, a 30-point rule for the volume integral of the interpolated
    flux, GL weights in time for the Riemann flux (as the scheme prescribes)."""
    xi = o.table("xi")
    n = o.n
    w_time = o.table("w")  # time quadrature of the interface flux
    gx, gw = np.polynomial.legendre.leggauss(30)
    gx, gw = 0.5 * (gx + 1), 0.5 * gw
    Phi = lagrange(xi, gx)                                  # [n, 30]
    DPhi = lagrange_deriv(xi, gx)                           # [n, 30]
    mass = (Phi**2 * gw).sum(axis=1)                        # int phi_k^2
    ph0 = lagrange(xi, 0.0)[:, 0]
    ph1 = lagrange(xi, 1.0)[:, 0]
    nc = u.shape[0]
    f = lam * np_flux(q)                                    # [nc, n, n, 3]
    # volume: int_0^1 int_0^1 phi_k'(xi) f(tau, xi) dtau dxi
    f_xi = np.einsum("ctlr,lg->ctgr", f, Phi)               # interpolant at xi quad points
    f_tau = np.einsum("ctgr,tG,G->cgr", f_xi, Phi, gw)      # integrate in tau (exact)
    vol = np.einsum("cgr,kg,g->ckr", f_tau, DPhi, gw)
    qR = np.einsum("ctpr,p->ctr", q, ph1)
    qL = np.einsum("ctpr,p->ctr", q, ph0)
    G = np.einsum("ctr,t->cr", lam * np_rusanov(qR, np.roll(qL, -1, axis=0)), w_time)
    inter = ph1[None, :, None] * G[:, None, :] - ph0[None, :, None] * np.roll(G, 1, axis=0)[:, None, :]
    return u + (vol - inter) / mass[None, :, None]


@pytest.mark.parametrize("N,nc", [(1, 1), (1, 3), (2, 2), (3, 3), (5, 4), (7, 2)])
def test_dg_corrector_brute_force(oracle_mod, N, nc):
    o = oracle_mod.Oracle(N)
    rng = np.random.default_rng(10 * N + nc)
    u = W.random_state(rng, (nc, o.n))
    # arbitrary space-time coefficients near a physical state, so that every
    # trace extrapolated to xi = 0, 1 stays physical
    base = W.random_state(rng, (nc, 1, 1))
    q = base * (1 + 0.02 * rng.uniform(-1, 1, size=(nc, o.n, o.n, 3)))
    lam = 0.05
    got = o.dg_correct(u, q, dx=1.0, dt=lam).reshape(nc, o.n, 3)
    ref = _brute_force_correct(o, u, q, lam)
    assert np.all(np.isfinite(ref)) and np.all(np.isfinite(got))
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * max(1, np.abs(ref).max()))


def test_dg_N0_is_first_order_rusanov(oracle_mod):
    o = oracle_mod.Oracle(0)
    rng = np.random.default_rng(5)
    nc = 12
    u = W.random_state(rng, (nc, 1))
    dx, dt = 0.1, 0.01
    got, _, _, rc = o.dg_step(u, dx, dt)
    v = u[:, 0]
    G = np_rusanov(v, np.roll(v, -1, axis=0))
    expect = v - dt / dx * (G - np.roll(G, 1, axis=0))
    assert rc == 0
    np.testing.assert_allclose(got.reshape(nc, 3), expect, rtol=0, atol=1e-14)


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7])
def test_dg_step_conserves_mass_momentum_energy(oracle_mod, N):
    o = oracle_mod.Oracle(N)
    nc = 16
    f = W.Field1D(rho_amp=np.array([0.3, 0.1]), rho_phase=np.array([0.4, 2.0]),
                  rho_k=np.array([1.0, 3.0]), u=0.6, p_amp=np.array([0.2]),
                  p_phase=np.array([1.0]), p_k=np.array([2.0]))
    u = W.nodal_state(f, o.node_x(nc))
    dx = 1.0 / nc
    dt = o.dg_dt(u, dx)
    w = o.table("w")
    total = lambda a: dx * np.einsum("ckr,k->r", a.reshape(nc, o.n, 3), w)
    un, _, st, rc = o.dg_step(u, dx, dt)
    assert rc == 0
    np.testing.assert_allclose(total(un), total(u), rtol=2e-15, atol=0)
    # and the update is not trivial
    assert np.abs(un.ravel() - u.ravel()).max() > 1e-4


@pytest.mark.parametrize("N", [1, 4, 7])
def test_dg_free_stream(oracle_mod, N):
    o = oracle_mod.Oracle(N)
    U = W.conserved(0.9, 0.4, 1.1)
    u = np.tile(U, (8, o.n, 1))
    un, _, _, rc = o.dg_step(u, 0.125, 0.01)
    np.testing.assert_allclose(un.reshape(u.shape), u, rtol=0, atol=2e-14)


@pytest.mark.parametrize("N,cells", [(1, [20, 40, 80]), (2, [25, 50, 100]), (3, [10, 20, 40]),
                                     (4, [8, 16, 32])])
def test_dg_convergence_order(oracle_mod, N, cells):
    # Table conv_orders_pde_2d: empirical orders N+1 on the advected sine wave
    o = oracle_mod.Oracle(N)
    f = W.sine()
    errs = []
    for nc in cells:
        u = W.nodal_state(f, o.node_x(nc))
        uu, steps, t, rc = o.solve("dg", u, 1.0 / nc, t_end=1.0)
        assert rc == 0 and t == 1.0
        errs.append(oracle_mod.dg_density_errors(o, uu, lambda x: f.rho(x, 1.0))[0])
    orders = [oracle_mod.order(errs[i], errs[i + 1], 1 / cells[i], 1 / cells[i + 1])
              for i in range(len(cells) - 1)]
    assert abs(orders[-1] - (N + 1)) < 0.2, orders


def test_dg_high_degree_reaches_round_off(oracle_mod):
    o = oracle_mod.Oracle(7)
    f = W.sine()
    nc = 20
    u = W.nodal_state(f, o.node_x(nc))
    uu, steps, t, rc = o.solve("dg", u, 1.0 / nc, t_end=1.0)
    l1, linf = oracle_mod.dg_density_errors(o, uu, lambda x: f.rho(x, 1.0))
    assert l1 < 1e-12 and linf < 1e-11


# ---------------------------------------------------------------------------
# WENO
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N", [2, 4, 6])
def test_weno_reproduces_polynomials(oracle_mod, N):
    o = oracle_mod.Oracle(N)
    nc = 3 * N + 4
    rng = np.random.default_rng(N)
    c = rng.uniform(-1, 1, size=N + 1)
    c[0] = 3.0
    P = np.poly1d(c[::-1])
    Pint = P.integ()
    # cell j = [j, j+1] in units of the cell size; cell averages of P
    edges = np.arange(nc + 1, dtype=float)
    avg = Pint(edges[1:]) - Pint(edges[:-1])
    v = np.stack([avg, 0.5 * avg, 2 * avg], axis=-1)
    xi = o.table("xi")
    # interior cell far from the periodic seam: all stencils see the polynomial
    i = nc // 2
    w, om = o.weno_cell(v, i)
    np.testing.assert_allclose(w[:, 0], P(i + xi), rtol=0, atol=1e-10 * np.abs(P(i + xi)).max())
    np.testing.assert_allclose(w[:, 1], 0.5 * P(i + xi), rtol=0, atol=1e-10 * np.abs(P(i + xi)).max())


@pytest.mark.parametrize("N", [2, 4])
def test_weno_conserves_cell_average_and_linear_weights(oracle_mod, N):
    o = oracle_mod.Oracle(N)
    rng = np.random.default_rng(1)
    v = W.random_state(rng, (20,))
    wr = o.weno_reconstruct(v)
    np.testing.assert_allclose(np.einsum("ckr,k->cr", wr, o.table("w")), v, rtol=1e-13)
    # constant data: every stencil reproduces the constant; a component that is
    # exactly zero has sigma = 0 in floating point too, so its weights are the
    # normalised linear weights (other components carry round-off in sigma that
    # is comparable with eps = 1e-14, which moves weights but not the result)
    vc = np.tile(W.conserved(1.0, 0.0, 2.0), (20, 1))
    wc, om = o.weno_cell(vc, 7)
    np.testing.assert_allclose(wc, np.broadcast_to(vc[0], wc.shape), rtol=1e-13, atol=0)
    lin = np.array([1e5, 1.0, 1.0])
    np.testing.assert_allclose(om[:, 1], lin / lin.sum(), rtol=1e-14)


@pytest.mark.parametrize("N", [2, 4, 6])
def test_weno_smoothness_closed_forms(oracle_mod, N):
    o = oracle_mod.Oracle(N)
    xi = o.table("xi")
    sig = np.array([[o.weno.sig[k][l] for l in range(o.n)] for k in range(o.n)])
    # sigma = sum_a int_0^1 (p^(a))^2:  p = xi -> 1;  p = xi^2 -> 4/3 + 4;
    # p = xi^3 -> 9/5 + 12 + 36 (N >= 3); constants -> 0
    cases = [(xi, 1.0), (xi**2, 4.0 / 3.0 + 4.0)]
    if N >= 3:
        cases.append((xi**3, 9.0 / 5.0 + 12.0 + 36.0))
    for c, expect in cases:
        assert abs(o.weno_sigma(c) - expect) < 1e-12 * expect
        # the assembled matrix form agrees up to its (larger) cancellation error
        assert abs(c @ sig @ c - expect) < 1e-8 * np.abs(sig).max()
    assert o.weno_sigma(np.full(o.n, 3.0)) < 1e-18  # far below eps = 1e-14


def test_weno_avoids_the_discontinuity(oracle_mod):
    o = oracle_mod.Oracle(4)
    nc = 30
    v = np.tile(W.conserved(1.0, 0.0, 2.5), (nc, 1))
    v[15:] = W.conserved(0.125, 0.0, 0.25)
    # cell 13: the right-biased stencil {13..17} and the central {11..15} cross the jump
    _, om = o.weno_cell(v, 13)
    assert om[1, 0] > 0.99 and om[0, 0] < 1e-6 and om[2, 0] < 1e-6


def test_weno_fv_order_five(oracle_mod):
    o = oracle_mod.Oracle(4)
    f = W.sine()
    cells = [20, 40, 80]
    errs = []
    for nc in cells:
        v = W.cell_average_state(f, nc)
        vv, s, t, rc = o.solve("fv", v, 1.0 / nc, t_end=1.0)
        assert rc == 0
        errs.append(oracle_mod.fv_density_errors(vv, lambda a, b: f.rho_avg(a, b, 1.0))[0])
    assert abs(oracle_mod.order(errs[1], errs[2], 1 / 40, 1 / 80) - 5.0) < 0.2


def test_fv_conservation_and_free_stream(oracle_mod):
    o = oracle_mod.Oracle(4)
    rng = np.random.default_rng(2)
    v = W.cell_average_state(W.modes4(), 40)
    v = v * (1 + 0.1 * rng.uniform(-1, 1, size=v.shape))
    dx = 1 / 40
    vn, st, rc = o.fv_step(v, dx, o.fv_dt(v, dx))
    np.testing.assert_allclose(vn.reshape(-1, 3).sum(0), v.sum(0), rtol=2e-15)
    vc = np.tile(W.conserved(0.9, -0.4, 1.1), (16, 1))
    vn, _, _ = o.fv_step(vc, 1 / 16, 0.005)
    np.testing.assert_allclose(vn.reshape(vc.shape), vc, rtol=0, atol=2e-14)


# ---------------------------------------------------------------------------
# sampled-cell variants agree with the full-mesh step; time loop clips to t_end
# ---------------------------------------------------------------------------

def test_cell_sampled_steps_match_full(oracle_mod):
    o = oracle_mod.Oracle(3)
    f = W.modes4()
    nc = 24
    u = W.nodal_state(f, o.node_x(nc))
    dx = 1 / nc
    dt = o.dg_dt(u, dx)
    full, _, _, _ = o.dg_step(u, dx, dt)
    cells = np.array([0, 5, 23])
    sel, rc = o.dg_step_cells(u, dx, dt, cells)
    np.testing.assert_array_equal(sel, full.reshape(nc, o.n, 3)[cells])
    o4 = oracle_mod.Oracle(4)
    v = W.cell_average_state(f, nc)
    dt = o4.fv_dt(v, dx)
    full, _, _ = o4.fv_step(v, dx, dt)
    sel, rc = o4.fv_step_cells(v, dx, dt, cells)
    np.testing.assert_array_equal(sel, full.reshape(nc, 3)[cells])


def test_solve_clips_last_step(oracle_mod):
    o = oracle_mod.Oracle(2)
    U = W.conserved(1.0, 1.0, 1.0)
    nc = 10
    u = np.tile(U, (nc, o.n, 1))
    dt = o.dg_dt(u, 1 / nc)
    t_end = 7.5 * dt
    _, steps, t, rc = o.solve("dg", u, 1 / nc, t_end=t_end)
    assert rc == 0 and steps == 8 and t == t_end
    _, steps, t, rc = o.solve("dg", u, 1 / nc, max_steps=5)
    assert steps == 5 and abs(t - 5 * dt) < 1e-15


def test_nonphysical_state_is_reported(oracle_mod):
    o = oracle_mod.Oracle(2)
    u = np.tile(W.conserved(1.0, 0.0, 1.0), (4, o.n, 1))
    u[2, 1, 0] = -1.0
    _, steps, t, rc = o.solve("dg", u, 0.25, max_steps=3)
    assert rc == oracle_mod.OB_ERR_NONPHYSICAL and steps == 0
