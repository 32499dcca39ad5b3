"""Pins of the oracle's ADER-DG scheme with a non-conservative product (eq.
pde_src with B != 0): the 1D Euler equations carrying a passive tracer phi in
non-conservative form, B(U) dU/dx = (0, 0, 0, u dphi/dx); nested Picard
predictor with b = (dt/dx) B(q) D^xi q in the inner loop (Algorithm
lst_dg_predictor:supp_2), the B volume term of eq. ader_dg_method_full and a
path-conservative Rusanov face (G +- Bt/2).

Independent pins: with u = 1 everywhere the non-conservative tracer equation is
the conservative equation of rho, so a tracer started equal to rho stays equal
to it through the scheme's different terms (a dropped half of the path term or
of the volume term breaks it); a constant tracer stays constant in any flow;
the converged predictor solves the Kronecker-assembled system K^tau q + K^xi f
+ M b(q) = F^0 u with b built from the derivative table (not k~); the path
integral is exact where u is constant or linear along the segment and matches
the closed-form integral otherwise; Euler components do not see the tracer."""
import numpy as np
import pytest

GAMMA = 1.4


def state(o, nc, phi_fn=None, u_fn=None, seed=0):
    x = o.node_x(nc)
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.05, 0.2, 3)
    rho = 1 + a[0] * np.sin(2 * np.pi * x + 0.4)
    u = u_fn(x) if u_fn else 0.7 + a[1] * np.cos(2 * np.pi * x)
    p = 1 + a[2] * np.sin(4 * np.pi * x)
    phi = phi_fn(x, rho) if phi_fn else 0.5 + 0.3 * np.cos(2 * np.pi * x)
    return np.stack([rho, rho * u, p / (GAMMA - 1) + 0.5 * rho * u * u, phi], -1)


def test_face_path_integral(oracle_mod):
    o = oracle_mod.NCOracle(1)
    # constant u along the segment: Bt = u (phi+ - phi-) exactly
    a = np.array([1.0, 0.5, 3.0, 0.2])
    b = np.array([2.0, 1.0, 4.0, 0.9])
    G, bt = o.face(a, b)
    assert bt == pytest.approx(0.5 * 0.7, rel=1e-15)
    # rho constant, m linear: u linear in s, the 3-point rule is exact
    b2 = np.array([1.0, 1.1, 3.5, -0.4])
    _, bt = o.face(a, b2)
    assert bt == pytest.approx(0.5 * (0.5 + 1.1) * (-0.6), rel=1e-14)
    # general segment: the closed form int_0^1 (m0 + s dm) / (r0 + s dr) ds
    b3 = np.array([1.6, -0.3, 3.2, 1.3])
    _, bt = o.face(a, b3)
    r0, dr, m0, dm = a[0], b3[0] - a[0], a[1], b3[1] - a[1]
    exact = dm / dr + (m0 * dr - dm * r0) / dr ** 2 * np.log((r0 + dr) / r0)
    assert bt == pytest.approx(exact * (b3[3] - a[3]), rel=1e-4)
    # the Rusanov part: the Euler flux and no conservative flux of phi, so its phi
    # component is the dissipation alone, with the speed s read off the rho part
    Fa, Fb = o.flux(a), o.flux(b)
    assert Fa[3] == 0.0 and Fb[3] == 0.0
    s = (0.5 * (Fa[0] + Fb[0]) - G[0]) * 2 / (b[0] - a[0])
    assert s > 0
    assert G[3] == pytest.approx(-0.5 * s * (b[3] - a[3]), rel=1e-13)


@pytest.mark.parametrize("N", range(0, 6))
def test_tracer_equal_to_rho_in_uniform_flow(oracle_mod, N):
    """u = 1, p = 1, phi = rho: the tracer's non-conservative update reproduces the
    conservative update of rho over 20 steps"""
    o = oracle_mod.NCOracle(N)
    nc = 12
    U = state(o, nc, phi_fn=lambda x, rho: rho, u_fn=lambda x: np.ones_like(x))
    U[..., 2] = 1 / (GAMMA - 1) + 0.5 * U[..., 0]
    out, steps, t, rc = o.solve(U, 1.0 / nc, max_steps=20)
    assert rc == 0 and steps == 20
    out = out.reshape(nc, N + 1, 4)
    assert np.abs(out[..., 3] - out[..., 0]).max() < 1e-12
    assert np.abs(out[..., 0] - U[..., 0]).max() > 1e-3  # the wave did move


def test_constant_tracer_stays_constant(oracle_mod):
    o = oracle_mod.NCOracle(3)
    nc = 10
    U = state(o, nc, phi_fn=lambda x, rho: 0.37 + 0 * x)
    out, steps, t, rc = o.solve(U, 1.0 / nc, max_steps=15)
    assert rc == 0
    np.testing.assert_allclose(out.reshape(nc, 4, 4)[..., 3], 0.37, rtol=0, atol=1e-14)


def test_euler_part_is_the_euler_scheme(oracle_mod):
    """the tracer does not act on rho, m, E: their step equals the Euler oracle's"""
    N, nc = 4, 9
    o = oracle_mod.NCOracle(N)
    U = state(o, nc, seed=3)
    dt = o.dt(U, 1.0 / nc)
    out, rc, _ = o.step(U, 1.0 / nc, dt)
    ref = o.base.dg_step(np.ascontiguousarray(U[..., :3]), 1.0 / nc, dt)[0]
    assert rc == 0
    np.testing.assert_allclose(out.reshape(nc, N + 1, 4)[..., :3], ref.reshape(nc, N + 1, 3),
                               rtol=0, atol=1e-14)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_predictor_solves_the_kronecker_system(oracle_mod, N):
    o = oracle_mod.NCOracle(N, tol=1e-15, max_iter=200)
    n = N + 1
    U = state(o, 1, seed=N)[0]
    lam = 0.06
    q, it, rc = o.predict_cell(U, lam)
    assert rc == 0
    Ups, Lam, Xi, psi0, dphi = (o.table(t) for t in ("ups", "lam", "xi_m", "psi0", "dphi"))
    F = np.array([[lam * o.flux(q[a, c]) for c in range(n)] for a in range(n)])
    # b: (dt/dx) u (d phi / d xi) at every node, the derivative from phi_k'(xi_l)
    dq = np.einsum("kl,akr->alr", dphi, q)
    b = np.zeros_like(q)
    b[..., 3] = lam * q[..., 1] / q[..., 0] * dq[..., 3]
    res = (np.kron(Ups, Lam) @ q.reshape(-1, 4) + np.kron(Lam, Xi) @ F.reshape(-1, 4)
           + np.kron(Lam, Lam) @ b.reshape(-1, 4) - np.kron(psi0[:, None], Lam) @ U)
    assert np.abs(res).max() < 1e-13
