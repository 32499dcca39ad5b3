"""GPU parity of the ADER-DG path with algebraic sources (the 1D two-component
reacting flow: nested Picard predictor, corrector with the source term) against
the oracle's source-term family, plus the ODE initial-value problem of Sec. 2.1
against the (N, N+1) Pade form of DG in time.  Bar: 1e-12 relative L-inf per
step, 1e-10 after a solve."""
import numpy as np
import pytest

import workloads as W
from conftest import rel_linf
from test_gpu_dg import NCELLS, to_dev
from test_oracle_source import ODE_DX, pade_stability

pytestmark = pytest.mark.gpu
MRS = 5


def make(nc, N, **kw):
    from paper_2409_12483_gb300 import Context
    kw.setdefault("omega", 2.0)
    return Context(nc, N, "dg", system="reacting", **kw)


@pytest.mark.parametrize("N", range(0, 8))
@pytest.mark.parametrize("fixed", [False, True])
def test_predictor_parity(cuda, oracle_mod, N, fixed):
    import torch
    orc = oracle_mod.ReactingOracle(N, omega=2.0)
    u = W.reacting_state(orc.node_x(NCELLS), seed=N)
    dx = 1.0 / NCELLS
    dt = orc.dg_dt(u, dx)
    it = 4 if fixed else 0
    orc.set(fixed_iter=it)
    q_ref, iters = orc.predict(u, dt / dx, dt)
    ctx = make(NCELLS, N, picard_fixed_iter=it)
    q = torch.empty(ctx.predictor_count, dtype=torch.float64, device=cuda)
    ctx.ader_predict(to_dev(u, cuda), dt, q)
    torch.cuda.synchronize()
    assert rel_linf(q.cpu().numpy(), q_ref) < 1e-12
    st = ctx.ader_get_stats()
    assert st["status"] == 0 and st["cells"] == NCELLS
    if fixed:
        assert st["max_iters"] == it
    else:
        assert abs(st["max_iters"] - iters.max()) <= 1


@pytest.mark.parametrize("N", range(0, 8))
def test_step_parity(cuda, oracle_mod, N):
    import torch
    orc = oracle_mod.ReactingOracle(N, omega=2.0)
    u = W.reacting_state(orc.node_x(NCELLS), seed=10 + N)
    dx = 1.0 / NCELLS
    dt = orc.dg_dt(u, dx)
    ref, _, _, rc = orc.dg_step(u, dx, dt)
    assert rc == 0
    ctx = make(NCELLS, N)
    ud = to_dev(u, cuda)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, 0.0)  # CFL dt on the device
    torch.cuda.synchronize()
    assert rel_linf(out.cpu().numpy(), ref) < 1e-12
    assert abs(ctx.ader_compute_dt(ud) - dt) <= 1e-14 * dt


def test_predict_then_correct_equals_step(cuda, oracle_mod):
    import torch
    N = 4
    orc = oracle_mod.ReactingOracle(N, omega=2.0)
    u = W.reacting_state(orc.node_x(NCELLS), seed=3)
    dx = 1.0 / NCELLS
    dt = orc.dg_dt(u, dx)
    ctx = make(NCELLS, N)
    ud = to_dev(u, cuda)
    q = torch.empty(ctx.predictor_count, dtype=torch.float64, device=cuda)
    ctx.ader_predict(ud, dt, q)
    a = torch.empty_like(ud)
    ctx.ader_correct(ud, q, dt, a)
    b = torch.empty_like(ud)
    ctx.ader_step(ud, b, dt)
    torch.cuda.synchronize()
    assert rel_linf(a.cpu().numpy(), b.cpu().numpy()) < 1e-14
    ref, _, _, _ = orc.dg_step(u, dx, dt)
    assert rel_linf(a.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_ode_problem_against_oracle_and_pade(cuda, oracle_mod, N):
    """Sec. 2.1 ODE problem (eq. harm_osc): one uniform cell, omega = 1, K uniform
    steps to 2 pi; the species at the time nodes equal the oracle's and the
    (N, N+1) Pade approximant of exp(dt A)."""
    import torch
    K = 9
    dt = 2 * np.pi / K
    n = N + 1
    orc = oracle_mod.ReactingOracle(N, omega=1.0, tol=1e-14, max_iter=200)
    ctx = make(1, N, omega=1.0, picard_tol=1e-14, picard_max_iter=200, x1=ODE_DX)
    u = W.ode_state(n).ravel()
    ud = to_dev(u, cuda)
    R = pade_stability(N, dt * np.array([[0.0, 1.0], [-1.0, 0.0]]))
    v = np.array([1.0, 0.0])
    for _ in range(K):
        out = torch.empty_like(ud)
        ctx.ader_step(ud, out, dt)
        ud = out
        u, _, _, rc = orc.dg_step(u, ODE_DX, dt)
        v = R @ v
    torch.cuda.synchronize()
    got = ud.cpu().numpy().reshape(n, MRS)
    np.testing.assert_allclose(got, u.reshape(n, MRS), rtol=0, atol=1e-13)
    np.testing.assert_allclose(got[:, 3:], np.tile(v, (n, 1)), rtol=0, atol=1e-13)


def test_solve_parity_and_species_balance(cuda, oracle_mod):
    import torch
    N, nc = 3, 48
    orc = oracle_mod.ReactingOracle(N, omega=2.0)
    u = W.reacting_state(orc.node_x(nc), seed=21)
    ref, steps_ref, t_ref, rc = orc.solve(u, 1.0 / nc, t_end=0.05)
    assert rc == 0
    ctx = make(nc, N)
    ud = to_dev(u, cuda)
    steps, t, rc = ctx.ader_solve(ud, t_end=0.05)
    torch.cuda.synchronize()
    assert steps == steps_ref and t == 0.05
    got = ud.cpu().numpy()
    assert rel_linf(got, ref) < 1e-10
    # mass, momentum and energy are conserved exactly by the scheme
    w = orc.table("w")
    tot0 = np.einsum("ckr,k->r", u.reshape(nc, N + 1, MRS), w) / nc
    tot1 = np.einsum("ckr,k->r", got.reshape(nc, N + 1, MRS), w) / nc
    np.testing.assert_allclose(tot1[:3], tot0[:3], rtol=1e-13)


def test_full_size_n5_sampled(cuda, oracle_mod):
    """DG N = 5, 10^5 cells, reacting system: one step on sampled cells."""
    import torch
    N, nc = 5, 100_000
    orc = oracle_mod.ReactingOracle(N, omega=2.0)
    u = W.reacting_state(orc.node_x(nc), seed=7)
    dx = 1.0 / nc
    ctx = make(nc, N)
    ud = to_dev(u, cuda)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, 0.0)
    torch.cuda.synchronize()
    dt = orc.dg_dt(u, dx)
    cells = np.unique(np.concatenate([[0, 1, nc - 1], np.random.default_rng(4).integers(0, nc, 40)]))
    sel, rc = orc.dg_step_cells(u, dx, dt, cells)
    assert rel_linf(out.cpu().numpy().reshape(nc, N + 1, MRS)[cells], sel) < 1e-12
