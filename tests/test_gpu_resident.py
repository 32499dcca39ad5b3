"""The context-resident state calls (ader_set_state, ader_get_state,
ader_get_predictor, ader_state_step, ader_state_solve: the mesh-level form of
the paper's get_cell_local_solution(u_prev) / get_dg_solution(u_prev) of Sec.
1.1 and 1.2) against the oracle: set -> step -> get at 1e-12 relative L-inf per
step, the predictor of the resident state at 1e-12, and the resident time
carried across split solves bit for bit."""
import numpy as np
import pytest

import workloads as W
from conftest import rel_linf

pytestmark = pytest.mark.gpu

NCELLS = 32 * 3 + 7


def field(seed):
    g = np.random.default_rng(seed)
    k = np.arange(1, 4, dtype=float)
    return W.Field1D(rho_amp=g.uniform(0, 0.1, 3), rho_phase=g.uniform(0, 6.28, 3), rho_k=k,
                     u=0.5, p_amp=g.uniform(0, 0.1, 3), p_phase=g.uniform(0, 6.28, 3), p_k=k)


def test_set_get_round_trip_host_and_device(cuda):
    import torch
    from paper_2409_12483_gb300 import ADER_ERR_ARG, ADER_ERR_STATE, AderError, Context
    ctx = Context(NCELLS, 3, "dg")
    u = np.random.default_rng(1).uniform(0.5, 2.0, ctx.state_count)
    with pytest.raises(AderError) as e:
        ctx.ader_get_state(on_device=False)
    assert e.value.status == ADER_ERR_STATE
    ctx.ader_set_state(u)
    assert np.array_equal(ctx.ader_get_state(on_device=False), u)
    assert ctx.ader_get_state_time() == 0.0
    ud = torch.tensor(u[::-1].copy(), device=cuda)
    ctx.ader_set_state(ud)
    out = ctx.ader_get_state()
    torch.cuda.synchronize()
    assert torch.equal(out, ud)
    with pytest.raises(ValueError):
        ctx.ader_set_state(u[:-1])
    import ctypes as C
    rc = ctx._L.ader_set_state(ctx._ctx, u.ctypes.data_as(C.c_void_p), u.size - 1, 0)
    assert rc == ADER_ERR_ARG


@pytest.mark.parametrize("N", [0, 2, 5, 7])
def test_set_step_get_matches_oracle(cuda, oracle_mod, N):
    from paper_2409_12483_gb300 import Context
    o = oracle_mod.Oracle(N)
    u = W.nodal_state(field(N), o.node_x(NCELLS))
    dx = 1.0 / NCELLS
    ctx = Context(NCELLS, N, "dg")
    ctx.ader_set_state(u)
    dt = ctx.ader_state_step()  # CFL step of the resident state
    dt_ref = o.dg_dt(u, dx)
    assert abs(dt - dt_ref) <= 1e-14 * dt_ref
    ref, _, _, rc = o.dg_step(u, dx, dt)
    assert rc == 0
    assert rel_linf(ctx.ader_get_state(on_device=False), ref) < 1e-12
    assert ctx.ader_get_state_time() == dt
    # a second, fixed step
    ctx.ader_state_step(0.5 * dt)
    ref2, _, _, _ = o.dg_step(ref, dx, 0.5 * dt)
    assert rel_linf(ctx.ader_get_state(on_device=False), ref2) < 1e-12
    assert ctx.ader_get_state_time() == dt + 0.5 * dt


@pytest.mark.parametrize("N", [1, 4, 6])
def test_resident_predictor_matches_oracle(cuda, oracle_mod, N):
    from paper_2409_12483_gb300 import Context
    o = oracle_mod.Oracle(N)
    u = W.nodal_state(field(20 + N), o.node_x(NCELLS))
    dx = 1.0 / NCELLS
    dt = o.dg_dt(u, dx)
    o.set(fixed_iter=N + 3)
    q_ref, _ = o.predict(u, dt / dx)
    ctx = Context(NCELLS, N, "dg", picard_fixed_iter=N + 3)
    ctx.ader_set_state(u)
    q = ctx.ader_get_predictor(dt)
    assert rel_linf(q.cpu().numpy(), q_ref.ravel()) < 1e-12
    q0 = ctx.ader_get_predictor(0.0)  # the CFL step: the same dt here
    assert rel_linf(q0.cpu().numpy(), q_ref.ravel()) < 1e-12
    assert np.array_equal(ctx.ader_get_state(on_device=False), u.ravel())  # state unchanged


def test_resident_solve_split_equals_one_solve_and_oracle(cuda, oracle_mod):
    """A resident solve split by max_steps continues from the resident time and
    equals one solve bit for bit; a split at an intermediate t_end (which adds a
    clipped step) matches the oracle split the same way at 1e-10."""
    import torch
    from paper_2409_12483_gb300 import Context
    N, nc = 2, 100
    o = oracle_mod.Oracle(N)
    u = W.nodal_state(W.sine(), o.node_x(nc))
    one = Context(nc, N, "dg")
    ud = torch.tensor(u.ravel(), device=cuda)
    steps, t, _ = one.ader_solve(ud, t_end=0.1)
    ref, steps_ref, t_ref, rc = o.solve("dg", u, 1.0 / nc, t_end=0.1)
    assert steps_ref == steps and rel_linf(ud.cpu().numpy(), ref) < 1e-10
    ctx = Context(nc, N, "dg")
    ctx.ader_set_state(u)
    s1, t1, _ = ctx.ader_state_solve(max_steps=7)
    assert s1 == 7 and ctx.ader_get_state_time() == t1
    s2, t2, _ = ctx.ader_state_solve(t_end=0.1)
    assert s1 + s2 == steps and t2 == t
    assert np.array_equal(ctx.ader_get_state(on_device=False), ud.cpu().numpy())
    # split at t = 0.03: one more (clipped) step on both sides
    ctx.ader_set_state(u)
    a1, _, _ = ctx.ader_state_solve(t_end=0.03)
    assert ctx.ader_get_state_time() == 0.03
    a2, _, _ = ctx.ader_state_solve(t_end=0.1)
    r1, b1, _, _ = o.solve("dg", u, 1.0 / nc, t_end=0.03)
    r2, b2, _, _ = o.solve("dg", r1, 1.0 / nc, t_end=0.1 - 0.03)
    assert (a1, a2) == (b1, b2)
    assert rel_linf(ctx.ader_get_state(on_device=False), r2) < 1e-10
    with pytest.raises(Exception):
        ctx.ader_state_solve(t_end=0.05)  # already past it


def test_fv_resident_step_matches_oracle(cuda, oracle_mod):
    from paper_2409_12483_gb300 import Context
    N, nc = 4, 133
    o = oracle_mod.Oracle(N)
    v = W.cell_average_state(field(3), nc)
    ctx = Context(nc, N, "fv")
    ctx.ader_set_state(v)
    dt = ctx.ader_state_step()
    dt_ref = o.fv_dt(v, 1.0 / nc)
    assert abs(dt - dt_ref) <= 1e-14 * dt_ref
    ref, _, rc = o.fv_step(v, 1.0 / nc, dt)
    assert rc == 0 and rel_linf(ctx.ader_get_state(on_device=False), ref) < 1e-12
