"""GPU parity of the outflow boundary and the a posteriori subcell limiter
(PAD / NAD on subcell averages, the ADER-WENO2 scheme on the subcells, pseudo-
inverse reconstruction; mode 2 recomputes every cell) against the oracle's
ob_dgl_* family, and the four
classical Riemann problems of Sec. 2 (Table classical_tests_1d) through the GPU
path.  Bar: 1e-12 relative L-inf per step (and the same troubled cells),
1e-10 after a solve."""
import numpy as np
import pytest

import workloads as W
from conftest import rel_linf
from test_gpu_dg import NCELLS, field_nonlinear, to_dev
from test_oracle_limiter import conserved, riemann_state

pytestmark = pytest.mark.gpu


def make(nc, N, **kw):
    from paper_2409_12483_gb300 import Context
    return Context(nc, N, "dg", **kw)


@pytest.mark.parametrize("N", range(0, 8))
def test_outflow_step_parity(cuda, oracle_mod, N):
    import torch
    o = oracle_mod.Oracle(N)
    u = W.nodal_state(field_nonlinear(50 + N), o.node_x(NCELLS))
    dx = 1.0 / NCELLS
    dt = o.dg_dt(u, dx)
    ref, tr, rc = o.dgl_step(u, dx, dt, bc="outflow", limiter=False)
    assert rc == 0
    ctx = make(NCELLS, N, bc="outflow")
    ud = to_dev(u, cuda)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, dt)
    torch.cuda.synchronize()
    assert rel_linf(out.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("N", range(1, 8))
@pytest.mark.parametrize("test", [1, 2])
def test_limited_step_parity(cuda, oracle_mod, N, test):
    """one step on the Sod / Lax data: the same cells are troubled and the
    limited state matches"""
    import torch
    o = oracle_mod.Oracle(N)
    nc = 64
    u = riemann_state(o, nc, test)
    dx = 1.0 / nc
    dt = o.dg_dt(u, dx)
    ref, tr, rc = o.dgl_step(u, dx, dt, bc="outflow", limiter=True)
    assert rc == 0 and tr.any()
    ctx = make(nc, N, bc="outflow", limiter=1)
    ud = to_dev(u, cuda)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, dt)
    flags = ctx.ader_get_troubled().cpu().numpy()
    torch.cuda.synchronize()
    assert ctx.ader_get_stats()["troubled_cells"] == int(tr.sum())
    np.testing.assert_array_equal(flags, tr)
    assert rel_linf(out.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("test", [1, 2, 3, 4])
def test_riemann_problem_solve_parity(cuda, oracle_mod, test):
    """DG N = 3, 100 cells, outflow, limiter, to t_final = 0.15: the full solves
    take the same steps, limit the same cells and agree to 1e-11 at the end
    (measured 5e-15 .. 5e-14 over 574 .. 1238 steps), and 50-step segments
    started from common states along the trajectory agree to 1e-11."""
    import torch
    N, nc = 3, 100
    o = oracle_mod.Oracle(N)
    u = riemann_state(o, nc, test)
    ref, steps_ref, t_ref, rc, ttot = o.dgl_solve(u, 1.0 / nc, t_end=0.15, bc="outflow",
                                                  limiter=True)
    assert rc == 0
    ctx = make(nc, N, bc="outflow", limiter=1)
    ud = to_dev(u, cuda)
    steps, t, rc = ctx.ader_solve(ud, t_end=0.15)
    torch.cuda.synchronize()
    got = ud.cpu().numpy()
    assert steps == steps_ref and t == 0.15
    assert ctx.ader_get_stats()["troubled_cells"] == ttot
    assert rel_linf(got, ref) < 1e-11
    # segment parity from common states along the trajectory
    seg = make(nc, N, bc="outflow", limiter=1)
    g = to_dev(u, cuda)
    for _ in range(steps_ref // 50):
        start = g.cpu().numpy()
        ref_seg, _, _, rc, _ = o.dgl_solve(start, 1.0 / nc, max_steps=50, bc="outflow", limiter=True)
        seg.ader_solve(g, max_steps=50)
        torch.cuda.synchronize()
        assert rel_linf(g.cpu().numpy(), ref_seg) < 1e-11


def test_limiter_leaves_smooth_solutions_alone(cuda, oracle_mod):
    import torch
    N, nc = 3, 120
    o = oracle_mod.Oracle(N)
    u = W.nodal_state(W.sine(), o.node_x(nc))
    a = to_dev(u, cuda)
    b = to_dev(u, cuda)
    lim = make(nc, N, limiter=1)
    plain = make(nc, N)
    s1, t1, _ = lim.ader_solve(a, max_steps=40)
    s2, t2, _ = plain.ader_solve(b, max_steps=40)
    torch.cuda.synchronize()
    assert lim.ader_get_stats()["troubled_cells"] == 0
    assert s1 == s2 and t1 == t2
    assert rel_linf(a.cpu().numpy(), b.cpu().numpy()) < 1e-14


def test_limited_periodic_solve_is_conservative(cuda, oracle_mod):
    import torch
    N, nc = 4, 80
    o = oracle_mod.Oracle(N)
    x = o.node_x(nc)
    inside = (x > 0.25) & (x < 0.75)
    u = conserved(np.where(inside, 1.0, 0.125), np.zeros(x.shape), np.where(inside, 1.0, 0.1))
    ctx = make(nc, N, limiter=1)
    ud = to_dev(u, cuda)
    steps, t, rc = ctx.ader_solve(ud, max_steps=60)
    torch.cuda.synchronize()
    assert rc == 0 and ctx.ader_get_stats()["troubled_cells"] > 0
    w = o.table("w")
    tot = lambda U: np.einsum("ckr,k->r", U.reshape(nc, N + 1, 3), w) / nc
    np.testing.assert_allclose(tot(ud.cpu().numpy()), tot(u), rtol=2e-14, atol=2e-15)


def density_wave(o, nc):
    x = o.node_x(nc)
    return conserved(1 + 0.2 * np.sin(2 * np.pi * x), np.ones(x.shape), np.ones(x.shape))


@pytest.mark.parametrize("N", range(1, 8))
@pytest.mark.parametrize("fixed", [0, 3])
def test_every_cell_on_subcells_step_parity(cuda, oracle_mod, N, fixed):
    """limiter 2: every cell recomputed by the subcell ADER-WENO2 scheme (the
    degree-1 predictor in tolerance and in fixed-iteration mode); periodic jump
    data and outflow Lax data"""
    import torch
    nc = 48
    o = oracle_mod.Oracle(N, fixed_iter=fixed)
    x = o.node_x(nc)
    inside = (x > 0.25) & (x < 0.625)
    cases = (("periodic", conserved(np.where(inside, 1.0, 0.125), np.where(inside, 0.4, 0.0),
                                    np.where(inside, 1.0, 0.1))),
             ("outflow", riemann_state(o, nc, 2)))
    for bc, u in cases:
        dt = o.dg_dt(u, 1.0 / nc)
        ref, tr, rc = o.dgl_step(u, 1.0 / nc, dt, bc=bc, limiter=2)
        assert rc == 0 and tr.all()
        ctx = make(nc, N, bc=bc, limiter=2, picard_fixed_iter=fixed)
        ud = to_dev(u, cuda)
        out = torch.empty_like(ud)
        ctx.ader_step(ud, out, dt)
        torch.cuda.synchronize()
        assert ctx.ader_get_stats()["troubled_cells"] == nc
        assert rel_linf(out.cpu().numpy(), ref) < 1e-12, bc


@pytest.mark.parametrize("N", [1, 2, 5])
def test_every_cell_on_subcells_solve_parity(cuda, oracle_mod, N):
    """limiter 2 on the smooth density wave to t = 0.25 (periodic): the GPU and
    the oracle agree to 1e-10 after the solve"""
    import torch
    nc = 32
    o = oracle_mod.Oracle(N)
    u = density_wave(o, nc)
    ref, steps_ref, t_ref, rc, ttot = o.dgl_solve(u, 1.0 / nc, t_end=0.25, limiter=2)
    assert rc == 0
    ctx = make(nc, N, limiter=2)
    ud = to_dev(u, cuda)
    steps, t, rc = ctx.ader_solve(ud, t_end=0.25)
    torch.cuda.synchronize()
    assert rc == 0 and steps == steps_ref and t == 0.25
    assert ctx.ader_get_stats()["troubled_cells"] == ttot == nc * steps
    assert rel_linf(ud.cpu().numpy(), ref) < 1e-10


@pytest.mark.parametrize("N", [2, 5])
@pytest.mark.parametrize("delta0,eps", [(0.0, 0.0), (1e-9, 1e-6), (1e-4, 1e-3)])
def test_nad_decisions_near_the_threshold(cuda, oracle_mod, N, delta0, eps):
    """smooth data with a strict or tight discrete maximum principle: many
    subcell averages sit at the edge of the NAD interval, where the FP32 screen
    must hand the decision to the FP64 detectors; the troubled cells are the
    oracle's exactly"""
    import torch
    o = oracle_mod.Oracle(N)
    nc = 64
    u = W.nodal_state(field_nonlinear(80 + N), o.node_x(nc))
    dx = 1.0 / nc
    dt = o.dg_dt(u, dx)
    ref, tr, rc = o.dgl_step(u, dx, dt, limiter=True, delta0=delta0, eps=eps)
    assert rc == 0
    ctx = make(nc, N, limiter=1, nad_delta0=delta0, nad_eps=eps)
    ud = to_dev(u, cuda)
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, dt)
    flags = ctx.ader_get_troubled().cpu().numpy()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(flags, tr)
    assert rel_linf(out.cpu().numpy(), ref) < 1e-12
    if delta0 == 0.0:
        assert tr.any()  # the strict principle flags the cells at smooth extrema
