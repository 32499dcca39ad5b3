"""GPU parity of the ADER-WENO finite-volume path (WENO reconstruction, LST-DG
predictor on the reconstruction, Rusanov FV update) against the oracle."""
import numpy as np
import pytest

import workloads as W
from conftest import rel_linf

pytestmark = pytest.mark.gpu

NCELLS = 32 * 3 + 7


def to_dev(a, cuda):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=cuda)


def fv_state(nc, seed):
    g = np.random.default_rng(seed)
    k = np.arange(1, 4, dtype=float)
    f = W.Field1D(rho_amp=g.uniform(0, 0.1, 3), rho_phase=g.uniform(0, 6.28, 3), rho_k=k, u=0.5,
                  p_amp=g.uniform(0, 0.1, 3), p_phase=g.uniform(0, 6.28, 3), p_k=k)
    return W.cell_average_state(f, nc)


@pytest.mark.parametrize("N", [2, 4])
@pytest.mark.parametrize("kind", ["smooth", "jump"])
def test_weno_parity(cuda, oracle_mod, N, kind):
    import torch
    from paper_2409_12483_gb300 import Context
    o = oracle_mod.Oracle(N)
    v = fv_state(NCELLS, N)
    if kind == "jump":
        v[40:70] = W.conserved(0.125, 0.0, 0.1)
    ref = o.weno_reconstruct(v)
    ctx = Context(NCELLS, N, "fv")
    w = torch.empty(NCELLS * (N + 1) * 3, dtype=torch.float64, device=cuda)
    ctx.ader_weno_reconstruct(to_dev(v, cuda), w)
    torch.cuda.synchronize()
    assert rel_linf(w.cpu().numpy(), ref.ravel()) < 1e-12


def fronts_state(nc, kind):
    """Cell averages on a fine mesh: smooth modes, or fronts resolved over a
    few cells (where the stencil polynomials differ by amounts that put the
    FP32-weight screen near its limit) plus a jump."""
    x = (np.arange(nc) + 0.5) / nc
    if kind == "smooth":
        return W.cell_average_state(W.modes4(7), nc)
    h = 1.0 / nc
    rho = 1.0 + 0.3 * np.tanh((x - 0.2) / (3 * h)) + 0.2 * np.tanh((x - 0.45) / (10 * h))
    rho += 0.1 * np.tanh((x - 0.7) / (30 * h)) + 0.5 * (x > 0.85)
    u = 0.5 + 0.2 * np.sin(2 * np.pi * x)
    p = 1.0 + 0.05 * np.cos(4 * np.pi * x)
    return W.conserved(rho, u, p)


@pytest.mark.parametrize("N", [2, 4])
@pytest.mark.parametrize("kind", ["smooth", "fronts"])
def test_weno_parity_fine_mesh(cuda, oracle_mod, N, kind):
    """20000 cells: the screened FP32 weights are taken on smooth stretches
    (the stencil polynomials agree to ~h^(N+1)) and refused near the fronts and
    the jump; every reconstructed value agrees with the FP64 oracle to 1e-13
    (a weight error the screen let through would show at ~1e-7 of the stencil
    differences)."""
    import torch
    from paper_2409_12483_gb300 import Context
    nc = 20000
    o = oracle_mod.Oracle(N)
    v = fronts_state(nc, kind)
    ref = o.weno_reconstruct(v)
    ctx = Context(nc, N, "fv")
    w = torch.empty(nc * (N + 1) * 3, dtype=torch.float64, device=cuda)
    ctx.ader_weno_reconstruct(to_dev(v, cuda), w)
    torch.cuda.synchronize()
    got = w.cpu().numpy().reshape(nc, N + 1, 3)
    ref = np.asarray(ref).reshape(nc, N + 1, 3)
    for r in range(3):  # per variable, relative to its own scale
        scale = np.max(np.abs(ref[..., r]))
        assert np.max(np.abs(got[..., r] - ref[..., r])) <= 1e-13 * scale


@pytest.mark.parametrize("N", [2, 4])
def test_fv_predictor_and_step_parity(cuda, oracle_mod, N):
    import torch
    from paper_2409_12483_gb300 import Context
    o = oracle_mod.Oracle(N)
    v = fv_state(NCELLS, 10 + N)
    dx = 1.0 / NCELLS
    dt = o.fv_dt(v, dx)
    ctx = Context(NCELLS, N, "fv")
    vd = to_dev(v, cuda)
    q = torch.empty(ctx.predictor_count, dtype=torch.float64, device=cuda)
    ctx.ader_predict(vd, dt, q)
    q_ref, _ = o.predict(o.weno_reconstruct(v), dt / dx)
    torch.cuda.synchronize()
    assert rel_linf(q.cpu().numpy(), q_ref.ravel()) < 1e-12
    ref, st, rc = o.fv_step(v, dx, dt)
    out = torch.empty_like(vd)
    ctx.ader_step(vd, out, dt)
    torch.cuda.synchronize()
    assert rel_linf(out.cpu().numpy(), ref.ravel()) < 1e-12
    out2 = torch.empty_like(vd)
    ctx.ader_correct(vd, to_dev(q_ref, cuda), dt, out2)
    torch.cuda.synchronize()
    assert rel_linf(out2.cpu().numpy(), ref.ravel()) < 1e-12


def test_fv_solve_parity(cuda, oracle_mod):
    import torch
    from paper_2409_12483_gb300 import Context
    N, nc = 4, 80
    o = oracle_mod.Oracle(N)
    f = W.sine()
    v = W.cell_average_state(f, nc)
    ref, steps_ref, t_ref, rc = o.solve("fv", v, 1.0 / nc, t_end=0.25)
    ctx = Context(nc, N, "fv")
    vd = to_dev(v, cuda)
    steps, t, rc = ctx.ader_solve(vd, t_end=0.25)
    torch.cuda.synchronize()
    assert steps == steps_ref and t == 0.25
    assert rel_linf(vd.cpu().numpy(), ref) < 1e-10


def test_fv_full_size_sampled(cuda, oracle_mod):
    """ADER-WENO5 (N = 4), 10^6 cells: one device-CFL step on sampled cells."""
    import torch
    from paper_2409_12483_gb300 import Context
    N, nc = 4, 1_000_000
    o = oracle_mod.Oracle(N)
    v = W.cell_average_state(W.modes4(), nc)
    dx = 1.0 / nc
    ctx = Context(nc, N, "fv")
    vd = to_dev(v, cuda)
    out = torch.empty_like(vd)
    ctx.ader_step(vd, out, 0.0)
    torch.cuda.synchronize()
    dt = o.fv_dt(v, dx)
    cells = np.unique(np.concatenate([[0, 1, 2, nc - 1, nc - 3],
                                      np.random.default_rng(1).integers(0, nc, 40)]))
    sel, rc = o.fv_step_cells(v, dx, dt, cells)
    assert rel_linf(out.cpu().numpy().reshape(nc, 3)[cells], sel) < 1e-12
    mass0 = v.sum(0)
    steps, t, rc = ctx.ader_solve(vd, max_steps=20)
    torch.cuda.synchronize()
    np.testing.assert_allclose(vd.cpu().numpy().reshape(nc, 3).sum(0), mass0, rtol=1e-13)
