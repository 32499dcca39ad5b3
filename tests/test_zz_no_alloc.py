"""ader_step_noalloc: the one-step entry point for callers that cannot allocate
device memory (and so cannot bind the workspace every other entry point needs).
Its scratch is the library's static device array; its result must equal
ader_step's on the same input, on two calls in a row (the second call reuses
the array the first one left behind).  This file is collected last."""
import numpy as np
import pytest

import workloads as W
from conftest import rel_linf

pytestmark = pytest.mark.gpu


def _state(scheme, N, nc):
    x = (np.arange(nc)[:, None] + (np.arange(N + 1)[None, :] + 0.5) / (N + 1)) / nc
    f = W.Field1D(rho_amp=np.array([0.1, 0.05]), rho_phase=np.array([0.3, 1.1]),
                  rho_k=np.array([1.0, 3.0]), u=0.7, p_amp=np.array([0.08]),
                  p_phase=np.array([2.0]), p_k=np.array([2.0]))
    if scheme == "dg":
        return W.nodal_state(f, x)
    return W.cell_average_state(f, nc)


@pytest.mark.parametrize("scheme,N,nc", [("dg", 5, 1003), ("dg", 7, 29126), ("dg", 0, 77),
                                         ("fv", 4, 4099)])
def test_noalloc_step_matches_step_twice(cuda, scheme, N, nc):
    import torch
    from paper_2409_12483_gb300 import Context
    from paper_2409_12483_gb300.capi import NoAllocStep
    u0 = torch.tensor(_state(scheme, N, nc), device=cuda).reshape(-1).contiguous()
    ref_ctx = Context(nc, N, scheme)
    dt = ref_ctx.ader_compute_dt(u0)
    a_ref = torch.empty_like(u0)
    b_ref = torch.empty_like(u0)
    ref_ctx.ader_step(u0, a_ref, dt)
    ref_ctx.ader_step(a_ref, b_ref, dt)
    stepper = NoAllocStep(nc, N, scheme)
    a = torch.full_like(u0, float("nan"))
    b = torch.full_like(u0, float("nan"))
    stepper.step(u0, a, dt)
    stepper.step(a, b, dt)
    torch.cuda.synchronize()
    assert rel_linf(a.cpu().numpy(), a_ref.cpu().numpy()) < 1e-12
    assert rel_linf(b.cpu().numpy(), b_ref.cpu().numpy()) < 1e-12
    assert np.abs(b.cpu().numpy() - u0.cpu().numpy()).max() > 0.0


def test_noalloc_rejects_meshes_beyond_the_static_scratch(cuda):
    import torch
    from paper_2409_12483_gb300 import ADER_ERR_ARG, AderError
    from paper_2409_12483_gb300.capi import NoAllocStep
    nc = 38836  # one cell more than fits at N = 5
    stepper = NoAllocStep(nc, 5, "dg")
    u = torch.ones(stepper.state_count, dtype=torch.float64, device=cuda)
    with pytest.raises(AderError) as e:
        stepper.step(u, torch.empty_like(u), 1e-6)
    assert e.value.status == ADER_ERR_ARG and "static scratch" in str(e.value)
    ok = NoAllocStep(nc - 1, 5, "dg")  # the largest mesh that fits is accepted
    u = torch.tensor(_state("dg", 5, nc - 1), device=cuda).reshape(-1).contiguous()
    out = torch.empty_like(u)
    ok.step(u, out, 1e-7)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()


@pytest.mark.parametrize("prec,kw", [("fp32", {"fp64_sweeps": 2}), ("ff", {})])
def test_noalloc_step_other_precisions(cuda, prec, kw):
    """The FP32-predictor and float-float forms through the no-alloc step equal
    the same forms through ader_step (same kernels, same inputs)."""
    import torch
    from paper_2409_12483_gb300 import Context
    from paper_2409_12483_gb300.capi import NoAllocStep
    N, nc = 5, 2011
    u0 = torch.tensor(_state("dg", N, nc), device=cuda).reshape(-1).contiguous()
    ref_ctx = Context(nc, N, "dg", precision=prec, **kw)
    dt = ref_ctx.ader_compute_dt(u0)
    a_ref = torch.empty_like(u0)
    ref_ctx.ader_step(u0, a_ref, dt)
    stepper = NoAllocStep(nc, N, "dg", precision=prec, **kw)
    a = torch.full_like(u0, float("nan"))
    b = torch.full_like(u0, float("nan"))
    stepper.step(u0, a, dt)
    stepper.step(u0, b, dt)
    torch.cuda.synchronize()
    assert rel_linf(a.cpu().numpy(), a_ref.cpu().numpy()) < 1e-12
    assert rel_linf(b.cpu().numpy(), a_ref.cpu().numpy()) < 1e-12


def test_noalloc_reports_the_iteration_cap(cuda):
    """A step whose Picard iteration hits the cap returns ADER_ERR_NOT_CONVERGED
    (the state is still written and equals ader_step's); the next, uncapped step
    on the same static array returns OK again."""
    import torch
    from paper_2409_12483_gb300 import ADER_ERR_NOT_CONVERGED, ADER_OK, Context
    from paper_2409_12483_gb300.capi import NoAllocStep
    N, nc = 5, 300
    u0 = torch.tensor(_state("dg", N, nc), device=cuda).reshape(-1).contiguous()
    capped = dict(picard_max_iter=1, picard_tol=1e-15)
    ref_ctx = Context(nc, N, "dg", **capped)
    dt = 4.0 * ref_ctx.ader_compute_dt(u0)
    a_ref = torch.empty_like(u0)
    ref_ctx.ader_step(u0, a_ref, dt)
    assert ref_ctx.ader_get_stats()["status"] == ADER_ERR_NOT_CONVERGED
    stepper = NoAllocStep(nc, N, "dg", **capped)
    a = torch.full_like(u0, float("nan"))
    rc = stepper.step(u0, a, dt, allow=(ADER_ERR_NOT_CONVERGED,))
    assert rc == ADER_ERR_NOT_CONVERGED
    assert rel_linf(a.cpu().numpy(), a_ref.cpu().numpy()) < 1e-12
    ok = NoAllocStep(nc, N, "dg")
    assert ok.step(u0, a, dt / 4.0) == ADER_OK


def test_noalloc_reports_a_nonphysical_result(cuda):
    """A state with negative pressure in one cell gives ADER_ERR_NONPHYSICAL."""
    import numpy as np
    import torch
    from paper_2409_12483_gb300 import ADER_ERR_NONPHYSICAL
    from paper_2409_12483_gb300.capi import NoAllocStep
    N, nc = 3, 64
    u = _state("dg", N, nc).reshape(nc, N + 1, 3).copy()
    u[10, :, 2] = 0.5 * u[10, :, 1] ** 2 / u[10, :, 0] - 0.1  # E below the kinetic energy
    ud = torch.tensor(u, device=cuda).reshape(-1).contiguous()
    stepper = NoAllocStep(nc, N, "dg")
    out = torch.empty_like(ud)
    rc = stepper.step(ud, out, 1e-4, allow=(ADER_ERR_NONPHYSICAL,))
    assert rc == ADER_ERR_NONPHYSICAL
    assert np.isfinite(out.cpu().numpy()[: 9 * (N + 1) * 3]).all()
