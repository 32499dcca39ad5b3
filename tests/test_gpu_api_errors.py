"""Error behaviour of the entry points added for the multi-D, limiter and
tracer paths: each refuses what it does not support with ADER_ERR_ARG and a
message, and the context stays usable."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_one_d_only_calls_refuse_multi_d_contexts(cuda):
    import torch
    from paper_2409_12483_gb300 import ADER_ERR_ARG, AderError, Context2D, Context3D
    for ctx in (Context2D(3, 2, 2), Context3D(2, 2, 2, 1)):
        u = torch.zeros(ctx.state_count, dtype=torch.float64, device="cuda")
        q = torch.zeros(ctx.predictor_count, dtype=torch.float64, device="cuda")
        with pytest.raises(AderError) as e:
            ctx.ader_predict(u, 0.001, q)
        assert e.value.status == ADER_ERR_ARG and "1D" in str(e.value)
        with pytest.raises(AderError) as e:
            ctx.ader_correct(u, q, 0.001, torch.zeros_like(u))
        assert e.value.status == ADER_ERR_ARG
        with pytest.raises(AderError) as e:
            ctx.ader_get_troubled(torch.zeros(ctx.n_cells, dtype=torch.int32, device="cuda"))
        assert e.value.status == ADER_ERR_ARG
        # still usable: a uniform state steps to itself
        one = np.ones(ctx.state_shape())
        one[..., -1] = 2.5
        ud = torch.tensor(one.ravel(), device="cuda")
        out = torch.empty_like(ud)
        ctx.ader_step(ud, out, 0.0)
        torch.cuda.synchronize()
        assert torch.allclose(out, ud, rtol=0, atol=1e-14)


def test_troubled_flags_need_the_limiter(cuda):
    import torch
    from paper_2409_12483_gb300 import ADER_ERR_ARG, AderError, Context
    ctx = Context(16, 3, "dg")
    with pytest.raises(AderError) as e:
        ctx.ader_get_troubled()
    assert e.value.status == ADER_ERR_ARG and "limiter" in str(e.value)
    lim = Context(16, 3, "dg", limiter=1)
    with pytest.raises(AderError):
        lim.ader_get_troubled(torch.zeros(15, dtype=torch.int32, device="cuda"))


def test_tracer_predict_is_refused_but_step_works(cuda):
    """the tracer system runs through ader_step / ader_solve only (its predictor
    is not exposed on its own)"""
    import torch
    from paper_2409_12483_gb300 import ADER_ERR_ARG, AderError, Context
    ctx = Context(8, 2, "dg", system="tracer")
    x = ctx.node_coords()
    u = np.stack([np.ones_like(x), 0.5 * np.ones_like(x), 2.5 + 0.125 * np.ones_like(x),
                  np.cos(2 * np.pi * x)], -1)
    ud = torch.tensor(u.ravel(), device="cuda")
    q = torch.zeros(ctx.predictor_count, dtype=torch.float64, device="cuda")
    with pytest.raises(AderError) as e:
        ctx.ader_predict(ud, 0.001, q)
    assert e.value.status == ADER_ERR_ARG
    out = torch.empty_like(ud)
    ctx.ader_step(ud, out, 0.0)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
