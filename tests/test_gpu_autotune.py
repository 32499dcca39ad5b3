"""Autotuned launch shapes change speed, not results: every tile shape computes
each cell with the same arithmetic, so results are identical."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,nc,scheme", [(5, 20000, "dg"), (3, 5000, "dg"), (4, 8000, "fv")])
def test_autotune_keeps_results(cuda, N, nc, scheme):
    import torch
    from paper_2409_12483_gb300 import Context
    ref = Context(nc, N, scheme)
    if scheme == "dg":
        u0 = W.nodal_state(W.modes4(), ref.node_coords())
    else:
        u0 = W.cell_average_state(W.modes4(), nc)
    u = torch.tensor(u0, device=cuda).reshape(-1)
    a = u.clone()
    ref.ader_solve(a, max_steps=6)
    tuned = Context(nc, N, scheme)
    t = tuned.ader_autotune(u, reps=2)
    assert t["predict_cells_per_block"] in (16, 32, 64)
    assert t["face_cells_per_block"] in (32, 64)
    assert t["graph_steps"] in (4, 8, 16, 32, 64)
    assert t["predict_ms"] > 0 and t["face_ms"] > 0 and t["solve_ms_per_step"] > 0
    assert torch.equal(u, torch.tensor(u0, device=cuda).reshape(-1))  # input untouched
    b = u.clone()
    tuned.ader_solve(b, max_steps=6)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    # every valid predictor shape gives the same step
    outs = []
    for cpb in (16, 32, 64):
        valid = (((cpb * (N + 1)) % 32 == 0 or cpb == 16) and cpb * (N + 1) <= 512
                 and (N <= 5 or cpb <= 32))
        if not valid:
            continue
        tuned.ader_set_tuning(predict_cells_per_block=cpb, face_cells_per_block=32, graph_steps=8)
        o = torch.empty_like(u)
        tuned.ader_step(u, o, 1e-6)
        outs.append(o.cpu().numpy())
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
