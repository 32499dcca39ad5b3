"""Continuous-batching server: every solve's result equals the same solve run alone
(same kernels per cell, 1e-12 relative L-inf), admission respects slots, memory
and arrival times, and requests that arrive while others run join the batch."""
import numpy as np
import pytest

import workloads as W
from conftest import rel_linf

pytestmark = pytest.mark.gpu


def request_state(N, nc, seed):
    g = np.random.default_rng(seed)
    k = np.arange(1, 4, dtype=float)
    f = W.Field1D(rho_amp=g.uniform(0, 0.1 / 3, 3), rho_phase=g.uniform(0, 6.28, 3), rho_k=k,
                  u=0.5, p_amp=g.uniform(0, 0.1 / 3, 3), p_phase=g.uniform(0, 6.28, 3), p_k=k)
    # nodes from the library's own coordinates
    from paper_2409_12483_gb300.capi import NoAllocStep  # noqa: F401  (host-only ctx)
    import ctypes as C
    from paper_2409_12483_gb300.capi import Mesh, default_options, load
    L = load()
    ctx = C.c_void_p()
    assert L.ader_init(C.byref(Mesh(nc, 0.0, 1.0)), N, 0, C.byref(default_options()), C.byref(ctx)) == 0
    x = np.zeros(nc * (N + 1))
    assert L.ader_node_coords(ctx, x.ctypes.data_as(C.c_void_p), x.size) == 0
    L.ader_destroy(ctx)
    return W.nodal_state(f, x.reshape(nc, N + 1)).ravel()


def alone(cuda, N, nc, u0, t_end, **opts):
    import torch
    from paper_2409_12483_gb300 import Context
    ctx = Context(nc, N, "dg", **opts)
    u = torch.tensor(u0, device=cuda)
    steps, t, rc = ctx.ader_solve(u, t_end=t_end)
    torch.cuda.synchronize()
    return u.cpu().numpy(), steps, t


def drain(srv, limit=100000):
    now = 0.0
    for _ in range(limit):
        run, que = srv.progress(now)
        now += 1.0
        if run == 0 and que == 0:
            return
    raise AssertionError("server did not drain")


MIX = [(1, 37, 0.02), (2, 100, 0.01), (3, 65, 0.01), (4, 200, 0.004), (5, 33, 0.01),
       (6, 129, 0.002), (7, 64, 0.003), (5, 300, 0.001)]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "ff", "fp32ff", "incr"])
def test_results_equal_alone(cuda, precision):
    """the batched kernels (16-cell predictor tiles, 32-cell face tiles, one graph
    branch per degree) give every solve the result of its own context"""
    from paper_2409_12483_gb300.capi import REQ_DONE, Server
    extra = {"precision": precision}
    if precision in ("fp32", "fp32ff"):
        extra["fp64_sweeps"] = 2
    srv = Server(pool_bytes=256 << 20, max_slots=16, ticks_per_round=8, **extra)
    ids = []
    states = []
    for i, (N, nc, t_end) in enumerate(MIX):
        u0 = request_state(N, nc, i)
        states.append(u0)
        ids.append(srv.submit(N, u0, t_end))
    drain(srv)
    for (N, nc, t_end), rid, u0 in zip(MIX, ids, states):
        r = srv.poll(rid, want_state=True)
        assert r["state"] == REQ_DONE and r["status"] == 0
        ref, steps, t = alone(cuda, N, nc, u0, t_end, **extra)
        assert r["steps"] == steps and r["t"] == t == t_end
        assert rel_linf(r["u"], ref) < 1e-12
    tot = srv.totals()
    assert tot["cell_updates"] == sum(srv.poll(i)["steps"] * nc for i, (_, nc, _) in zip(ids, MIX))


def test_slots_limit_and_late_arrivals_join(cuda):
    from paper_2409_12483_gb300.capi import REQ_DONE, REQ_QUEUED, REQ_RUNNING, Server
    srv = Server(pool_bytes=128 << 20, max_slots=2, ticks_per_round=4)
    specs = [(3, 50, 0.2, 0.0), (3, 50, 0.002, 0.0), (2, 40, 0.005, 0.0), (4, 30, 0.05, 5.0)]
    ids = [srv.submit(N, request_state(N, nc, 10 + i), t_end, arrival=a)
           for i, (N, nc, t_end, a) in enumerate(specs)]
    seen_run = 0
    now = 0.0
    late_admitted_while_running = False
    for _ in range(10000):
        run, que = srv.progress(now)
        seen_run = max(seen_run, run)
        st = [srv.poll(i)["state"] for i in ids]
        if st[3] == REQ_QUEUED:
            assert now < 5.0 or run == 2  # not before its arrival; later only if no slot
        if st[3] == REQ_RUNNING and st[0] == REQ_RUNNING:
            late_admitted_while_running = True
        now += 1.0
        if run == 0 and que == 0:
            break
    assert seen_run == 2
    assert late_admitted_while_running  # the late request joined a running batch
    for i, (N, nc, t_end, a) in zip(ids, specs):
        r = srv.poll(i, want_state=True)
        assert r["state"] == REQ_DONE and r["admitted"] >= a
        ref, steps, t = alone(cuda, N, nc, request_state(N, nc, 10 + ids.index(i)), t_end)
        assert rel_linf(r["u"], ref) < 1e-12


def test_admission_by_memory(cuda):
    from paper_2409_12483_gb300 import ADER_ERR_NOMEM, AderError
    from paper_2409_12483_gb300.capi import REQ_DONE, Server
    need = Server.request_bytes(5, 1000)
    # control and work-list region (~40 KB here) + room for exactly one such request
    srv = Server(pool_bytes=need + (64 << 10), max_slots=8, ticks_per_round=4)
    ids = [srv.submit(5, request_state(5, 1000, 20 + i), 0.0005) for i in range(3)]
    max_run = 0
    now = 0.0
    while True:
        run, que = srv.progress(now)
        max_run = max(max_run, run)
        now += 1
        if run == 0 and que == 0:
            break
    assert max_run == 1
    for i in ids:
        assert srv.poll(i)["state"] == REQ_DONE
    with pytest.raises(AderError) as e:
        srv.submit(5, request_state(5, 2000, 0), 0.001)
    assert e.value.status == ADER_ERR_NOMEM


def test_failed_solve_is_reported_and_others_finish(cuda):
    from paper_2409_12483_gb300 import ADER_ERR_NONPHYSICAL
    from paper_2409_12483_gb300.capi import REQ_DONE, REQ_FAILED, Server
    srv = Server(pool_bytes=64 << 20, max_slots=4, ticks_per_round=4)
    good = srv.submit(2, request_state(2, 50, 1), 0.002)
    u_bad = request_state(3, 40, 2)
    u_bad[5 * 12] = -1.0  # negative density
    bad = srv.submit(3, u_bad, 0.002)
    drain(srv)
    assert srv.poll(good)["state"] == REQ_DONE
    r = srv.poll(bad)
    assert r["state"] == REQ_FAILED and r["status"] == ADER_ERR_NONPHYSICAL
