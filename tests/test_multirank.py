"""Multi-rank plumbing of bench.py on CPU (gloo, world size 2): every rank solves
its own replica, the job time is the maximum over ranks and the value is the
units of all ranks over that time."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    m = bench.max_over_ranks(times[rank], dist, "cpu")
    dist.barrier()
    out[rank] = (m, bench.whole_job_rate(1000.0, world, m))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    times = [1.5, 2.5]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        m, rate = out[r]
        assert m == 2.5
        assert rate == pytest.approx(2 * 1000.0 / 2.5)


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(3.0) == 3.0
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
