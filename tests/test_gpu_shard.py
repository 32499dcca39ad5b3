"""A 1D mesh split over shard contexts (ader_init_shard) and advanced in
lockstep by paper_2409_12483_gb300.shard equals the single-context solve.

Ranks are processes on the one GPU, exchanging halos through host memory over
gloo and min-reducing the time step; none of their kernels waits on another
rank.  Bar: 1e-12 relative L-inf against the single context after every solve
(the same kernels on the same values: the result is in fact bit-identical),
and the same number of steps and final time."""
import os
import socket

import numpy as np
import pytest

import workloads as W
from conftest import rel_linf

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _initial(scheme, N, n_global):
    import oracle
    o = oracle.Oracle(N)
    if scheme == "dg":
        return W.nodal_state(W.modes4(3), o.node_x(n_global)).reshape(n_global, -1)
    return W.cell_average_state(W.modes4(3), n_global).reshape(n_global, -1)


def _opts(prec):
    """'fp64', 'ff', ... or 'fp64+nodal' (cfl_mode 1) as Context options"""
    parts = prec.split("+")
    o = {"precision": parts[0]}
    if "nodal" in parts[1:]:
        o["cfl_mode"] = "nodal"
    return o


def _rank(rank, world, port, scheme, N, n_global, t_end, prec, out):
    import torch
    import torch.distributed as dist

    from paper_2409_12483_gb300 import shard
    from paper_2409_12483_gb300.capi import ShardContext
    dist_ = None
    if world > 1:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        dist_ = dist
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    first, nl = shard.partition(n_global, world, rank)
    ctx = ShardContext(n_global, first, nl, N, scheme, device=dev, **_opts(prec))
    H, vpc = ctx.halo, ctx.values_per_cell
    u0 = _initial(scheme, N, n_global)
    u = torch.full((ctx.state_count,), float("nan"), dtype=torch.float64, device=dev)
    u[H * vpc:(H + nl) * vpc] = torch.tensor(u0[first:first + nl].ravel(), device=dev)
    ex = shard.HaloExchange(nl, H, vpc, dist_)
    uf, steps, t = shard.sharded_solve(shard.ContextStepper(ctx), u, ex, t_end=t_end, dist=dist_)
    torch.cuda.synchronize()
    out[rank] = (first, nl, uf[H * vpc:(H + nl) * vpc].cpu().numpy(), steps, t,
                 ex.bytes_per_fill)
    if dist_ is not None:
        dist.destroy_process_group()


@pytest.mark.parametrize("scheme,N,n_global,world,prec", [
    ("dg", 5, 1001, 1, "fp64"), ("dg", 5, 1001, 2, "fp64"), ("dg", 3, 777, 3, "fp64"),
    ("fv", 4, 900, 2, "fp64"), ("dg", 5, 640, 2, "ff"), ("dg", 5, 1001, 2, "fp64+nodal")])
def test_sharded_equals_single_context(cuda, oracle_mod, scheme, N, n_global, world, prec):
    import torch
    import torch.multiprocessing as mp

    from paper_2409_12483_gb300 import Context
    t_end = 0.01
    u0 = _initial(scheme, N, n_global)
    one = Context(n_global, N, scheme, **_opts(prec))
    ud = torch.tensor(u0.ravel(), device=cuda)
    steps_ref, t_ref, _ = one.ader_solve(ud, t_end=t_end)
    ref = ud.cpu().numpy()
    if world == 1:
        out = {}
        _rank(0, 1, 0, scheme, N, n_global, t_end, prec, out)
    else:
        ctx = mp.get_context("spawn")
        mgr = ctx.Manager()
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, scheme, N, n_global, t_end, prec,
                                                out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=600)
            assert p.exitcode == 0
    blocks = sorted(out[r] for r in range(world))
    got = np.concatenate([b[2] for b in blocks])
    for _, _, _, steps, t, nbytes in blocks:
        assert steps == steps_ref and t == t_ref
        H = 1 if scheme == "dg" else N + 1
        assert nbytes == 2 * H * (u0.shape[1]) * 8
    assert rel_linf(got, ref) < 1e-12
    # conservation of the split solve: the global sums are those of the single solve
    assert steps_ref > 3


def test_shard_rejects_the_device_time_loop(cuda):
    import torch
    from paper_2409_12483_gb300 import ADER_ERR_ARG, AderError
    from paper_2409_12483_gb300.capi import ShardContext
    ctx = ShardContext(100, 10, 40, 3, "dg")
    u = torch.ones(ctx.state_count, dtype=torch.float64, device=cuda)
    with pytest.raises(AderError) as e:
        ctx.ader_solve(u, t_end=0.1)
    assert e.value.status == ADER_ERR_ARG and "shard" in str(e.value)
