"""Host logic of the 1D domain decomposition (paper_2409_12483_gb300.shard) on
CPU: the partition, the periodic halo fill, the min-reduction of the time step
and the lockstep loop, run by 1, 2 and 3 gloo ranks with the oracle as each
rank's stepper on its [halo | block | halo] array.  The concatenated blocks
must equal the oracle's single-mesh solve step for step (same time steps, same
clipped last step), which holds only if every halo holds its neighbour's cells
and the time step is the global one."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleStepper:
    """Each rank's stepper for the test: the oracle's CFL step and time step on
    the shard's extended array (periodic within it, as the library's kernels)."""

    def __init__(self, o, scheme, dx):
        self.o, self.scheme, self.dx = o, scheme, dx

    def compute_dt(self, u, t):
        a = u.numpy()
        return self.o.dg_dt(a, self.dx) if self.scheme == "dg" else self.o.fv_dt(a, self.dx)

    def step(self, u, u_new, dt):
        import torch
        if self.scheme == "dg":
            out, _, _, rc = self.o.dg_step(u.numpy(), self.dx, dt)
        else:
            out, _, rc = self.o.fv_step(u.numpy(), self.dx, dt)
        assert rc == 0
        u_new.copy_(torch.from_numpy(out))


def _initial(scheme, N, n_global):
    import oracle
    import workloads as W
    o = oracle.Oracle(N)
    if scheme == "dg":
        return W.nodal_state(W.modes4(7), o.node_x(n_global)).reshape(n_global, -1)
    return W.cell_average_state(W.modes4(7), n_global).reshape(n_global, -1)


def _run_rank(rank, world, port, scheme, N, n_global, t_end, out):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2409_12483_gb300 import shard
    dist_ = None
    if world > 1:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        dist_ = dist
    oracle.build()
    o = oracle.Oracle(N)
    H = 1 if scheme == "dg" else N + 1
    first, nl = shard.partition(n_global, world, rank)
    u0 = _initial(scheme, N, n_global)
    vpc = u0.shape[1]
    ext = np.concatenate([u0[(first - H + np.arange(H)) % n_global], u0[first:first + nl],
                          u0[(first + nl + np.arange(H)) % n_global]]).ravel()
    u = torch.tensor(ext)
    u[: H * vpc] = float("nan")  # the halo must come from the exchange, not the set-up
    u[(nl + H) * vpc:] = float("nan")
    ex = shard.HaloExchange(nl, H, vpc, dist_)
    uf, steps, t = shard.sharded_solve(OracleStepper(o, scheme, 1.0 / n_global), u, ex,
                                       t_end=t_end, dist=dist_)
    out[rank] = (first, nl, uf[H * vpc:(H + nl) * vpc].numpy().copy(), steps, t)
    if dist_ is not None:
        dist.destroy_process_group()


@pytest.mark.parametrize("scheme,N,n_global,world", [("dg", 3, 37, 2), ("dg", 2, 30, 3),
                                                     ("fv", 4, 23, 2), ("dg", 5, 11, 1)])
def test_sharded_solve_equals_single_mesh(scheme, N, n_global, world):
    import torch.multiprocessing as mp

    import oracle
    oracle.build()
    o = oracle.Oracle(N)
    u0 = _initial(scheme, N, n_global)
    t_end = 0.05
    ref, steps_ref, t_ref, rc = o.solve(scheme, u0.ravel(), 1.0 / n_global, t_end=t_end)
    assert rc == 0 and steps_ref > 5
    if world == 1:
        out = {}
        _run_rank(0, 1, 0, scheme, N, n_global, t_end, out)
    else:
        ctx = mp.get_context("spawn")
        mgr = ctx.Manager()
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_run_rank, args=(r, world, port, scheme, N, n_global, t_end,
                                                    out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
            assert p.exitcode == 0
    blocks = sorted(out[r] for r in range(world))
    assert sum(b[1] for b in blocks) == n_global
    got = np.concatenate([b[2] for b in blocks])
    for first, nl, _, steps, t in blocks:
        assert steps == steps_ref and t == t_ref
    assert np.array_equal(got, ref)  # the same arithmetic on the same values


def test_partition_and_neighbours():
    from paper_2409_12483_gb300 import shard
    for n, w in [(10, 3), (7, 7), (100, 8), (5, 1)]:
        blocks = [shard.partition(n, w, r) for r in range(w)]
        assert blocks[0][0] == 0 and sum(b[1] for b in blocks) == n
        for (f0, n0), (f1, _) in zip(blocks, blocks[1:]):
            assert f0 + n0 == f1
        assert max(b[1] for b in blocks) - min(b[1] for b in blocks) <= 1
    assert shard.neighbours(0, 4) == (3, 1) and shard.neighbours(3, 4) == (2, 0)
    with pytest.raises(ValueError):
        shard.partition(3, 4, 0)
    assert shard.clip_dt(0.9, 0.2, 1.0) == (pytest.approx(0.1), True)
    assert shard.clip_dt(0.5, 0.2, 1.0) == (0.2, False)
    assert shard.clip_dt(0.5, 0.2, 0.0) == (0.2, False)
