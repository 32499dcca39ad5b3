"""Host side of the 1D domain decomposition (contexts from ader_init_shard).

A periodic mesh of n_global cells is cut into contiguous blocks, one per rank.
Each rank's state array is [left halo | local cells | right halo]; one time step
of the global scheme is: fill the halos from the neighbouring ranks, reduce the
time step to the minimum over ranks (8 bytes), run the ordinary step on the
whole array.  The halo cells are recomputed by each rank, so the DG face traces
and the WENO reconstructions next to a block edge come out exactly as on one
mesh.  The time step follows the CFL rule of Sec. 1.5 with the last step
clipped to t_end, as the single-mesh device loop does.

This module holds no arithmetic of the method: every step runs in the library
through the `stepper` it is given; it only moves halo values between ranks and
reduces one scalar.  The exchange uses torch.distributed (gloo or NCCL); CUDA
tensors on a gloo group are staged through host memory.
"""
from __future__ import annotations


def partition(n_global: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous block of rank `rank`: (first cell, cell count); the first
    n_global % world ranks hold one cell more."""
    if world < 1 or not 0 <= rank < world or n_global < world:
        raise ValueError("need 0 <= rank < world <= n_global")
    base, extra = divmod(n_global, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def neighbours(rank: int, world: int) -> tuple[int, int]:
    """(left, right) ranks on the periodic ring."""
    return (rank - 1) % world, (rank + 1) % world


class HaloExchange:
    """Fills the halo cells of a shard's state array (a 1D torch tensor of
    (n_local + 2 halo) * values_per_cell values) from the neighbouring ranks.
    With no process group (or world size 1) the mesh is one periodic block and
    the halos wrap around it."""

    def __init__(self, n_local: int, halo: int, values_per_cell: int, dist=None, group=None):
        if n_local < halo:
            raise ValueError("a block must hold at least as many cells as its halo")
        self.n_local, self.halo, self.vpc = int(n_local), int(halo), int(values_per_cell)
        self.dist, self.group = dist, group
        self.world = dist.get_world_size(group) if dist is not None else 1
        self.rank = dist.get_rank(group) if dist is not None else 0
        self.bytes_per_fill = 2 * self.halo * self.vpc * 8  # sent (= received) per rank

    def _slices(self):
        H, L, v = self.halo, self.n_local, self.vpc
        return {"left_halo": slice(0, H * v), "first_local": slice(H * v, 2 * H * v),
                "last_local": slice(L * v, (L + H) * v),
                "right_halo": slice((L + H) * v, (L + 2 * H) * v)}

    def fill(self, u):
        s = self._slices()
        if self.world == 1:
            u[s["left_halo"]] = u[s["last_local"]]
            u[s["right_halo"]] = u[s["first_local"]]
            return u
        left, right = neighbours(self.rank, self.world)
        staged = u.is_cuda and self.dist.get_backend(self.group) == "gloo"

        def wire(t):
            return t.cpu() if staged else t.contiguous()

        # phase 0: first local cells -> left rank's right halo; phase 1: last
        # local cells -> right rank's left halo (one send and one receive per
        # rank and phase, so the pairs match with any backend)
        for tag, (src, dst, to, frm) in enumerate((("first_local", "right_halo", left, right),
                                                   ("last_local", "left_halo", right, left))):
            send = wire(u[s[src]])
            recv = wire(u[s[dst]].clone())
            reqs = [self.dist.isend(send, to, group=self.group, tag=tag),
                    self.dist.irecv(recv, frm, group=self.group, tag=tag)]
            for r in reqs:
                r.wait()
            u[s[dst]] = recv.to(u.device) if staged else recv
        return u


def min_over_ranks(x: float, dist=None, group=None, device="cpu") -> float:
    """Minimum of a per-rank scalar over the group (identity without one)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    return float(t.item())


def clip_dt(t: float, dt: float, t_end: float) -> tuple[float, bool]:
    """The last step reaches t_end exactly: (dt, is_last), with the same test the
    device time loop uses (t + dt >= t_end)."""
    if t_end > 0.0 and t + dt >= t_end:
        return t_end - t, True
    return dt, False


class ContextStepper:
    """The stepper of a shard context: local CFL step and one time step."""

    def __init__(self, ctx):
        self.ctx = ctx

    def compute_dt(self, u, t: float) -> float:
        return self.ctx.ader_compute_dt(u, t, 0.0)

    def step(self, u, u_new, dt: float) -> None:
        self.ctx.ader_step(u, u_new, dt)


def sharded_solve(stepper, u, exchange: HaloExchange, t_end: float = 0.0, max_steps: int = 0,
                  dist=None, group=None, reduce_device="cpu"):
    """Advance a shard's state array to t_end (or max_steps steps) in lockstep
    with the other ranks: per step, fill the halos, take the minimum of the
    ranks' CFL steps, clip it to t_end, and step.  Returns (u, steps, t) with u
    the array holding the final state (halos stale)."""
    if not (t_end > 0.0) and max_steps <= 0:
        raise ValueError("need t_end > 0 or max_steps > 0")
    u_new = u.clone() if hasattr(u, "clone") else u.copy()
    t, steps = 0.0, 0
    while True:
        if (t_end > 0.0 and t >= t_end) or (max_steps > 0 and steps >= max_steps):
            break
        exchange.fill(u)
        dt_local = stepper.compute_dt(u, t)
        dt = min_over_ranks(dt_local, dist, group, reduce_device)
        if not (dt > 0.0):
            raise RuntimeError(f"non-positive time step {dt} at t = {t}")
        dt, last = clip_dt(t, dt, t_end)
        stepper.step(u, u_new, dt)
        u, u_new = u_new, u
        t = t_end if last else t + dt
        steps += 1
    return u, steps, t
