"""Sharding one state set over several GPUs (one process per GPU).

States are independent in the Picard sweep (the coefficient map acts state by state), so
each rank solves a contiguous block of the states with the Philox counter offset by the
block's first global index (it draws exactly the samples of the unsharded solve).  The only
exchange is the residual of Algorithm 1: per sweep, the ranks' (sum dv^2, sum v^2, max |dv|)
are combined with one all-reduce of a [K, 3] FP64 tensor (sums and a maximum), after which
every rank holds the global relative residual.  Nothing on the data path moves between GPUs.
"""
from __future__ import annotations

import numpy as np


def shard_bounds(M: int, world: int, rank: int):
    """Contiguous block [lo, hi) of M states for `rank` of `world` (sizes differ by <= 1)."""
    base, extra = divmod(M, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def combine_residual_parts(parts: np.ndarray, group=None):
    """Global (relative L2 residual, sup-norm change) per sweep from this rank's parts
    [K, 3] = (sum dv^2, sum v^2, max |dv|); all-reduces over the default process group (or
    `group`) when torch.distributed is initialised, else uses the local parts."""
    import torch
    import torch.distributed as dist
    p = np.asarray(parts, dtype=np.float64).reshape(-1, 3)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        backend = dist.get_backend(group)
        dev = "cuda" if backend == "nccl" else "cpu"
        sums = torch.tensor(p[:, :2].copy(), dtype=torch.float64, device=dev)
        mx = torch.tensor(p[:, 2].copy(), dtype=torch.float64, device=dev)
        dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(mx, op=dist.ReduceOp.MAX, group=group)
        p = np.concatenate([sums.cpu().numpy(), mx.cpu().numpy()[:, None]], axis=1)
    rel = np.sqrt(p[:, 0]) / np.sqrt(p[:, 1])
    return rel, p[:, 2]


class ShardedSolver:
    """One rank's share of a sharded solve: a Solver over this rank's block of the states
    (Philox counter offset by the block's first global index) and the global residual."""

    def __init__(self, game: str, nu: float, T: float, N: int, M_total: int, world: int,
                 rank: int, group=None, **kw):
        from .solver import Solver
        self.lo, self.hi = shard_bounds(M_total, world, rank)
        self.group = group
        self.solver = Solver(game, nu, T, N, point_offset=self.lo, **kw)

    def set_points(self, x_global):
        self.solver.set_points(x_global[self.lo:self.hi].contiguous())

    def picard_sweep(self, n_sweeps: int):
        self.solver.picard_sweep(n_sweeps)
        return combine_residual_parts(self.solver.residual_parts(n_sweeps), self.group)

    def get_state(self):
        return self.solver.get_state()

    def close(self):
        self.solver.close()
