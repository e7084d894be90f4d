"""Cell sharding across ranks (one process per GPU).

Cells are independent (the paper's multi-cell setting: every grid cell is its
own chemistry problem), so the forward solve shards with no exchange: rank r
of N owns the contiguous cell range cell_range(C, r, N) of a global batch of C
cells.  The one collective is in the adjoint: dL/dtheta is a sum over all
cells of a vector of n_reactions values, reduced here in a fixed rank order so
the result does not depend on the reduction tree.  dL/dy0 stays sharded.
"""
from __future__ import annotations

import numpy as np


def cell_range(n_cells: int, rank: int, world: int) -> tuple[int, int]:
    """[begin, end) of rank's cells: contiguous, sizes differ by at most one,
    the larger shards first."""
    if world < 1 or not (0 <= rank < world) or n_cells < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_cells, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def reduce_theta_grad(g_local, group=None):
    """Sum of every rank's dL/dtheta (a float64 vector of n_reactions values),
    added in rank order 0..N-1 on every rank.  g_local: numpy array or torch
    tensor on the rank's device; the result has the same type and device."""
    import torch
    import torch.distributed as dist

    is_np = isinstance(g_local, np.ndarray)
    t = torch.from_numpy(np.ascontiguousarray(g_local, np.float64)) if is_np else g_local.to(torch.float64)
    world = dist.get_world_size(group)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t.contiguous(), group=group)
    total = parts[0].clone()
    for p in parts[1:]:
        total += p
    return total.numpy() if is_np else total
