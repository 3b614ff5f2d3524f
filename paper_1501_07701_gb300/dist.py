"""Multi-process helpers: how stream work is split over ranks.

Streams are independent (one status per stream, Sec. 3.2), so the path shards
by stream with no data exchange: every rank owns its own streams and writes
its own outputs.  Two splits are used:

* weak scaling (the benchmark): each rank runs its own instance of a
  workload, its stream seeds offset by rank * n_streams, so per-GPU work is
  fixed as ranks are added;
* strong scaling: one set of streams is cut into contiguous ranges, one per
  rank, so the job's total work is fixed as ranks are added.

The only collectives are host-side bookkeeping (barrier, max of elapsed
times); none touches generated data.
"""
from __future__ import annotations

import numpy as np


def weak_seeds(seeds: np.ndarray, rank: int) -> np.ndarray:
    """Seeds of rank `rank`'s instance: the workload's seeds shifted by
    rank * len(seeds) (mod 2^32)."""
    n = seeds.size
    return (seeds.astype(np.uint64) + np.uint64(rank * n)).astype(np.uint32)


def strong_range(n_streams: int, rank: int, world: int):
    """Contiguous [start, stop) of the streams owned by `rank`."""
    base, extra = divmod(n_streams, world)
    start = rank * base + min(rank, extra)
    stop = start + base + (1 if rank < extra else 0)
    return start, stop


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of a float over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(value: float, device=None) -> float:
    """Max of a float over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
