"""Sharding of independent pose graphs across ranks (one process per GPU).

The batched form's graphs are independent problems, so N ranks split them
with no exchange on the data path: each rank solves its own share and only
the timing (max over ranks) and the counts are reduced.  The split is
longest-processing-time first by edge count: graphs in decreasing size
(ties by index), each to the rank with the least work so far (ties by rank).
It depends only on the sizes, so every rank computes the same split locally.
"""
from __future__ import annotations

import heapq

import numpy as np


def shard_graphs(sizes, world: int) -> list[np.ndarray]:
    """Returns, for each rank, the sorted indices of its graphs."""
    if world < 1:
        raise ValueError("world must be >= 1")
    sizes = np.asarray(sizes, dtype=np.int64)
    order = np.lexsort((np.arange(sizes.size), -sizes))
    heap = [(0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for g in order:
        load, r = heapq.heappop(heap)
        out[r].append(int(g))
        heapq.heappush(heap, (load + int(sizes[g]), r))
    return [np.array(sorted(x), dtype=np.int64) for x in out]


def max_over_ranks(value: float) -> float:
    """Max of a float over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float) -> float:
    """Sum of a float over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
