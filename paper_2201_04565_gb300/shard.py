"""Specimen sharding across ranks (one process per GPU).

A batch of specimens partitions into independent problems: each rank steps
its own share in its own batched context and no data crosses ranks during
the run. The only collective is the timing reduction (max over ranks).
"""
from __future__ import annotations

import heapq


def partition(costs, world: int):
    """Split specimens with the given costs (e.g. spring counts) into `world`
    shares by longest-processing-time-first: specimens in descending cost
    (ties by index) go to the currently lightest share (ties by rank).
    Deterministic; returns one ascending index list per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda q: (-costs[q], q))
    heap = [(0, r) for r in range(world)]
    shares = [[] for _ in range(world)]
    for q in order:
        load, r = heapq.heappop(heap)
        shares[r].append(q)
        heapq.heappush(heap, (load + costs[q], r))
    return [sorted(sh) for sh in shares]


def my_share(costs, rank: int, world: int):
    return partition(costs, world)[rank]


def max_over_ranks(value: float) -> float:
    """The maximum of a float over all ranks of the default process group
    (the value itself without one)."""
    import torch
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()) or td.get_world_size() == 1:
        return float(value)
    dev = "cuda" if td.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())
