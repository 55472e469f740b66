"""Host-side helpers for running the solver on several GPUs of one node.

Instances are independent, so a batch shards across ranks with no exchange on
the data path: each rank solves its own shard on its own GPU.  The only
collective is the max-over-ranks reduction of a step time (or any scalar).
"""
from __future__ import annotations

import heapq

import numpy as np


def instance_work(N, n):
    """Work estimate of each instance: (N_i + 1) n_i^2 (one block factorisation
    and one block solve per stage)."""
    return (np.asarray(N, dtype=np.float64) + 1.0) * np.asarray(n, dtype=np.float64) ** 2


def lpt_shards(work, world: int):
    """Longest-processing-time-first partition of the instances into `world`
    shards of balanced total work.  Returns a list of sorted index arrays."""
    work = np.asarray(work, dtype=np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = np.argsort(-work, kind="stable")
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(i))
        heapq.heappush(heap, (load + float(work[i]), r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def shard_of(work, world: int, rank: int):
    """Indices of the instances rank `rank` solves."""
    return lpt_shards(work, world)[rank]


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a scalar over the ranks of the default process group (the
    value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
