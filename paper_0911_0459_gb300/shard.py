"""Sharding of independent capillaries across ranks (one process per GPU).

Capillaries of a sweep are independent, so a multi-GPU sweep needs no exchange
on the data path: every rank runs the capillaries assigned to it and the
filling curves are gathered once at the end.  Assignment is longest-processing
-time-first on the estimated cost (fluid nodes x steps), which keeps the
largest load within a few percent of the mean for sweeps of hundreds of
uneven capillaries.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


def cost(cap) -> float:
    """Estimated work of one capillary: all nodes x steps (walls are a small fraction)."""
    return float(cap.nx) * float(cap.ny) * float(getattr(cap, "steps", 1))


def partition(costs: Sequence[float], world: int) -> List[List[int]]:
    """Greedy LPT: indices of each rank, each list in increasing index order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def my_share(caps, rank: int, world: int) -> List[int]:
    return partition([cost(c) for c in caps], world)[rank]


def gather(local_idx: Sequence[int], local_values: np.ndarray, n_total: int, group=None) -> np.ndarray:
    """Reassemble per-capillary results (rows of local_values) in sweep order on every
    rank with one all_gather_object (the only collective of a sharded sweep)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    items = [None] * world
    dist.all_gather_object(items, (list(local_idx), np.asarray(local_values)), group=group)
    shape = None
    for idx, vals in items:
        if len(idx):
            shape = vals.shape[1:]
            break
    out = np.full((n_total,) + (shape or ()), np.nan)
    for idx, vals in items:
        for j, i in enumerate(idx):
            out[i] = vals[j]
    return out
