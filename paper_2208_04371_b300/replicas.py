"""Independent-instance sharding across ranks (one process per GPU).

Batched sweeps and surrogate training data consist of independent line instances, so they
shard without any data-path exchange: each rank solves its own subset and the small results
(S-matrices) are gathered once at the end.  Instances are assigned greedily, largest cost
first, to the rank with the least work so far (cost = cells x steps), which keeps the ranks
within one instance of each other.  The single large line does not decompose here: several
GPUs run independent replicas of it.
"""
from __future__ import annotations

from typing import Callable, List, Sequence

import numpy as np


def shard(costs: Sequence[float], world: int) -> List[List[int]]:
    """Instance indices per rank, each list in ascending order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def run_sharded(n: int, costs: Sequence[float], solve: Callable[[List[int]], np.ndarray],
                rank: int, world: int, dist=None) -> np.ndarray:
    """Solve this rank's shard with solve(indices) -> array [len(indices), ...] and gather the
    full [n, ...] result on every rank (a single all_gather_object of the small results)."""
    mine = shard(costs, world)[rank]
    part = solve(mine)
    if world == 1 or dist is None:
        pieces = [(mine, part)]
    else:
        pieces = [None] * world
        dist.all_gather_object(pieces, (mine, part))
    first = next(p for _, p in pieces if len(p))
    out = np.zeros((n,) + tuple(np.asarray(first).shape[1:]), dtype=np.asarray(first).dtype)
    seen = np.zeros(n, dtype=np.int64)
    for idx, p in pieces:
        for k, i in enumerate(idx):
            out[i] = p[k]
            seen[i] += 1
    if not np.all(seen == 1):
        raise RuntimeError("sharded results do not cover every instance exactly once")
    return out
