"""Scene sharding for several GPUs (one process per GPU).

Batched scenes are independent, so N ranks each take a contiguous range of
scene ids and step it with no collective on the data path.  The ranges are
balanced by the per-scene cost, taken as n_s^2 (the all-pairs broad phase of a
scene dominates its step).  A single scene does not shard: its LCP couples all
constraints in every iteration, so several GPUs run independent replicas.
"""
from __future__ import annotations

import numpy as np


def shard_scenes(sizes, world: int) -> list[tuple[int, int]]:
    """Contiguous [start, end) scene ranges, one per rank, covering every scene
    once, with the cost sum(n_s^2) split as evenly as contiguous cuts allow:
    rank r ends at the first scene where the running cost reaches
    (r + 1) / world of the total."""
    sizes = np.asarray(sizes, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    S = int(sizes.shape[0])
    cost = np.cumsum(sizes.astype(np.float64) ** 2 + 1.0)  # +1: an empty scene still costs a queue slot
    total = float(cost[-1]) if S else 0.0
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        k = int(np.searchsorted(cost, target, side="left")) + 1 if S else 0
        cuts.append(min(max(k, cuts[-1]), S))
    cuts.append(S)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def shard_cost(sizes, shards) -> list[float]:
    sizes = np.asarray(sizes, dtype=np.float64)
    return [float(np.sum(sizes[a:b] ** 2 + 1.0)) for a, b in shards]
