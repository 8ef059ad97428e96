"""Sharding of independent point sets over GPUs (one process per GPU).

The sets of a batched build are independent (each is its own tree), so they
split over ranks with no data exchange: every rank builds its share with one
kdb_build_batched call.  Shares are made by longest-processing-time-first
(LPT) list scheduling: sets in decreasing order of estimated cost, each to
the rank with the least cost so far.  The result depends only on the sizes
and the number of ranks, so every rank computes the same assignment without
communicating.
"""
from __future__ import annotations

import heapq
import math
from typing import Sequence


def build_cost(n: int) -> float:
    """Estimated work of one set: points times levels (each level touches
    every live point once)."""
    return float(n) * max(1, math.ceil(math.log2(n + 1)))


def lpt_shards(sizes: Sequence[int], world: int) -> list[list[int]]:
    """Set indices of every rank, each list in increasing index order.

    Ties are broken by set index, then by rank, so the assignment is a
    deterministic function of (sizes, world)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    heap = [(0.0, r) for r in range(world)]
    shards: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + build_cost(int(sizes[i])), r))
    return [sorted(s) for s in shards]


def shard_cost(sizes: Sequence[int], shard: Sequence[int]) -> float:
    return sum(build_cost(int(sizes[i])) for i in shard)
