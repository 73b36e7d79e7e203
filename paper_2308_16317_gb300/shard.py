"""Host-side sharding of independent tau_00 solves over ranks.

Every (LIZ, energy, spin) solve is independent (the paper distributes atoms
over MPI ranks, Sec. 4.2), so a multi-GPU run partitions the LIZs over ranks
with no collective on the data path.  The partition balances the
elimination cost, which grows like n^3 per matrix.
"""
from __future__ import annotations

import heapq


def balanced_shards(orders, world_size: int):
    """Split LIZ indices into `world_size` disjoint lists with nearly equal
    sum of n^3 (longest-processing-time greedy: largest first onto the
    least-loaded rank).  Returns a list of sorted index lists."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    heap = [(0.0, r) for r in range(world_size)]
    heapq.heapify(heap)
    shards = [[] for _ in range(world_size)]
    for i in sorted(range(len(orders)), key=lambda k: (-orders[k], k)):
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + float(orders[i]) ** 3, r))
    return [sorted(s) for s in shards]


def shard_cost(orders, shard) -> float:
    return sum(float(orders[i]) ** 3 for i in shard)
