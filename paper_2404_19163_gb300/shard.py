"""Sharding of batched factorizations across ranks (one process per GPU).

Instances are independent, so a batch is partitioned by instance with no data-path
collective: greedy longest-processing-time assignment by N^3 (the work of one iteration),
each rank factorizing its own share.  Only host metadata (iteration counts, residuals) is
gathered, for reporting."""
from __future__ import annotations

from typing import List, Sequence


def assign(sizes: Sequence[int], world_size: int) -> List[List[int]]:
    """Instance indices per rank, largest first onto the least-loaded rank (ties: lower rank)."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]) ** 3, i))
    load = [0] * world_size
    out: List[List[int]] = [[] for _ in range(world_size)]
    for i in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += int(sizes[i]) ** 3
    return out


def mine(sizes: Sequence[int], rank: int, world_size: int) -> List[int]:
    return assign(sizes, world_size)[rank]


def imbalance(sizes: Sequence[int], world_size: int) -> float:
    """max rank load / mean rank load (1.0 = perfect)."""
    parts = assign(sizes, world_size)
    loads = [sum(int(sizes[i]) ** 3 for i in p) for p in parts]
    return max(loads) / (sum(loads) / world_size)
