"""Sharding of batched factorizations across ranks (one process per GPU).

Instances are independent, so a batch is partitioned by instance with no data-path
collective: greedy longest-processing-time assignment by N^3 (the work of one iteration),
each rank factorizing its own share.  Only host metadata (iteration counts, residuals) is
gathered, for reporting."""
from __future__ import annotations

from typing import Any, Dict, List, Sequence


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


def gather(local: Dict[int, Any], count: int) -> List[Any]:
    """Every rank's per-instance results ({instance index: result}) gathered on all ranks and
    returned in instance order (host metadata only, through torch.distributed's object
    all-gather).  Raises if an instance is missing or reported twice."""
    import torch.distributed as dist
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, dict(local))
    out: List[Any] = [None] * count
    seen = set()
    for part in parts:
        for i, v in part.items():
            if i in seen or not 0 <= i < count:
                raise ValueError("instance %d reported twice or out of range" % i)
            seen.add(i)
            out[i] = v
    if len(seen) != count:
        raise ValueError("missing instances: %s" % sorted(set(range(count)) - seen)[:8])
    return out
