"""Sharding independent registration problems across ranks (one GPU each).

The problems of a batch are independent, so ranks split them and need no
collective on the data path: each rank solves its own share and only the
per-problem reports are gathered at the end.
"""
from __future__ import annotations


def partition(costs, world):
    """Greedy size-balanced assignment: problems in decreasing cost order each
    go to the rank with the least total so far (ties to the lower rank).
    Deterministic, so every rank computes the same split."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += costs[i]
    return [sorted(p) for p in parts]


def gather_reports(local, world, rank):
    """All ranks' {index: report} dicts merged on every rank (torch.distributed)."""
    import torch.distributed as dist
    out = [None] * world
    dist.all_gather_object(out, local)
    merged = {}
    for part in out:
        merged.update(part)
    return merged
