"""Sharding of independent graphs across ranks (one process per GPU).

The batched and served forms cluster independent graphs, so a multi-GPU run
partitions the graphs and needs no exchange on the data path: each rank
clusters its share with its own lc_cluster_batch call or lc_server.  Only
the results are collected, on the host, after the timed work.  A single
graph is not sharded (every pass needs all neighbours' labels and the
global cluster weights), so single-graph runs are replicas.
"""
from __future__ import annotations

import heapq


def assign(weights, world: int) -> list[list[int]]:
    """Longest-processing-time assignment of items (weight = expected work,
    e.g. stored edges) to `world` ranks: heaviest first, each to the rank
    with the least work so far (ties to the lower rank).  Deterministic;
    each rank's list is in ascending item order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    heap = [(0, r) for r in range(world)]
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + weights[i], r))
    return [sorted(x) for x in out]


def local(weights, rank: int, world: int) -> list[int]:
    """The items rank `rank` clusters."""
    return assign(weights, world)[rank]


def gather(local_items: list[int], local_results: list, group=None) -> list | None:
    """Collects every rank's (item, result) pairs on rank 0, in item order
    (torch.distributed object collective on the host; None elsewhere)."""
    import torch.distributed as dist

    pairs = list(zip(local_items, local_results))
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return [r for _, r in sorted(pairs, key=lambda p: p[0])]
    rank = dist.get_rank(group)
    buf = [None] * dist.get_world_size(group) if rank == 0 else None
    dist.gather_object(pairs, buf, dst=0, group=group)
    if rank != 0:
        return None
    merged = [p for part in buf for p in part]
    return [r for _, r in sorted(merged, key=lambda p: p[0])]
