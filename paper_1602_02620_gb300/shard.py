"""Sharding by points across GPUs (one process per GPU).

The index shards naturally by point ids: rank k indexes the contiguous id range
shard_range(n, k, world) with the same parameters (same seed), a query batch is
answered by every rank against its shard, and the per-shard answers, each sorted
and offset to global ids, are concatenated in rank order.  Because the ranges
are contiguous and ascending, the concatenation of sorted shard answers is the
sorted global answer, and #Collisions / #Candidates add up across shards.  The
only exchange is this gather of results; the build needs none.
"""
from __future__ import annotations

import numpy as np


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous id range [lo, hi) of `rank`; sizes differ by at most one."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def merge(parts):
    """Merge per-shard answers [(offs, ids, collisions, candidates, id_offset), ...] given in rank order."""
    nq = len(parts[0][0]) - 1
    counts = sum(np.diff(p[0]) for p in parts)
    offs = np.zeros(nq + 1, np.uint64)
    np.cumsum(counts, out=offs[1:])
    ids = np.zeros(int(offs[-1]), np.uint32)
    coll = np.zeros(nq, np.uint64)
    cand = np.zeros(nq, np.uint64)
    fill = offs[:-1].copy()
    for o, i, c, d, lo in parts:
        for q in range(nq):
            a, b = int(o[q]), int(o[q + 1])
            ids[int(fill[q]):int(fill[q]) + (b - a)] = i[a:b] + np.uint32(lo)
            fill[q] += b - a
        coll += c
        cand += d
    return offs, ids, coll, cand


def gather_answers(local, id_offset: int, group=None):
    """All-gather each rank's (offs, ids, collisions, candidates) and merge them on every rank."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    objs = [None] * world
    payload = tuple(np.asarray(x) for x in local) + (id_offset,)
    dist.all_gather_object(objs, payload, group=group)
    return merge(objs)
