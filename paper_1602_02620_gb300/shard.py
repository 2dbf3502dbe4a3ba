"""Sharding by points across GPUs (one process per GPU).

The index shards naturally by point ids: rank k indexes the contiguous id range
shard_range(n, k, world) with the same parameters (same seed, and the same number of
parts or copies of Algorithm 1, fixed from the whole set), a query batch is answered by
every rank against its shard, and the per-shard answers, each sorted and offset to
global ids, are concatenated in rank order.  Because the ranges are contiguous and
ascending, the concatenation of sorted shard answers is the sorted global answer, and
#Collisions / #Candidates add up across shards (both count over points, and the shards
hold disjoint points).  The only exchange is this gather of results; the build needs none.
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
    """Merge per-shard answers [(offs, ids, collisions, candidates, id_offset), ...] given in rank
    order: query q's ids are the shards' ids for q, each offset to global ids, in rank order."""
    nq = len(parts[0][0]) - 1
    counts = [np.diff(np.asarray(p[0], np.int64)) for p in parts]
    total = np.sum(counts, axis=0) if counts else np.zeros(nq, np.int64)
    offs = np.zeros(nq + 1, np.uint64)
    np.cumsum(total, out=offs[1:])
    ids = np.zeros(int(offs[-1]), np.uint32)
    coll = np.zeros(nq, np.uint64)
    cand = np.zeros(nq, np.uint64)
    base = offs[:-1].astype(np.int64)          # where the next shard's ids of each query go
    for (o, i, c, d, lo), cnt in zip(parts, counts):
        o = np.asarray(o, np.int64)
        owner = np.repeat(np.arange(nq), cnt)
        within = np.arange(len(i), dtype=np.int64) - np.repeat(o[:-1], cnt)
        ids[base[owner] + within] = np.asarray(i, np.uint32) + np.uint32(lo)
        base += cnt
        coll += np.asarray(c, np.uint64)
        cand += np.asarray(d, np.uint64)
    return offs, ids, coll, cand


def gather_answers(local, id_offset: int, group=None):
    """All-gather each rank's (offs, ids, collisions, candidates) and merge them on every rank."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):   # a single process: its own shard only
        return merge([tuple(np.asarray(x) for x in local) + (id_offset,)])
    world = dist.get_world_size(group)
    objs = [None] * world
    payload = tuple(np.asarray(x) for x in local) + (id_offset,)
    dist.all_gather_object(objs, payload, group=group)
    return merge(objs)


def global_shape(n_total: int, d: int, r: int, seed: int, t=None, replicate: int = 0, approx_c: float = 0.0):
    """Algorithm 1's parts t and copies rep for the whole set of n_total points, so that every
    shard builds the same tables (the rule for approx_c depends on n)."""
    from . import fclsh

    sh = fclsh.derive_params(n_total, d, r, seed, t=t, replicate=replicate, approx_c=approx_c)
    return sh["t"], sh["rep"]


class ShardedIndex:
    """This rank's shard of an index sharded by points, and the batched query over all shards.

    points: this rank's points (the rows of its shard_range) or all n_total points (the
    shard's rows are taken); a torch CUDA tensor or a host array.  Every rank passes the
    same d, r, seed and options; group is the torch.distributed group of the shards."""

    def __init__(self, points, n_total: int, d: int, r: int, seed: int, rank: int, world: int, group=None, **opts):
        from . import fclsh

        self.lo, self.hi = shard_range(n_total, rank, world)
        t, rep = global_shape(n_total, d, r, seed, t=opts.pop("t", None), replicate=opts.pop("replicate", 0),
                              approx_c=opts.pop("approx_c", 0.0))
        self.t, self.rep = t, rep
        local = points[self.lo:self.hi] if points.shape[0] == n_total and world > 1 else points
        self.index = None
        if self.hi > self.lo:
            self.index = fclsh.build(local, d, r, seed, t=t, replicate=rep if rep > 1 else 0, **opts)
        self.group = group

    def local_query(self, queries, radius: int, radii=None):
        """This shard's answers (local ids) as (offs, ids, collisions, candidates)."""
        nq = queries.shape[0] if len(queries.shape) > 1 else 1
        if self.index is None:
            z = np.zeros(nq, np.uint64)
            return np.zeros(nq + 1, np.uint64), np.zeros(0, np.uint32), z, z
        res = self.index.query(queries, radius, radii)
        return res.offs, res.ids, res.collisions, res.candidates

    def query(self, queries, radius: int, radii=None):
        """Every shard's answers, merged into global ids (a collective over the group)."""
        from . import fclsh

        offs, ids, coll, cand = gather_answers(self.local_query(queries, radius, radii), self.lo, self.group)
        return fclsh.QueryResult(offs, ids, coll, cand)

    def free(self):
        if self.index is not None:
            self.index.free()
            self.index = None
