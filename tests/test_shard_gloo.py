"""Sharding by points on CPU: gloo ranks each index their own contiguous id range with the
same parameters and answer a batch by the oracle's Strategy 2 query (Sec. 2.2, S1-S3 of
Sec. 4.1) over their shard; the gather must give exactly the single-process answer --
ids and the #Collisions / #Candidates counters, which add up over disjoint shards."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1602_02620_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _strategy2(pts, qs, d, r, seed, radius):
    """The oracle's Strategy 2 answers of a batch over `pts` (local ids), as the arrays a shard sends."""
    p = oracle.derive_params(seed, d, r)
    tables = oracle.build_tables(p, pts)
    offs, ids, coll, cand = [0], [], [], []
    for q in qs:
        i, c, k = oracle.query(p, pts, tables, q, radius)
        ids.extend(i.tolist())
        offs.append(len(ids))
        coll.append(c)
        cand.append(k)
    return (np.array(offs, np.uint64), np.array(ids, np.uint32), np.array(coll, np.uint64),
            np.array(cand, np.uint64))


def _worker(rank, world, port, pts, qs, d, r, seed, radius, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = shard.shard_range(pts.shape[0], rank, world)
    local = _strategy2(pts[lo:hi], qs, d, r, seed, radius)
    offs, ids, coll, cand = shard.gather_answers(local, lo)
    if rank == 0:
        np.savez(out_path, offs=offs, ids=ids, coll=coll, cand=cand)
    dist.barrier()
    dist.destroy_process_group()


def _data(n=3001, d=64, nq=24, seed=0):
    rng = np.random.default_rng(seed)
    pts = rng.integers(0, 2**63, size=(n, 1), dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=(n, 1),
                                                                                           dtype=np.uint64)
    pts[100:140] = pts[7]                                   # copies of one point in the first shard's range
    pts[1600:1620] = pts[7]                                 # ... and in the next one's
    qs = pts[rng.integers(0, n, size=nq)].copy()
    for i in range(nq):
        for pos in rng.choice(d, size=rng.integers(0, 4), replace=False):
            qs[i, pos >> 6] ^= np.uint64(1) << np.uint64(pos & 63)
    qs[0] = pts[7]
    return pts, qs


def test_shard_ranges_cover_once():
    for n in (1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            ranges = [shard.shard_range(n, k, world) for k in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(ranges[k][1] == ranges[k + 1][0] for k in range(world - 1))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("world", [2, 3])
def test_merge_of_shard_answers_equals_the_whole_index(world):
    """The merge alone (no processes): Strategy 2 on each shard, merged, equals Strategy 2 on all."""
    pts, qs = _data()
    d, r, seed = 64, 3, 11
    parts = []
    for k in range(world):
        lo, hi = shard.shard_range(pts.shape[0], k, world)
        parts.append(_strategy2(pts[lo:hi], qs, d, r, seed, r) + (lo,))
    offs, ids, coll, cand = shard.merge(parts)
    want = _strategy2(pts, qs, d, r, seed, r)
    assert np.array_equal(offs, want[0]) and np.array_equal(ids, want[1])
    assert np.array_equal(coll, want[2]) and np.array_equal(cand, want[3])
    assert int(coll[0]) > 0 and int(want[1].size) > 0


def test_two_gloo_ranks_gather_equals_single_process(tmp_path):
    pts, qs = _data()
    d, r, seed = 64, 3, 11
    out = str(tmp_path / "merged.npz")
    mp.spawn(_worker, args=(2, _free_port(), pts, qs, d, r, seed, r, out), nprocs=2, join=True)
    got = np.load(out)
    want = _strategy2(pts, qs, d, r, seed, r)
    assert np.array_equal(got["offs"], want[0]) and np.array_equal(got["ids"], want[1])
    assert np.array_equal(got["coll"], want[2]) and np.array_equal(got["cand"], want[3])
