"""Multi-process sharding logic on CPU: two gloo ranks, each answering for its
own contiguous id range, gather to exactly the single-process answer."""
import os
import socket

import numpy as np
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


def _answers(pts, qs, radius):
    offs, ids = [0], []
    for q in qs:
        r = oracle.linear_scan(pts, q, radius)
        ids.extend(r.tolist())
        offs.append(len(ids))
    n = len(qs)
    return (np.array(offs, np.uint64), np.array(ids, np.uint32), np.zeros(n, np.uint64), np.zeros(n, np.uint64))


def _worker(rank, world, port, pts, qs, radius, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = shard.shard_range(pts.shape[0], rank, world)
    local = _answers(pts[lo:hi], qs, radius)
    offs, ids, _, _ = shard.gather_answers(local, lo)
    if rank == 0:
        np.savez(out_path, offs=offs, ids=ids)
    dist.barrier()
    dist.destroy_process_group()


def test_shard_ranges_cover_once():
    for n in (1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            ranges = [shard.shard_range(n, k, world) for k in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(ranges[k][1] == ranges[k + 1][0] for k in range(world - 1))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1


def test_two_ranks_gather_equals_single_process(tmp_path):
    rng = np.random.default_rng(0)
    pts = rng.integers(0, 2**63, size=(3001, 2), dtype=np.uint64)
    qs = pts[rng.integers(0, 3001, size=20)].copy()
    qs[:, 0] ^= np.uint64(0b101)
    radius = 40
    out = str(tmp_path / "merged.npz")
    mp.spawn(_worker, args=(2, _free_port(), pts, qs, radius, out), nprocs=2, join=True)
    got = np.load(out)
    want = _answers(pts, qs, radius)
    assert np.array_equal(got["offs"], want[0]) and np.array_equal(got["ids"], want[1])
