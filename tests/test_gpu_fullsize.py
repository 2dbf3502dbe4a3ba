"""Parity at the full workload sizes, in the launch configuration the benchmark times.

For each workload the index is built from device-resident points in the
benchmark's configuration (the autotuner's kernel shapes and hash kernel).  The oracle then checks what it can compute one by
one at that size: the parameters, every key of sampled points in every table,
complete buckets of sampled tables, and sampled queries' answers (linear scan,
the plain definition).  All queries are checked against the GPU linear scan
(an independent kernel), and every reported id is re-verified on the host.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1602_02620_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

torch = pytest.importorskip("torch")

_POP = np.array([bin(i).count("1") for i in range(256)], dtype=np.uint8)


def _popcount_rows(a: np.ndarray) -> np.ndarray:
    return _POP[a.view(np.uint8)].reshape(a.shape[0], -1).sum(axis=1)


@pytest.mark.parametrize("cfg", [2, 3, 4, 5, 8])
def test_full_size_workload(cfg):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02620_gb300 import fclsh

    c = wl.CONFIGS[cfg]
    pts = wl.points(cfg)
    nq = c["nq"] if c["nq"] else 20_000
    qs, _ = wl.queries(cfg, pts, nq)
    seed = c["seed"] + 1000
    d, r = c["d"], c["r"]
    bopts = wl.build_options(cfg)                                 # e.g. replication
    p = oracle.derive_params(seed, d, r, rep=bopts.get("replicate", 1))
    # the benchmark's launch configuration: kernel shapes and hash kernel from the autotuner
    # (the same cache file bench.py uses), then an index built with them
    pts_dev = torch.from_numpy(pts.view(np.int64)).cuda()
    q_dev = torch.from_numpy(qs.view(np.int64)).cuda()
    cache = os.path.join(ROOT, "paper_1602_02620_gb300", "_build", "autotune.json")
    idx0 = fclsh.build(pts_dev, d, r, seed, **bopts)
    tuned = idx0.autotune(q_dev[: min(nq, 4096)], r, cache)
    idx0.free()
    idx = fclsh.build(pts_dev, d, r, seed, hash_tile=tuned["hash_tile"], **bopts)
    idx.set_tuning(**tuned)
    assert idx.n == c["n"] and idx.T == p.T

    perm, part_off, m, b = idx.params()
    assert np.array_equal(perm, p.perm) and np.array_equal(m, p.m) and np.array_equal(b, p.b)

    rng = np.random.default_rng(cfg)
    sample = np.sort(rng.choice(c["n"], size=64, replace=False))
    assert np.array_equal(idx.hash(pts[sample]), oracle.keys_direct(p, pts[sample]))

    for tau in (0, p.T // 2 + 1, p.T - 1):                       # complete buckets of sampled tables
        ok, oi = oracle.table(p, pts, tau)
        probe = np.unique(ok[rng.integers(0, c["n"], size=40)])
        for key in probe[:20]:
            assert np.array_equal(idx.bucket(tau, int(key)), oi[ok == key]), (tau, int(key))

    res = idx.query(q_dev, r)                                     # the batched path, as benchmarked
    brute = idx.bruteforce(q_dev, r)
    assert np.array_equal(res.offs, brute.offs) and np.array_equal(res.ids, brute.ids)
    for i in rng.choice(nq, size=12, replace=False):
        assert np.array_equal(res.of(i), oracle.linear_scan(pts, qs[i], r)), i
    counts = np.diff(res.offs)
    owner = np.repeat(np.arange(nq), counts.astype(np.int64))
    dist = _popcount_rows(pts[res.ids] ^ qs[owner])
    assert np.all(dist <= r)
    assert np.all(res.candidates >= counts) and np.all(res.collisions >= res.candidates)

    if cfg == 5:                                                  # served form on the full index
        reqs = wl.request_stream(5, 24, rate_per_s=2000.0)
        srv = fclsh.Server(idx, slots=4)
        at, tickets = 0, []
        for _, size, radius in reqs:
            size = min(size, 800)
            blk = qs[at % (nq - size): at % (nq - size) + size]
            tickets.append((srv.submit(blk, radius), blk, radius))
            at += size
        for t, blk, radius in tickets:
            got, _ = srv.wait(t)
            want = idx.query(blk, radius)
            assert np.array_equal(got.offs, want.offs) and np.array_equal(got.ids, want.ids)
            j = blk.shape[0] // 2
            assert np.array_equal(got.of(j), oracle.linear_scan(pts, blk[j], radius))
        srv.close()
    idx.free()
