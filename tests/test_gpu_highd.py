"""Very high-dimensional sparse points (the Enron and MovieLens shapes of Table 2) on the GPU.

Parts of tens of thousands of positions do not fit the hash kernels' staged column
lists, so the index sketches by scattering each point's set bits (hash_tile 3).  Keys,
tables, queries and counters must equal the oracle's bit for bit; where both the
column-list gather and the scatter sketch apply they must agree.
"""
import numpy as np
import pytest

import oracle
from paper_1602_02620_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02620_gb300 import fclsh

    fclsh.lib()


def F():
    from paper_1602_02620_gb300 import fclsh

    return fclsh


def rand_points(rng, n, d):
    words = (d + 63) // 64
    a = rng.integers(0, 2**63, size=(n, words), dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=(n, words), dtype=np.uint64)
    if d % 64:
        a[:, -1] &= np.uint64((1 << (d % 64)) - 1)
    return a


@pytest.mark.parametrize("cfg,n", [(6, 3000), (7, 2500)])
def test_highd_keys_tables_queries(cfg, n):
    w = wl.make(cfg, n=n, nq=40)
    idx = F().build(w.points, w.d, w.r, w.index_seed)
    p = oracle.derive_params(w.index_seed, w.d, w.r)
    assert (idx.t, idx.W, idx.T) == (p.t, p.W, p.T)
    if cfg == 7:
        assert idx.tuning()["hash_tile"] == 3          # parts of ~70,000 positions: scatter sketch
    sample = w.points[:64]
    want = oracle.keys_fht(p, sample)
    assert np.array_equal(idx.hash(sample), want)
    for tau in sorted({0, p.T // 2, p.T - 1}):
        keys, ids = idx.export_table(tau)
        order = np.lexsort((ids, keys))
        ok, oi = oracle.table(p, w.points, tau)
        assert np.array_equal(keys[order], ok) and np.array_equal(ids[order], oi)
    res = idx.query(w.queries, w.r)
    plain = idx.query_plain(w.queries[:6], w.r)
    for i, q in enumerate(w.queries):
        truth = oracle.linear_scan(w.points, q, w.r).tolist()
        assert res.of(i).tolist() == truth
        if i < 6:
            assert plain.of(i).tolist() == truth
    # counters of a few queries against the oracle's Strategy 2, on tables sorted from the
    # oracle's Algorithm 2 keys of every point (the direct route would take minutes here)
    kall = oracle.keys_fht(p, w.points)
    ids_all = np.tile(np.arange(n, dtype=np.uint32), (p.T, 1))
    order = np.argsort(kall, axis=1, kind="stable")          # (key, id) order: ids ascend within a key
    tables = (np.ascontiguousarray(np.take_along_axis(kall, order, 1)),
              np.ascontiguousarray(np.take_along_axis(ids_all, order, 1)))
    for i in range(0, 40, 4):
        ids, ncoll, ncand = oracle.query(p, w.points, tables, w.queries[i], w.r)
        assert ids.tolist() == res.of(i).tolist()
        assert (int(res.collisions[i]), int(res.candidates[i])) == (ncoll, ncand)
    idx.free()


@pytest.mark.parametrize("d,r,t,n", [
    (64, 3, None, 3000),       # W = 16: the small-W scatter kernel
    (128, 8, None, 2000),      # W = 512, specific construction
    (1024, 20, None, 1500),    # t = 2, W = 2048 per part
    (300, 7, 3, 1200),         # general construction per part
    (40_000, 4, None, 800),    # W = 32 over 40,000 positions (column lists too long to stage)
    (20_000, 13, 2, 900),      # W = 128, two parts of 10,000
    (8_192, 4, None, 700),     # dense long points: too many set bits to list, the packed words are read
])
def test_scatter_sketch_matches_oracle(d, r, t, n):
    rng = np.random.default_rng(d + r)
    if d > 8192:   # sparse rows (a few hundred set bits), like the high-dimensional sets
        pts = np.zeros((n, (d + 63) // 64), np.uint64)
        for i in range(n):
            for c in rng.choice(d, size=int(rng.integers(20, 300)), replace=False):
                pts[i, c >> 6] |= np.uint64(1) << np.uint64(c & 63)
    else:
        pts = rand_points(rng, n, d)
    pts[0] = 0
    pts[7] = pts[3]
    seed = 31 + d + r
    p = oracle.derive_params(seed, d, r, t=t)
    want = oracle.keys_fht(p, pts[:300])
    idx = F().build(pts, d, r, seed, t=t, hash_tile=3)
    assert idx.tuning()["hash_tile"] == 3
    assert np.array_equal(idx.hash(pts[:300]), want)
    keys, ids = idx.export_table(p.T - 1)
    order = np.lexsort((ids, keys))
    ok, oi = oracle.table(p, pts, p.T - 1)
    assert np.array_equal(keys[order], ok) and np.array_equal(ids[order], oi)
    # queries (S1 by scatter for parts of >= 2,048 positions, one warp per distance for
    # points of >= 32 words) report the linear-scan answer
    qs = pts[rng.integers(0, n, size=24)].copy()
    for i in range(24):
        for c in rng.choice(d, size=int(rng.integers(0, r + 2)), replace=False):
            qs[i, c >> 6] ^= np.uint64(1) << np.uint64(c & 63)
    res = idx.query(qs, r)
    for i in range(24):
        assert res.of(i).tolist() == oracle.linear_scan(pts, qs[i], r).tolist()
    # the gather kernels give the same keys where their column lists fit
    try:
        idx.set_tuning(**dict(idx.tuning(), hash_tile=0))
    except F().FclshError:
        pass
    else:
        assert np.array_equal(idx.hash(pts[:300]), want)
    idx.free()


def test_scatter_refuses_overfull_columns():
    """W = 2 puts every position of a 20,000-bit part on column 1: the 64-bit scatter sums
    could wrap, so the index refuses the scatter sketch (and falls back where lists fit)."""
    rng = np.random.default_rng(3)
    d = 20_000
    pts = np.zeros((50, (d + 63) // 64), np.uint64)
    pts[:, :4] = rng.integers(0, 2**63, size=(50, 4), dtype=np.uint64)
    with pytest.raises(F().FclshError):
        F().build(pts, d, 0, 1, hash_tile=3)
    with pytest.raises(F().FclshError):
        F().build(pts, d, 0, 1)                          # neither staged lists nor the scatter fit
