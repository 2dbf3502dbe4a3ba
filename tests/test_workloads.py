"""The seeded input generators: shapes, determinism and the stated structure."""
import numpy as np

import oracle
from paper_1602_02620_gb300 import workloads as wl


def _popcount_rows(a):
    return np.array([sum(bin(int(w)).count("1") for w in row) for row in a])


def test_uniform_planted_queries():
    w = wl.make(1)
    assert w.points.shape == (10_000, 1) and w.queries.shape == (200, 1)
    again = wl.make(1)
    assert np.array_equal(w.points, again.points) and np.array_equal(w.queries, again.queries)
    planted = w.meta["planted"]
    assert planted.sum() == 100
    for i in np.nonzero(planted)[0]:
        src, k = int(w.meta["src"][i]), int(w.meta["k"][i])
        assert 0 <= k <= 3 and oracle.hamming(w.points[src], w.queries[i]) == k
    frac = _popcount_rows(w.points[:2000]).mean() / 64
    assert abs(frac - 0.5) < 0.01


def test_prefix_stable_and_masked():
    a = wl.points(2, 5000)
    b = wl.points(2, 1000)
    assert np.array_equal(a[:1000], b)
    q, meta = wl.queries(2, a, 40)
    q2, _ = wl.queries(2, a, 20, first=20)
    assert np.array_equal(q[20:], q2)


def test_clustered_noise_levels():
    pts = wl.points(3, 20_000)
    c = wl.centres(wl.CONFIGS[3])
    assert c.shape == (4096, 4)
    # each point is within a few flips of some centre: distance to its nearest centre ~ 0.05 * 256
    q, meta = wl.queries(3, pts, 200)
    d = [oracle.hamming(q[i], c[meta["centre"][i]]) for i in range(200)]
    assert 2 <= np.mean(d) / 256 * 100 <= 9          # p in [0.02, 0.08] -> 5% on average


def test_sparse_near_duplicates():
    pts = wl.points(4, 20_000)
    dens = _popcount_rows(pts[:3000]).mean() / 1024
    assert abs(dens - 0.02) < 0.003
    q, meta = wl.queries(4, pts, 50)
    for i in np.nonzero(meta["planted"])[0]:
        assert oracle.hamming(pts[meta["src"][i]], q[i]) == meta["k"][i] <= 20


def test_request_stream():
    reqs = wl.request_stream(5, 500, rate_per_s=1000.0)
    t = np.array([r[0] for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert 0.3 < t[-1] / 0.5 < 3.0
    assert {r[2] for r in reqs} <= {4, 8, 12, 16}
    assert all(1 <= r[1] <= 4096 for r in reqs)


def test_sparse_skewed_highd():
    """The Enron- and MovieLens-shaped sets: d bits, ~lmin + lmean set bits, low coordinates
    popular, near-duplicate planted queries at the stated distances, prefix-stable."""
    for cfg, mean_lo, mean_hi in ((6, 120, 175), (7, 65, 105)):
        c = wl.CONFIGS[cfg]
        pts = wl.points(cfg, 3000)
        assert pts.shape == (3000, (c["d"] + 63) // 64)
        assert np.array_equal(wl.points(cfg, 500), pts[:500])
        nnz = _popcount_rows(pts[:600])
        assert mean_lo < nnz.mean() < mean_hi and nnz.min() >= c["lmin"]
        last = pts[:, -1]
        assert not np.any(last >> np.uint64(c["d"] % 64)) if c["d"] % 64 else True   # no bit past d
        bits = np.unpackbits(pts[:600].view(np.uint8), axis=1, bitorder="little")[:, : c["d"]]
        lowq, highq = bits[:, : c["d"] // 4].sum(), bits[:, 3 * c["d"] // 4:].sum()
        assert lowq > 2.5 * highq                               # density ~ 1/sqrt(c): skewed to low c
        q, meta = wl.queries(cfg, pts, 30)
        for i in np.nonzero(meta["planted"])[0]:
            assert oracle.hamming(pts[meta["src"][i]], q[i]) == meta["k"][i] <= c["r"]


def test_replicated_workload_options():
    """Workload 8 is workload 2's shape at r = 2, indexed with four copies (Algorithm 1)."""
    assert wl.build_options(8) == {"replicate": 4}
    assert wl.build_options(2) == {}
    w = wl.make(8, n=2000, nq=20)
    for i in np.nonzero(w.meta["planted"])[0]:
        assert oracle.hamming(w.points[w.meta["src"][i]], w.queries[i]) == w.meta["k"][i] <= 2
