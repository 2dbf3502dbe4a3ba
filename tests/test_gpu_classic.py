"""Classic bit-sampling LSH on the GPU (Sec. 2.2; the baseline of Sec. 4.1) against the
classic oracle: its samples and seed vector, the keys the build stored in every table, and
every query's ids and #Collisions / #Candidates through the batched and plain paths.  The
index has false negatives (recall below 1 at distance r, about delta), which covering LSH
on the same points does not."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _points(rng, n, d):
    words = (d + 63) // 64
    a = rng.integers(0, 2**63, size=(n, words), dtype=np.uint64) * np.uint64(2) + rng.integers(
        0, 2, size=(n, words), dtype=np.uint64)
    if d % 64:
        a[:, -1] &= np.uint64((1 << (d % 64)) - 1)
    return a


def _planted(rng, pts, d, dist, count):
    q = pts[:count].copy()
    for i in range(count):
        for c in rng.choice(d, size=dist, replace=False):
            q[i, c >> 6] ^= np.uint64(1) << np.uint64(c & 63)
    return q


# (d, r, n, tables): the covering table count with one part and with two (t chunks of W - 1
# tables), and a count of its own (one chunk of 100 tables)
@pytest.mark.parametrize("d,r,n,tables", [(128, 6, 3000, 0), (1024, 12, 1500, 0), (100, 5, 2500, 100)])
def test_classic_index_matches_the_classic_oracle(d, r, n, tables):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02620_gb300 import fclsh

    rng = np.random.default_rng(d + r)
    pts = _points(rng, n, d)
    seed, delta = 31 + d, 0.1
    idx = fclsh.build(pts, d, r, seed, classic_delta=delta, classic_tables=tables)
    L = idx.T
    if tables:
        assert L == tables
    else:
        assert L == oracle.derive_params(seed, d, r).T       # the covering index's table count
    k = oracle.classic_rule_k(L, r, d, delta)
    cp = oracle.classic_params(seed, d, L, k)
    samples, b = idx.classic_params()
    assert np.array_equal(samples, cp.samples) and np.array_equal(b, cp.b)
    keys = oracle.classic_keys(cp, pts)
    assert np.array_equal(idx.export_keys(np.arange(n, dtype=np.uint32)), keys)
    assert np.array_equal(idx.hash(pts[:300]), keys[:, :300])
    qs = np.concatenate([_planted(rng, pts, d, r, 40), _planted(rng, pts[40:], d, r // 2, 20), _points(rng, 10, d)])
    want = [oracle.classic_query(cp, pts, keys, q, r) for q in qs]
    for res in (idx.query(torch.from_numpy(qs.view(np.int64)).cuda(), r), idx.query_plain(qs, r)):
        for i, (ids, ncoll, ncand) in enumerate(want):
            assert np.array_equal(res.of(i), ids), i
            assert int(res.collisions[i]) == ncoll and int(res.candidates[i]) == ncand, i
    with pytest.raises(fclsh.FclshError):
        idx.params()                                          # no covering parameters
    idx.free()


def test_classic_misses_planted_neighbours_that_covering_lsh_finds():
    """Points planted at distance exactly r: classic LSH (delta = 0.1) misses about a tenth of
    them, covering LSH none (Tables 3 and 4 of the paper show the same contrast)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02620_gb300 import fclsh

    rng = np.random.default_rng(1)
    d, r, n = 128, 8, 20_000
    pts = _points(rng, n, d)
    qs = _planted(rng, pts, d, r, 2000)
    q_dev = torch.from_numpy(qs.view(np.int64)).cuda()
    cov = fclsh.build(pts, d, r, 5)
    cls = fclsh.build(pts, d, r, 5, classic_delta=0.1)
    found_cov = cov.query(q_dev, r)
    found_cls = cls.query(q_dev, r)
    hit_cov = np.array([i in found_cov.of(i) for i in range(len(qs))])
    hit_cls = np.array([i in found_cls.of(i) for i in range(len(qs))])
    assert hit_cov.all()
    k = oracle.classic_rule_k(cls.T, r, d, 0.1)
    miss_p = (1 - (1 - r / d) ** k) ** cls.T
    miss = 1 - hit_cls.mean()
    assert 0 < miss and abs(miss - miss_p) < 4 * (miss_p * (1 - miss_p) / len(qs)) ** 0.5
    cov.free()
    cls.free()
