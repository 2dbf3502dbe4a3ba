"""Edge sizes on the GPU against the oracle: the largest dimension the library takes
(262,144 bits, 4,096 words per point) and the largest per-part code (W = 2,048) with three
parts."""
import numpy as np
import pytest

import oracle

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


def test_largest_dimension():
    fc = F()
    rng = np.random.default_rng(262)
    d, r, n = 262_144, 5, 300
    words = d // 64
    pts = np.zeros((n, words), np.uint64)
    for i in range(n):
        for c in rng.choice(d, size=int(rng.integers(10, 200)), replace=False):
            pts[i, c >> 6] |= np.uint64(1) << np.uint64(c & 63)
    pts[7] = pts[3]
    pts[8] = pts[3]
    pts[8, words - 1] ^= np.uint64(1) << np.uint64(63)      # the last coordinate, d - 1
    idx = fc.build(pts, d, r, 9)
    p = oracle.derive_params(9, d, r)
    assert idx.words == words and idx.tuning()["hash_tile"] == 3
    assert np.array_equal(idx.hash(pts[:20]), oracle.keys_fht(p, pts[:20]))
    keys, ids = idx.export_table(p.T - 1)
    order = np.lexsort((ids, keys))
    ok, oi = oracle.table(p, pts, p.T - 1)
    assert np.array_equal(keys[order], ok) and np.array_equal(ids[order], oi)
    qs = pts[[3, 8, 100, 250]].copy()
    qs[2, 0] ^= np.uint64(5)
    res = idx.query(qs, r)
    plain = idx.query_plain(qs, r)
    for i in range(qs.shape[0]):
        want = oracle.linear_scan(pts, qs[i], r).tolist()
        assert res.of(i).tolist() == want and plain.of(i).tolist() == want
    assert res.of(0).tolist() == [3, 7, 8]
    idx.free()


def test_largest_code_with_three_parts():
    fc = F()
    rng = np.random.default_rng(32)
    d, r, n = 96, 32, 400                              # t = 3 parts of 32 bits, r' = 10, W = 2,048
    pts = rng.integers(0, 2**63, size=(n, 2), dtype=np.uint64)
    pts[:, 1] &= np.uint64((1 << 32) - 1)
    idx = fc.build(pts, d, r, 4)
    p = oracle.derive_params(4, d, r)
    assert (idx.t, idx.W, idx.T) == (3, 2048, 3 * 2047) == (p.t, p.W, p.T)
    assert np.array_equal(idx.hash(pts[:50]), oracle.keys_fht(p, pts[:50]))
    qs = pts[rng.integers(0, n, size=12)].copy()
    for i in range(12):
        for c in rng.choice(d, size=int(rng.integers(0, 34)), replace=False):
            qs[i, c >> 6] ^= np.uint64(1) << np.uint64(c & 63)
    for rho in (0, 10, 32):
        res = idx.query(qs, rho)
        for i in range(12):
            assert res.of(i).tolist() == oracle.linear_scan(pts, qs[i], rho).tolist()
    idx.free()
