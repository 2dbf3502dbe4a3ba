"""Checkpoint and resume: an index saved and loaded back has the same parameters, tuning,
keys, buckets and answers as the one that was saved."""
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


def rand_points(rng, n, d):
    words = (d + 63) // 64
    a = rng.integers(0, 2**63, size=(n, words), dtype=np.uint64)
    if d % 64:
        a[:, -1] &= np.uint64((1 << (d % 64)) - 1)
    return a


@pytest.mark.parametrize("d,r,kw", [
    (64, 3, {}),                              # one part, W = 16
    (128, 8, {"hash_tile": 2}),               # the tensor-core hash, W = 512
    (256, 16, {}),                            # two parts
    (40, 2, {"replicate": 3}),                # replication
    (20_000, 5, {"hash_tile": 3}),            # high d, scatter sketch
])
def test_save_load_round_trip(tmp_path, d, r, kw):
    fc = F()
    rng = np.random.default_rng(d + r)
    n = 3000
    pts = rand_points(rng, n, d)
    pts[5:9] = pts[4]
    seed = 21 + d
    a = fc.build(pts, d, r, seed, **kw)
    a.set_tuning(**dict(a.tuning(), query_block=512, hash_set_log2=11, probe_rows=1))
    path = str(tmp_path / "index.fclsh")
    a.save(path)
    b = fc.load(path)
    assert a.info == b.info
    assert a.tuning() == b.tuning()
    for x, y in zip(a.params(), b.params()):
        assert np.array_equal(x, y)
    p = oracle.derive_params(seed, d, r, t=a.t, rep=a.rep)
    assert np.array_equal(b.params()[2], p.m) and np.array_equal(b.params()[3], p.b)
    for tau in sorted({0, a.T // 2, a.T - 1}):
        ka, ia = a.export_table(tau)
        kb, ib = b.export_table(tau)
        oa, ob = np.lexsort((ia, ka)), np.lexsort((ib, kb))
        assert np.array_equal(ka[oa], kb[ob]) and np.array_equal(ia[oa], ib[ob])
    qs = pts[rng.integers(0, n, size=40)].copy()
    for i in range(40):
        for c in rng.choice(d, size=int(rng.integers(0, r + 2)), replace=False):
            qs[i, c >> 6] ^= np.uint64(1) << np.uint64(c & 63)
    for rho in sorted({0, r // 2, r}):
        ra, rb = a.query(qs, rho), b.query(qs, rho)
        assert np.array_equal(ra.offs, rb.offs) and np.array_equal(ra.ids, rb.ids)
        assert np.array_equal(ra.collisions, rb.collisions) and np.array_equal(ra.candidates, rb.candidates)
        for i in range(0, 40, 10):
            assert rb.of(i).tolist() == oracle.linear_scan(pts, qs[i], rho).tolist()
    a.free()
    b.free()
