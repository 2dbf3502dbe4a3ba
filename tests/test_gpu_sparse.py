"""Sparse (CSR) input: rows of set coordinates packed into bit vectors on the device, and an
index built from them equal to the one built from the same rows packed on the host."""
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


def to_csr(pts, d):
    """Host reference: the set coordinates of each packed row (ascending)."""
    bits = np.unpackbits(pts.view(np.uint8).reshape(pts.shape[0], -1), axis=1, bitorder="little")[:, :d]
    rows, cols = np.nonzero(bits)
    indptr = np.zeros(pts.shape[0] + 1, np.uint64)
    np.add.at(indptr, rows + 1, 1)
    return np.cumsum(indptr).astype(np.uint64), cols.astype(np.uint32)


def test_pack_sparse_matches_host_packing():
    fc = F()
    rng = np.random.default_rng(2)
    for d in (1, 64, 100, 1000, 140_214):
        n = 700
        lens = rng.integers(0, 40, size=n)
        indptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
        indices = rng.integers(0, d, size=int(indptr[-1])).astype(np.uint32)   # unsorted, with repeats
        want = np.zeros((n, (d + 63) // 64), np.uint64)
        for i in range(n):
            for c in indices[indptr[i]:indptr[i + 1]]:
                want[i, c >> 6] |= np.uint64(1) << np.uint64(c & 63)
        assert np.array_equal(fc.pack_sparse(indptr, indices, d), want), d
        out = torch.zeros((n, (d + 63) // 64), dtype=torch.int64, device="cuda")
        fc.pack_sparse(torch.from_numpy(indptr.view(np.int64)).cuda(), torch.from_numpy(indices.view(np.int32)).cuda(),
                       d, out=out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint64), want), d


def test_pack_sparse_rejects_bad_rows():
    fc = F()
    indptr = np.array([0, 2, 3], np.uint64)
    with pytest.raises(fc.FclshError) as e:
        fc.pack_sparse(indptr, np.array([1, 64, 5], np.uint32), 64)          # 64 is not below d
    assert e.value.status == fc.EINVAL
    with pytest.raises(fc.FclshError):
        fc.pack_sparse(np.array([0, 3, 2], np.uint64), np.array([1, 2, 3], np.uint32), 64)   # runs backwards
    with pytest.raises(fc.FclshError):
        fc.pack_sparse(np.array([0, 2, 9], np.uint64), np.array([1, 2, 3], np.uint32), 64)   # past nnz
    ok = fc.pack_sparse(np.array([0, 0, 3], np.uint64), np.array([1, 2, 3], np.uint32), 64)   # an empty row
    assert ok[0, 0] == 0 and int(ok[1, 0]) == 0b1110


@pytest.mark.parametrize("cfg,n", [(7, 3000), (6, 2000)])
def test_build_sparse_equals_build(cfg, n):
    fc = F()
    w = wl.make(cfg, n=n, nq=30)
    indptr, indices = to_csr(w.points, w.d)
    a = fc.build(w.points, w.d, w.r, w.index_seed)
    b = fc.build_sparse(indptr, indices, w.d, w.r, w.index_seed)
    c = fc.build_sparse(torch.from_numpy(indptr.view(np.int64)).cuda(),
                        torch.from_numpy(indices.view(np.int32)).cuda(), w.d, w.r, w.index_seed)
    assert a.info == b.info == c.info
    for tau in (0, a.T - 1):
        ka, ia = a.export_table(tau)
        for other in (b, c):
            kb, ib = other.export_table(tau)
            oa, ob = np.lexsort((ia, ka)), np.lexsort((ib, kb))
            assert np.array_equal(ka[oa], kb[ob]) and np.array_equal(ia[oa], ib[ob])
    ra, rb = a.query(w.queries, w.r), b.query(w.queries, w.r)
    assert np.array_equal(ra.ids, rb.ids) and np.array_equal(ra.offs, rb.offs)
    for i in range(0, 30, 6):
        assert rb.of(i).tolist() == oracle.linear_scan(w.points, w.queries[i], w.r).tolist()
    for x in (a, b, c):
        x.free()
