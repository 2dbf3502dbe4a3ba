"""Bounded waits: when the tensor-core hash kernel's operand never arrives, its waits run
out (about two seconds), the kernel stops cleanly and the call returns FCLSH_ETIMEOUT; the
same index then hashes correctly, and a build that timed out leaks nothing.

The missing operand is a copy the kernel is told not to request (a flag nothing sets);
no fault, trap or endless loop is involved.
"""
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
    yield
    fclsh.debug_withhold_hash_loads(False)


def test_hash_wait_runs_out_and_the_index_stays_usable():
    from paper_1602_02620_gb300 import fclsh as fc

    rng = np.random.default_rng(1)
    d, r, n = 128, 6, 2000
    pts = rng.integers(0, 2**63, size=(n, 2), dtype=np.uint64)
    idx = fc.build(pts, d, r, 3, hash_tile=2)
    p = oracle.derive_params(3, d, r)
    want = oracle.keys_direct(p, pts[:200])
    fc.debug_withhold_hash_loads(True)
    try:
        with pytest.raises(fc.FclshError) as e:
            idx.hash(pts[:200])
        assert e.value.status == fc.ETIMEOUT
    finally:
        fc.debug_withhold_hash_loads(False)
    assert np.array_equal(idx.hash(pts[:200]), want)          # the device and the index still work
    res = idx.query(pts[:20], r)
    for i in range(20):
        assert res.of(i).tolist() == oracle.linear_scan(pts, pts[i], r).tolist()
    idx.free()

    base = fc.debug_pool_used()
    fc.debug_withhold_hash_loads(True)
    try:
        with pytest.raises(fc.FclshError) as e:
            fc.build(pts, d, r, 3, hash_tile=2)
        assert e.value.status == fc.ETIMEOUT
    finally:
        fc.debug_withhold_hash_loads(False)
    assert fc.debug_pool_used() == base
    again = fc.build(pts, d, r, 3, hash_tile=2)
    assert np.array_equal(again.hash(pts[:200]), want)
    again.free()


def test_hash_wait_runs_out_after_mmas_were_issued():
    """The third operand chunk is withheld: the MMAs of the first two chunks and the copy of
    the fourth are in flight when the wait runs out; the kernel drains them before it
    releases its tensor memory, and the index then hashes and queries correctly."""
    from paper_1602_02620_gb300 import fclsh as fc

    rng = np.random.default_rng(2)
    d, r, n = 128, 8, 3000                                    # W = 512: 22 chunks of 24 tables
    pts = rng.integers(0, 2**63, size=(n, 2), dtype=np.uint64)
    idx = fc.build(pts, d, r, 5, hash_tile=2)
    p = oracle.derive_params(5, d, r)
    want = oracle.keys_direct(p, pts[:300])
    fc.debug_withhold_hash_loads(True, chunk=2)
    try:
        with pytest.raises(fc.FclshError) as e:
            idx.hash(pts[:300])
        assert e.value.status == fc.ETIMEOUT
    finally:
        fc.debug_withhold_hash_loads(False)
    assert np.array_equal(idx.hash(pts[:300]), want)
    res = idx.query(pts[:20], r)
    for i in range(20):
        assert res.of(i).tolist() == oracle.linear_scan(pts, pts[i], r).tolist()
    idx.free()
