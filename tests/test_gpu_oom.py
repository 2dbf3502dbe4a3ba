"""Out-of-memory paths: every device allocation of a build, a query and a server can fail,
and each failure must return FCLSH_ENOMEM with nothing left allocated.

The failure is injected on the host (the library's allocation wrapper reports
cudaErrorMemoryAllocation for the k-th request), so no GPU runs out of memory.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02620_gb300 import fclsh

    fclsh.lib()
    yield
    fclsh.debug_fail_alloc(-1)


def F():
    from paper_1602_02620_gb300 import fclsh

    return fclsh


def _data(d=128, n=6000, nq=48, seed=3):
    rng = np.random.default_rng(seed)
    words = (d + 63) // 64
    pts = rng.integers(0, 2**63, size=(n, words), dtype=np.uint64)
    qs = pts[rng.integers(0, n, size=nq)].copy()
    for i in range(nq):
        for c in rng.choice(d, size=int(rng.integers(0, 5)), replace=False):
            qs[i, c >> 6] ^= np.uint64(1) << np.uint64(c & 63)
    return pts, qs


@pytest.mark.parametrize("hash_tile", [0, 2])
def test_build_fails_cleanly_at_every_allocation(hash_tile):
    fc = F()
    pts, qs = _data()
    ref = fc.build(pts, 128, 6, 11, hash_tile=hash_tile)
    want = ref.query(qs, 6)
    ref.free()
    base = fc.debug_pool_used()
    failures = 0
    for k in range(200):
        fc.debug_fail_alloc(k)
        try:
            idx = fc.build(pts, 128, 6, 11, hash_tile=hash_tile)
        except fc.FclshError as e:
            fc.debug_fail_alloc(-1)
            assert e.status == fc.ENOMEM, str(e)
            assert fc.debug_pool_used() == base, k
            failures += 1
            continue
        fc.debug_fail_alloc(-1)
        got = idx.query(qs, 6)                      # fewer than k allocations: the index is whole
        assert np.array_equal(got.offs, want.offs) and np.array_equal(got.ids, want.ids)
        idx.free()
        break
    else:
        pytest.fail("the build never completed")
    assert failures >= 5                            # the build allocates at several places
    assert fc.debug_pool_used() == base


def _run(fc, idx, qs, call):
    """One call of the given kind; whatever it created is released before it returns."""
    if call == "query":
        return idx.query(qs, 6)
    if call == "plain":
        return idx.query_plain(qs[:5], 6)
    if call == "context":
        ctx = None
        try:
            ctx = idx.context()
            ctx.query_async(torch.from_numpy(qs.view(np.int64)).cuda(), 6)
            ctx.wait()
            return ctx.fetch()
        finally:
            if ctx is not None:
                ctx.close()
    srv = None
    try:
        srv = fc.Server(idx, slots=2)
        got, _ = srv.wait(srv.submit(qs, 6))
        return got
    finally:
        if srv is not None:
            srv.close()


def test_queries_and_server_fail_cleanly():
    fc = F()
    pts, qs = _data(seed=5)
    idx = fc.build(pts, 128, 6, 12)
    want = idx.query(qs, 6)
    base = fc.debug_pool_used()
    for call in ("query", "plain", "context", "server"):
        failures = 0
        for k in range(100):
            fc.debug_fail_alloc(k)
            try:
                got = _run(fc, idx, qs, call)
            except fc.FclshError as e:
                fc.debug_fail_alloc(-1)
                assert e.status == fc.ENOMEM, (call, k, str(e))
                assert fc.debug_pool_used() == base, (call, k)
                failures += 1
                continue
            fc.debug_fail_alloc(-1)
            n = 5 if call == "plain" else qs.shape[0]
            assert np.array_equal(got.ids, want.ids[: int(want.offs[n])]), (call, k)
            break
        else:
            pytest.fail("%s never completed" % call)
        assert failures >= 1, call
        assert fc.debug_pool_used() == base, call
    idx.free()


def test_context_reused_after_failed_growth():
    """A query context whose buffers failed to grow answers later batches correctly: a
    failed growth leaves no capacity behind that looks usable, and a captured batch is
    never replayed on buffers that were replaced."""
    fc = F()
    pts, qs = _data(seed=9, nq=64)
    idx = fc.build(pts, 128, 6, 13)
    small = torch.from_numpy(qs[:16].view(np.int64)).cuda()
    big_np = np.tile(qs, (40, 1))                          # 2,560 queries: more than the first capacity
    big = torch.from_numpy(big_np.view(np.int64)).cuda()
    want_small = idx.query(qs[:16], 6)
    want_big = idx.query(big_np, 6)
    ctx = idx.context()
    try:
        for _ in range(3):                                 # eager, then captured, then replayed
            ctx.query_async(small, 6)
            ctx.wait()
            got = ctx.fetch()
            assert np.array_equal(got.ids, want_small.ids) and np.array_equal(got.offs, want_small.offs)
        failures = 0
        for k in range(12):
            fc.debug_fail_alloc(k)
            try:
                ctx.query_async(big, 6)
                ctx.wait()
                got = ctx.fetch()
                fc.debug_fail_alloc(-1)
                assert np.array_equal(got.ids, want_big.ids) and np.array_equal(got.offs, want_big.offs)
                break
            except fc.FclshError as e:
                fc.debug_fail_alloc(-1)
                assert e.status == fc.ENOMEM, str(e)
                failures += 1
            for _ in range(2):                             # the same context, right after the failure
                ctx.query_async(small, 6)
                ctx.wait()
                got = ctx.fetch()
                assert np.array_equal(got.ids, want_small.ids) and np.array_equal(got.offs, want_small.offs)
        assert failures >= 1
    finally:
        fc.debug_fail_alloc(-1)
        ctx.close()
    idx.free()
