"""The allocation-free one-query entry point (fclsh_query_plain_noalloc).

It serves callers that cannot allocate device memory while they query (code under an
allocator or pool it does not own, latency-bound loops that must not synchronise); all
of its scratch is one fixed device array inside the library.  Its answers must be
exactly the oracle's Strategy 2 answers -- ids, #Collisions and #Candidates -- and those
of the ordinary plain path, call after call, since every call reuses that array.  The
calls run while the library's allocation-failure hook is armed: an allocation by them
would fail, and the hook is shown to be still armed afterwards.  This file is collected
last so that a run stopping at the first failure has run everything else.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_1602_02620_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _oracle_tables(p, pts):
    keys = np.empty((p.T, pts.shape[0]), np.uint64)
    ids = np.empty((p.T, pts.shape[0]), np.uint32)

    def fill(tau):
        keys[tau], ids[tau] = oracle.table(p, pts, tau)

    with ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2)) as ex:
        list(ex.map(fill, range(p.T)))
    return keys, ids


# (workload, points, queries, hash kernel): the Walsh-Hadamard kernels and the tensor-core
# contraction (hash_tile 2), which the call launches for a single point
@pytest.mark.parametrize("cfg,n,nq,hash_tile", [(2, 30_000, 6, 0), (2, 30_000, 6, 2), (3, 20_000, 6, 0),
                                                (3, 20_000, 6, 2)])
def test_noalloc_matches_the_oracle_on_consecutive_calls(cfg, n, nq, hash_tile):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02620_gb300 import fclsh

    pts = wl.points(cfg, n)
    qs, _ = wl.queries(cfg, pts, nq)
    r, d = wl.CONFIGS[cfg]["r"], wl.CONFIGS[cfg]["d"]
    seed = 4242 + cfg
    idx = fclsh.build(_dev(pts), d, r, seed, hash_tile=hash_tile)
    assert idx.tuning()["hash_tile"] == hash_tile
    p = oracle.derive_params(seed, d, r)
    tables = _oracle_tables(p, pts)
    want = [oracle.query(p, pts, tables, qs[i], r) for i in range(nq)]
    plain = idx.query_plain(qs, r)
    for i in range(nq):
        assert np.array_equal(plain.of(i), want[i][0])
    cap = 4096
    ids = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    counts = torch.zeros(3, dtype=torch.int64, device="cuda")
    q_dev = _dev(qs)

    def check(i):
        ids.fill_(-1)
        idx.query_plain_noalloc(q_dev[i], r, ids, counts)
        torch.cuda.synchronize()
        c = counts.cpu().numpy()
        exp, ncoll, ncand = want[i]
        assert int(c[0]) == exp.shape[0]
        assert int(c[1]) == ncoll and int(c[2]) == ncand
        got = ids[: min(int(c[0]), cap)].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, exp[:cap])

    check(0)                                   # first call on this device sets up the scratch address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    fclsh.debug_fail_alloc(0)                  # the library's next device allocation fails
    try:
        for i in range(nq):                    # consecutive calls share the same scratch
            check(i)
        check(0)
        with pytest.raises(fclsh.FclshError) as e:   # the hook is still armed: nothing was allocated
            idx.query_plain(qs[:1], r)
        assert e.value.status == fclsh.ENOMEM
    finally:
        fclsh.debug_fail_alloc(-1)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    idx.free()


def test_noalloc_rejects_oversized_index_and_host_memory():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02620_gb300 import fclsh

    pts = np.zeros((1, 1), np.uint64)
    idx = fclsh.build(pts, 64, 20, 1)          # t = 2, W = 2048: T = 4,094 tables is the limit
    ids = torch.zeros(16, dtype=torch.int32, device="cuda")
    counts = torch.zeros(3, dtype=torch.int64, device="cuda")
    idx.query_plain_noalloc(_dev(pts)[0], 20, ids, counts)
    torch.cuda.synchronize()
    assert counts.cpu().tolist()[0] == 1 and ids[0].item() == 0
    # host memory is refused by the binding and by the library itself
    with pytest.raises(fclsh.FclshError) as e:
        idx.query_plain_noalloc(torch.zeros(1, dtype=torch.int64), 20, ids, counts)
    assert e.value.status == fclsh.EINVAL
    host_counts = np.zeros(3, np.int64)
    st = fclsh.lib().fclsh_query_plain_noalloc(idx.handle, _dev(pts).data_ptr(), 20, ids.data_ptr(), 16,
                                               host_counts.ctypes.data, None)
    assert st == fclsh.EINVAL
    with pytest.raises(fclsh.FclshError):
        idx.query_plain_noalloc(_dev(pts)[0], 20, ids, torch.zeros(2, dtype=torch.int64, device="cuda"))
    idx.free()
    idx = fclsh.build(pts, 64, 30, 1, t=3)     # T = 3 * 2047 = 6,141 tables: above the limit
    with pytest.raises(fclsh.FclshError) as e:
        idx.query_plain_noalloc(_dev(pts)[0], 30, ids, counts)
    assert e.value.status == fclsh.EINVAL
    idx.free()
