"""The allocation-free one-query entry point (fclsh_query_plain_noalloc).

It serves callers that cannot allocate device memory while they query; all of
its scratch is one fixed device array inside the library.  Its answers must be
exactly those of the ordinary plain path (fclsh_query_plain) for the same query,
call after call, since every call reuses that array.  This file is collected
last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

from paper_1602_02620_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


@pytest.mark.parametrize("cfg,n,nq", [(2, 60_000, 6), (3, 40_000, 6)])
def test_noalloc_matches_plain_path_on_consecutive_calls(cfg, n, nq):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02620_gb300 import fclsh

    pts = wl.points(cfg, n)
    qs, _ = wl.queries(cfg, pts, nq)
    r = wl.CONFIGS[cfg]["r"]
    d = wl.CONFIGS[cfg]["d"]
    idx = fclsh.build(_dev(pts), d, r, 4242 + cfg)
    want = idx.query_plain(qs, r)
    cap = 4096
    ids = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    counts = torch.zeros(3, dtype=torch.int64, device="cuda")
    q_dev = _dev(qs)

    def check(i):
        ids.fill_(-1)
        idx.query_plain_noalloc(q_dev[i], r, ids, counts)
        torch.cuda.synchronize()
        c = counts.cpu().numpy()
        exp = want.of(i)
        assert int(c[0]) == exp.shape[0]
        assert int(c[1]) == int(want.collisions[i]) and int(c[2]) == int(want.candidates[i])
        got = ids[: min(int(c[0]), cap)].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, exp[:cap])

    check(0)                                   # first call on this device sets up the scratch address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for i in range(nq):                        # consecutive calls share the same scratch
        check(i)
    check(0)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    idx.free()


def test_noalloc_rejects_oversized_index():
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
    idx.free()
    idx = fclsh.build(pts, 64, 30, 1, t=3)     # T = 3 * 2047 = 6,141 tables: above the limit
    with pytest.raises(fclsh.FclshError) as e:
        idx.query_plain_noalloc(_dev(pts)[0], 30, ids, counts)
    assert e.value.status == fclsh.EINVAL
    idx.free()
