"""The served form: continuous batching gives every request the answer it gets alone.

Requests of mixed size and radius (radius <= the build radius) are answered one
at a time by a one-slot server, then all at once by a four-slot server that
packs them into shared device batches.  Each request's ids and counters must be
identical in both runs, equal to the batched query path, and (on a sample)
equal to the oracle's linear scan.
"""
import numpy as np
import pytest

import oracle
from paper_1602_02620_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("probe_rows", [0, 1])
def test_served_answers_alone_equal_mixed(probe_rows):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02620_gb300 import fclsh

    pts = wl.points(5, 60_000)
    reqs = wl.request_stream(5, 40, rate_per_s=1000.0)
    qs, _ = wl.queries(5, pts, sum(min(s, 300) for _, s, _ in reqs))
    blocks, at = [], 0
    for _, size, radius in reqs:
        size = min(size, 300)
        blocks.append((qs[at:at + size], radius))
        at += size
    idx = fclsh.build(torch.from_numpy(pts.view(np.int64)).cuda(), 256, 16, 5005)
    idx.set_tuning(probe_rows=probe_rows)

    alone = fclsh.Server(idx, slots=1, max_batch_queries=1)
    res_alone = []
    for q, radius in blocks:
        t = alone.submit(q, radius)
        res_alone.append(alone.wait(t)[0])
    st1 = alone.stats()
    alone.close()
    assert st1["requests"] == len(blocks) and st1["batches"] == len(blocks)

    mix = fclsh.Server(idx, slots=4, max_batch_queries=2048)
    tickets = [mix.submit(q, radius) for q, radius in blocks]
    res_mix = [mix.wait(t)[0] for t in tickets]
    st2 = mix.stats()
    mix.close()
    assert st2["requests"] == len(blocks) and st2["batches"] < len(blocks)      # requests shared batches
    assert st2["p99_ms"] >= st2["p50_ms"] > 0

    for i, (q, radius) in enumerate(blocks):
        a, b = res_alone[i], res_mix[i]
        assert np.array_equal(a.offs, b.offs) and np.array_equal(a.ids, b.ids), i
        assert np.array_equal(a.collisions, b.collisions) and np.array_equal(a.candidates, b.candidates), i
        c = idx.query(q, radius)
        assert np.array_equal(c.ids, b.ids) and np.array_equal(c.offs, b.offs), i
        if i % 8 == 0:
            for j in range(0, q.shape[0], max(1, q.shape[0] // 3)):
                assert np.array_equal(b.of(j), oracle.linear_scan(pts, q[j], radius)), (i, j)
    idx.free()


def test_server_argument_errors():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02620_gb300 import fclsh

    pts = wl.points(1, 2000)
    idx = fclsh.build(pts, 64, 3, 1001)
    srv = fclsh.Server(idx, slots=2)
    with pytest.raises(fclsh.FclshError) as e:
        srv.submit(pts[:4], 4)
    assert e.value.status == fclsh.ERADIUS
    t = srv.submit(pts[:0], 3)                       # an empty request completes at once
    r, _ = srv.wait(t, timeout_ms=1000)
    assert len(r) == 0
    with pytest.raises(fclsh.FclshError):
        srv.wait(987654321)                           # unknown ticket
    srv.close()
    idx.free()
