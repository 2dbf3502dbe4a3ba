"""The point-sharded index on one GPU: the shards of ShardedIndex (contiguous id ranges, same
seed, Algorithm 1's shape fixed from the whole set) are built one after another, each
answers the batch, and shard.merge combines the answers -- the same ids and counters as
the unsharded index and the oracle's linear scan.  The gather between processes is tested
with gloo ranks on CPU (tests/test_shard_gloo.py)."""
import numpy as np
import pytest

import oracle
from paper_1602_02620_gb300 import shard
from paper_1602_02620_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("cfg,n,nq,world,opts", [(2, 50_000, 300, 3, {}), (4, 40_000, 200, 2, {}),
                                                 (1, 10_000, 200, 4, {"approx_c": 1.5})])
def test_sharded_answers_equal_the_whole_index(cfg, n, nq, world, opts):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02620_gb300 import fclsh

    c = wl.CONFIGS[cfg]
    pts = wl.points(cfg, n)
    qs, _ = wl.queries(cfg, pts, nq)
    d, r, seed = c["d"], c["r"], c["seed"] + 1000
    pts_dev = torch.from_numpy(pts.view(np.int64)).cuda()
    q_dev = torch.from_numpy(qs.view(np.int64)).cuda()
    t, rep = shard.global_shape(n, d, r, seed, **opts)
    whole = fclsh.build(pts_dev, d, r, seed, t=t, replicate=rep if rep > 1 else 0)
    want = whole.query(q_dev, r)
    parts = []
    for k in range(world):
        sh = shard.ShardedIndex(pts_dev, n, d, r, seed, k, world, **opts)
        assert (sh.t, sh.rep) == (t, rep) and sh.index.T == whole.T
        parts.append(tuple(sh.local_query(q_dev, r)) + (sh.lo,))
        sh.free()
    offs, ids, coll, cand = shard.merge(parts)
    assert np.array_equal(offs, want.offs) and np.array_equal(ids, want.ids)
    assert np.array_equal(coll, want.collisions) and np.array_equal(cand, want.candidates)
    for i in range(0, nq, max(1, nq // 12)):
        assert np.array_equal(ids[int(offs[i]):int(offs[i + 1])], oracle.linear_scan(pts, qs[i], r)), i
    whole.free()
