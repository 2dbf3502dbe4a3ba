"""Replication pre-processing (Algorithm 1, cr < log n) on the GPU against the oracle.

Parameters, keys (every hash kernel that applies), bucket tables and query results
of a replicated index must equal the oracle's bit for bit; the Algorithm 1 rule for
an approximation factor c picks the replication factor or the parts it states.
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


def F():
    from paper_1602_02620_gb300 import fclsh

    return fclsh


def rand_points(rng, n, d):
    words = (d + 63) // 64
    a = rng.integers(0, 2**63, size=(n, words), dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=(n, words), dtype=np.uint64)
    if d % 64:
        a[:, -1] &= np.uint64((1 << (d % 64)) - 1)
    return a


def near(rng, pts, d, kmax, count):
    q = pts[rng.integers(0, pts.shape[0], size=count)].copy()
    for i in range(count):
        for pos in rng.choice(d, size=rng.integers(0, kmax + 1), replace=False):
            q[i, pos >> 6] ^= np.uint64(1) << np.uint64(pos & 63)
    return q


# (d, r, rep, n, hash tiles): specific (d*rep <= W) and general (d*rep > W) constructions,
# W from 8 to 2048 (the paper's replication settings r = 2..5 with rep = 4, 3, 2, 2 among them)
REP_CASES = [
    (4, 1, 2, 300, (0,)),            # W = 8, D = 8: specific
    (10, 1, 4, 1000, (0,)),          # W = 32, D = 40: general
    (32, 2, 4, 1500, (0, 1, 2)),     # W = 512, D = 128: specific, the tensor-core route applies
    (128, 2, 4, 700, (0, 1)),        # W = 512, D = 512: specific (r = 2 with rep = 4)
    (128, 3, 3, 600, (0, 1)),        # W = 1024, D = 384: specific (r = 3 with rep = 3)
    (128, 4, 2, 900, (0, 1)),        # W = 512, D = 256: specific (r = 4 with rep = 2)
    (128, 5, 2, 300, (0,)),          # W = 2048, D = 256: specific (r = 5 with rep = 2)
    (300, 2, 2, 1100, (0, 1)),       # W = 32, D = 600: general
    (1000, 1, 3, 400, (0,)),         # W = 16, D = 3000: general, 16 words
]


@pytest.mark.parametrize("d,r,rep,n,tiles", REP_CASES)
def test_replicated_params_and_keys_bit_exact(d, r, rep, n, tiles):
    rng = np.random.default_rng(d * 31 + rep)
    pts = rand_points(rng, n, d)
    pts[0] = 0
    seed = 4242 + d + r + rep
    p = oracle.derive_params(seed, d, r, rep=rep)
    sample = pts[: min(n, 300)]
    want = oracle.keys_fht(p, sample)
    for tile in tiles:
        try:
            idx = F().build(pts, d, r, seed, replicate=rep, hash_tile=tile)
        except F().FclshError as e:
            # the wide tile may not fit the kernel's shared memory: a stated error
            assert tile == 1 and "EINVAL" in str(e), e
            continue
        assert (idx.rep, idx.t, idx.rp, idx.W, idx.T) == (rep, 1, r * rep, p.W, p.T)
        perm, part_off, m, b = idx.params()
        assert np.array_equal(perm, p.perm) and np.array_equal(part_off, p.part_off)
        assert np.array_equal(m, p.m) and np.array_equal(b, p.b)
        assert np.array_equal(idx.hash(sample), want), tile
        for tau in sorted({0, p.T // 3, p.T - 1}):
            keys, ids = idx.export_table(tau)
            order = np.lexsort((ids, keys))
            ok, oi = oracle.table(p, pts, tau)
            assert np.array_equal(keys[order], ok) and np.array_equal(ids[order], oi)
        idx.free()


@pytest.mark.parametrize("d,r,rep,n", [(32, 2, 3, 3000), (128, 2, 4, 2500), (100, 3, 2, 2000), (64, 1, 5, 1500)])
@pytest.mark.parametrize("probe_rows", [0, 1])
def test_replicated_queries_match_oracle(d, r, rep, n, probe_rows):
    """Batched and plain queries at every radius <= r: the linear-scan answer, and the
    oracle's #Collisions / #Candidates for the tables probed."""
    rng = np.random.default_rng(n + rep)
    pts = rand_points(rng, n, d)
    pts[20:40] = pts[3]
    seed = 99 + d + rep
    idx = F().build(pts, d, r, seed, replicate=rep)
    tu = idx.tuning()
    tu["probe_rows"] = probe_rows
    idx.set_tuning(**tu)
    p = oracle.derive_params(seed, d, r, rep=rep)
    tables = oracle.build_tables(p, pts)
    qs = np.concatenate([near(rng, pts, d, r + 1, 40), rand_points(rng, 10, d)])
    for rho in range(r + 1):
        res = idx.query(qs, rho)
        plain = idx.query_plain(qs[:12], rho)
        rows = oracle.probe_rows(p, rho) if probe_rows else 0
        for i, q in enumerate(qs):
            ids, ncoll, ncand = oracle.query(p, pts, tables, q, rho, rows=rows)
            assert res.of(i).tolist() == ids.tolist() == oracle.linear_scan(pts, q, rho).tolist()
            assert (int(res.collisions[i]), int(res.candidates[i])) == (ncoll, ncand)
            if i < 12:
                assert plain.of(i).tolist() == ids.tolist()
    idx.free()


def test_replicated_mixed_radii_and_served():
    """Per-query radii and the served form on a replicated index."""
    rng = np.random.default_rng(5)
    d, r, rep, n = 64, 2, 4, 4000
    pts = rand_points(rng, n, d)
    idx = F().build(pts, d, r, 5, replicate=rep)
    qs = near(rng, pts, d, r, 64)
    radii = rng.integers(0, r + 1, size=64).astype(np.uint32)
    res = idx.query(qs, r, radii=radii)
    for i in range(64):
        assert res.of(i).tolist() == oracle.linear_scan(pts, qs[i], int(radii[i])).tolist()
    srv = F().Server(idx)
    tickets = [srv.submit(qs[i:i + 8], int(radii[i])) for i in range(0, 64, 8)]
    for j, tk in enumerate(tickets):
        out, _ = srv.wait(tk)
        for i in range(8):
            q = qs[8 * j + i]
            assert out.of(i).tolist() == oracle.linear_scan(pts, q, int(radii[8 * j])).tolist()
    srv.close()
    idx.free()


def test_algorithm1_rule_for_c():
    """Algorithm 1 with log = log2 n on n = 4096: c r < 12 replicates floor(12 / (c r))
    times, c r > 12 partitions into ceil(c r / 12) parts, c r = 12 does neither."""
    rng = np.random.default_rng(8)
    n, d = 4096, 128
    pts = rand_points(rng, n, d)
    for r, c, t, rep in ((2, 2.0, 1, 3), (3, 1.5, 1, 2), (1, 1.1, 1, 10), (10, 2.0, 2, 1), (6, 2.0, 1, 1),
                         (5, 1.25, 1, 1), (4, 1.2, 1, 2)):
        idx = F().build(pts, d, r, 1, approx_c=c)
        assert (idx.t, idx.rep, idx.rp) == (t, rep, r * rep // t), (r, c)
        idx.free()
    # explicit t or replicate overrides the rule; both together are refused
    idx = F().build(pts, d, 2, 1, approx_c=2.0, replicate=2)
    assert (idx.t, idx.rep) == (1, 2)
    idx.free()
    with pytest.raises(F().FclshError):
        F().build(pts, d, 4, 1, t=2, replicate=2)
    with pytest.raises(F().FclshError):
        F().build(pts, d, 3, 1, replicate=4)          # r * rep = 12 > 10
