"""GPU path vs the CPU oracle, element by element, through the C ABI.

Keys, bucket contents and sorted result sets must be bit-exact (all integer
arithmetic).  Sizes span several kernel tiles with ragged tails; the edge cases
cover n = 1, empty batches, identical points (one huge bucket), r = 0 and
radii below the build radius.
"""
import numpy as np
import pytest

import oracle
from paper_1602_02620_gb300 import workloads as wl
from tests.conftest import bits_to_int, bits_to_words, read_golden

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


def dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


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


# (d, r, t, n): W from 2 to 2048; general (d' > W) and specific (d' <= W) constructions
HASH_CASES = [
    (64, 0, None, 777),      # W = 2, general
    (64, 1, None, 1000),     # W = 4
    (64, 3, None, 3001),     # W = 16, general (the small plain workload's shape)
    (40, 4, None, 1500),     # W = 32, specific, d not a multiple of 64
    (100, 5, None, 2049),    # W = 64, general, ragged tile
    (128, 6, None, 1025),    # W = 128, specific
    (200, 7, None, 999),     # W = 256, specific
    (128, 8, None, 1003),    # W = 512, specific (plain n=1M d=128 r=8 shape)
    (256, 16, None, 517),    # t = 2, W = 512 per part (clustered shape)
    (1024, 9, None, 300),    # W = 1024, specific, 16 words
    (1024, 20, None, 211),   # t = 2, W = 2048 (sparse shape)
    (300, 7, 3, 500),        # t = 3, general per part
    (2000, 10, 2, 130),      # t = 2, W = 64 per part?  no: r' = 5 -> W = 64, general d' = 1000
]


@pytest.mark.parametrize("d,r,t,n", HASH_CASES)
def test_params_and_keys_bit_exact(d, r, t, n):
    rng = np.random.default_rng(d * 1000 + r)
    pts = rand_points(rng, n, d)
    pts[0] = 0
    seed = 12345 + d + r
    idx = F().build(pts, d, r, seed, t=t)
    p = oracle.derive_params(seed, d, r, t=t)
    perm, part_off, m, b = idx.params()
    assert np.array_equal(perm, p.perm) and np.array_equal(part_off, p.part_off)
    assert np.array_equal(m, p.m) and np.array_equal(b, p.b)
    assert idx.T == p.T and idx.W == p.W
    sample = pts[: min(n, 400)]
    want = oracle.keys_direct(p, sample)
    got = idx.hash(sample)                                   # host in, host out
    assert np.array_equal(got, want)
    out = torch.zeros((idx.T, sample.shape[0]), dtype=torch.int64, device="cuda")
    idx.hash(dev(sample), out=out)                           # device in, device out
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint64), want)
    idx.free()


def test_example1_and_example2_on_gpu():
    """The worked examples (Sec. 2.3 and 3.1) through the GPU kernels, b_i = 2^i."""
    g1 = read_golden("example1_covering.txt")
    m = [int(s, 2) for s in g1["m"]]
    pts = np.stack([bits_to_words(g1["x"][0]), bits_to_words(g1["q"][0]), bits_to_words("1111")])
    idx = F().build(pts, 4, 2, 0, perm=[0, 1, 2, 3], part_off=[0, 4], m=m, b=[1, 2, 4, 8])
    keys = idx.hash(pts)
    for v in range(1, 8):
        assert int(keys[v - 1, 2]) == bits_to_int(g1["g%d" % v][0])
    coll = [v for v in range(1, 8) if keys[v - 1, 0] == keys[v - 1, 1]]
    assert coll == [4] and int(keys[3, 0]) == bits_to_int(g1["value"][0])
    idx.free()

    g2 = read_golden("example2_c78.txt")
    pts = np.stack([bits_to_words(g2[k][0]) for k in ("x", "y", "q")] + [bits_to_words("1" * 8)])
    idx = F().build(pts, 8, 2, 0, perm=list(range(8)), part_off=[0, 8], m=list(range(8)), b=[1 << i for i in range(8)])
    keys = idx.hash(pts)
    for v in range(1, 8):
        assert int(keys[v - 1, 3]) == bits_to_int(g2["C%d" % v][0])
    assert [v for v in range(1, 8) if keys[v - 1, 0] == keys[v - 1, 2]] == [3]
    assert not any(keys[v, 1] == keys[v, 2] for v in range(7))
    # radius 2 around q reports x (distance 2) and not y (distance 3), found through the tables
    res = idx.query(pts[2:3], 2)
    assert res.of(0).tolist() == [0, 2]
    idx.free()


@pytest.mark.parametrize("d,r,n", [(64, 3, 3000), (128, 6, 2500), (256, 12, 1800)])
def test_bucket_tables_bit_exact(d, r, n):
    rng = np.random.default_rng(n)
    pts = rand_points(rng, n, d)
    pts[10:60] = pts[5]                                      # one bucket of 51 equal points in every table
    seed = 77 + r
    idx = F().build(pts, d, r, seed)
    p = oracle.derive_params(seed, d, r)
    for tau in sorted({0, 1, p.T // 2, p.T - 1}):
        keys, ids = idx.export_table(tau)
        sl = keys & np.uint64((1 << idx.info["slot_bits"]) - 1)
        assert np.all(np.diff(sl.astype(np.int64)) >= 0)        # entries grouped by slot, slots ascending
        order = np.lexsort((ids, keys))
        ok, oi = oracle.table(p, pts, tau)
        assert np.array_equal(keys[order], ok) and np.array_equal(ids[order], oi)
        for key in {int(ok[0]), int(ok[len(ok) // 2]), int(keys[0])}:
            want = oi[ok == key]
            assert np.array_equal(idx.bucket(tau, key), want)
    assert idx.bucket(0, 12345).size in (0, 1) or True
    idx.free()


QUERY_CASES = [
    # d, r, t, n, nq, kmax
    (64, 3, None, 4000, 150, 4),
    (128, 8, None, 3000, 120, 9),
    (256, 16, None, 2500, 80, 18),
    (100, 5, None, 2000, 100, 6),
    (1024, 20, None, 600, 40, 22),
    (96, 12, 2, 3000, 100, 14),
]


def _oracle_answers(p, pts, qs, radius, with_counters):
    tables = oracle.build_tables(p, pts) if with_counters else None
    out = []
    for q in qs:
        if with_counters:
            out.append(oracle.query(p, pts, tables, q, radius))
        else:
            out.append((oracle.linear_scan(pts, q, radius), None, None))
    return out


@pytest.mark.parametrize("d,r,t,n,nq,kmax", QUERY_CASES)
def test_batched_plain_and_bruteforce_queries(d, r, t, n, nq, kmax):
    rng = np.random.default_rng(d + r + n)
    pts = rand_points(rng, n, d)
    pts[100:140] = pts[7]                                    # duplicates
    qs = np.concatenate([near(rng, pts, d, kmax, nq - 10), rand_points(rng, 10, d)])
    seed = 999 + d
    p = oracle.derive_params(seed, d, r, t=t)
    idx = F().build(dev(pts), d, r, seed, t=t)
    small = p.T * n <= 3_000_000
    ans = _oracle_answers(p, pts, qs, r, small)
    res = idx.query(dev(qs), r)
    plain = idx.query_plain(qs, r)
    brute = idx.bruteforce(dev(qs), r)
    for i in range(qs.shape[0]):
        want = ans[i][0]
        assert np.array_equal(res.of(i), want), i
        assert np.array_equal(plain.of(i), want), i
        assert np.array_equal(brute.of(i), oracle.linear_scan(pts, qs[i], r)), i
        if small:
            assert int(res.collisions[i]) == ans[i][1] and int(res.candidates[i]) == ans[i][2], i
            assert int(plain.collisions[i]) == ans[i][1] and int(plain.candidates[i]) == ans[i][2], i
    # smaller radii and per-query radii over the same index
    radii = rng.integers(0, r + 1, size=qs.shape[0]).astype(np.uint32)
    res2 = idx.query(dev(qs), r, radii=torch.from_numpy(radii.view(np.int32)).cuda())
    for i in range(qs.shape[0]):
        assert np.array_equal(res2.of(i), oracle.linear_scan(pts, qs[i], int(radii[i])))
    idx.free()


def test_edge_cases():
    fc = F()
    rng = np.random.default_rng(5)
    # n = 1
    one = rand_points(rng, 1, 64)
    idx = fc.build(one, 64, 3, 1)
    assert idx.query(one, 3).of(0).tolist() == [0]
    assert idx.query(np.zeros((1, 1), np.uint64) ^ ~one, 3).of(0).tolist() == []
    # empty batch
    r0 = idx.query(np.zeros((0, 1), np.uint64), 3)
    assert len(r0) == 0 and r0.offs.tolist() == [0]
    with pytest.raises(fc.FclshError) as e:
        idx.query(one, 4)
    assert e.value.status == fc.ERADIUS
    idx.free()
    # all points identical: one bucket of n entries in every table (bitmap dedup path)
    same = np.repeat(rand_points(rng, 1, 128), 20000, axis=0)
    idx = fc.build(dev(same), 128, 8, 3)
    res = idx.query(same[:3], 8)
    for i in range(3):
        assert np.array_equal(res.of(i), np.arange(20000, dtype=np.uint32))
        assert int(res.candidates[i]) == 20000 and int(res.collisions[i]) == 20000 * idx.T
    idx.free()
    # r = 0: exact-match queries
    pts = rand_points(rng, 5000, 64)
    pts[77] = pts[3]
    idx = fc.build(pts, 64, 0, 9)
    res = idx.query(pts[[3, 4]], 0)
    assert res.of(0).tolist() == [3, 77] and res.of(1).tolist() == [4]
    idx.free()


def test_forced_bitmap_dedup_and_graph_replay():
    """Shapes change speed only: tiny hash set (bitmap path), other blocks, graphs on/off."""
    fc = F()
    pts = wl.points(3, 30_000)
    qs, _ = wl.queries(3, pts, 200)
    idx = fc.build(dev(pts), 256, 16, 1003)
    base = idx.query(dev(qs), 16)
    for i in range(0, 200, 7):
        assert np.array_equal(base.of(i), oracle.linear_scan(pts, qs[i], 16))
    for tune in ({"hash_set_log2": 10, "inline_probe": 1}, {"query_block": 128, "use_graph": 0},
                 {"query_block": 512, "query_ctas_per_sm": 1, "hash_set_log2": 13, "inline_probe": 32}):
        idx.set_tuning(**tune)
        r2 = idx.query(dev(qs), 16)
        assert np.array_equal(r2.offs, base.offs) and np.array_equal(r2.ids, base.ids)
        assert np.array_equal(r2.collisions, base.collisions) and np.array_equal(r2.candidates, base.candidates)
    ctx = idx.context()
    q = dev(qs)
    for _ in range(3):                                       # replayed graph, same answers
        ctx.query_async(q, 16)
        r3 = ctx.fetch()
        assert np.array_equal(r3.ids, base.ids)
    ctx.close()
    idx.free()


@pytest.mark.parametrize("d,r,t,n", [(128, 8, None, 2500), (96, 12, 2, 2000), (256, 16, None, 1500)])
def test_row_restricted_probe_matches_oracle(d, r, t, n):
    """probe_rows = 1: every radius reports the linear-scan ids, and the counters equal the
    oracle's query over the rows v <= 2^(floor(radius/t)+1) - 1 of every part (batched,
    plain, per-query radii and the allocation-free entry point)."""
    rng = np.random.default_rng(d * 3 + r)
    pts = rand_points(rng, n, d)
    pts[50:70] = pts[3]
    qs = np.concatenate([near(rng, pts, d, r, 40), rand_points(rng, 5, d)])
    seed = 4242 + d
    p = oracle.derive_params(seed, d, r, t=t)
    tables = oracle.build_tables(p, pts)
    idx = F().build(dev(pts), d, r, seed, t=t)
    idx.set_tuning(probe_rows=1)
    for radius in sorted({0, 1, r // 3, r // 2, r}):
        rows = oracle.probe_rows(p, radius)
        res = idx.query(dev(qs), radius)
        plain = idx.query_plain(qs[:8], radius)
        for i in range(qs.shape[0]):
            ids, ncoll, ncand = oracle.query(p, pts, tables, qs[i], radius, rows=rows)
            assert np.array_equal(res.of(i), ids) and np.array_equal(ids, oracle.linear_scan(pts, qs[i], radius))
            assert (int(res.collisions[i]), int(res.candidates[i])) == (ncoll, ncand), (radius, i)
            if i < 8:
                assert np.array_equal(plain.of(i), ids)
                assert (int(plain.collisions[i]), int(plain.candidates[i])) == (ncoll, ncand)
        ids_d = torch.zeros(n, dtype=torch.int32, device="cuda")
        cnt_d = torch.zeros(3, dtype=torch.int64, device="cuda")
        idx.query_plain_noalloc(dev(qs[0]), radius, ids_d, cnt_d)
        torch.cuda.synchronize()
        c0 = cnt_d.cpu().numpy()
        want0 = oracle.query(p, pts, tables, qs[0], radius, rows=rows)
        assert np.array_equal(ids_d[: int(c0[0])].cpu().numpy().view(np.uint32), want0[0])
        assert (int(c0[1]), int(c0[2])) == (want0[1], want0[2])
    radii = rng.integers(0, r + 1, size=qs.shape[0]).astype(np.uint32)
    res2 = idx.query(dev(qs), r, radii=torch.from_numpy(radii.view(np.int32)).cuda())
    for i in range(qs.shape[0]):
        rad = int(radii[i])
        ids, ncoll, ncand = oracle.query(p, pts, tables, qs[i], rad, rows=oracle.probe_rows(p, rad))
        assert np.array_equal(res2.of(i), ids)
        assert (int(res2.collisions[i]), int(res2.candidates[i])) == (ncoll, ncand)
    idx.free()


@pytest.mark.parametrize("tile", [1, 2, 4])
@pytest.mark.parametrize("d,r,t", [(100, 5, None), (128, 6, None), (200, 7, None), (128, 8, None),
                                   (1024, 9, None), (256, 16, None), (2000, 10, 2), (96, 12, 2), (128, 9, 3)])
def test_hash_tiles_are_bit_exact(d, r, t, tile):
    """hash_tile = 1 (twice the points per WHT block), hash_tile = 2 (the O(dL) route as an
    exact tensor-core contraction) and hash_tile = 4 (the O(dL) route on CUDA cores, the basic
    construction without the transform) give the oracle's keys and the same directory."""
    fc = F()
    rng = np.random.default_rng(d + 5 * r)
    n = 1333
    pts = rand_points(rng, n, d)
    seed = 77 + d
    p = oracle.derive_params(seed, d, r, t=t)
    max_dk = int(np.max(np.diff(p.part_off)))
    if tile == 2 and (p.W < 64 or max_dk > 128):
        with pytest.raises(fc.FclshError):
            fc.build(dev(pts), d, r, seed, t=t, hash_tile=2)
        return
    a = fc.build(dev(pts), d, r, seed, t=t)
    b = fc.build(dev(pts), d, r, seed, t=t, hash_tile=tile)
    assert b.tuning()["hash_tile"] == tile
    assert np.array_equal(b.hash(pts[:300]), oracle.keys_direct(p, pts[:300]))
    for tau in (0, p.T // 2, p.T - 1):                          # the same tables (order inside a slot is free)
        ka, ia = a.export_table(tau)
        kb, ib = b.export_table(tau)
        oa, ob = np.lexsort((ia, ka)), np.lexsort((ib, kb))
        assert np.array_equal(ka[oa], kb[ob]) and np.array_equal(ia[oa], ib[ob])
        assert np.array_equal(ka & np.uint64((1 << a.info["slot_bits"]) - 1),
                              np.sort(ka & np.uint64((1 << a.info["slot_bits"]) - 1)))   # grouped by slot
    a.free()
    b.free()


def test_autotune_choices_keep_results(tmp_path):
    """The autotuner picks query shapes and a WHT tile, caches them, keeps probe_rows, and
    the chosen shapes give the same answers as the defaults."""
    fc = F()
    pts = wl.points(2, 20_000)
    qs, _ = wl.queries(2, pts, 300)
    idx = fc.build(dev(pts), 128, 8, 2002)
    base = idx.query(dev(qs), 8)
    idx.set_tuning(probe_rows=1)
    cache = str(tmp_path / "tune.json")
    chosen = idx.autotune(dev(qs), 8, cache)
    assert chosen["probe_rows"] == 1 and chosen["hash_tile"] in (0, 1) and chosen["use_graph"] == 1
    assert idx.tuning() == chosen
    again = idx.autotune(dev(qs), 8, cache)                      # served from the cache
    assert again == chosen
    res = idx.query(dev(qs), 8)
    assert np.array_equal(res.offs, base.offs) and np.array_equal(res.ids, base.ids)
    assert np.array_equal(res.collisions, base.collisions)       # radius 8 = r: every row is probed
    idx.free()


@pytest.mark.parametrize("hlog,heavy", [(10, 0), (13, 0), (10, 1), (13, 1024), (11, 2)])
def test_dedup_modes_match_oracle(hlog, heavy):
    """Queries in every dedup mode -- shared-memory set, returning bitmap, mark-and-sweep
    bitmap (bucket entries beyond the bitmap's word count), and more than 4,096 hits --
    report the oracle's ids and counters.  The very heavy queries are answered by the batch
    kernel's own sweep (heavy = 0) or by the heavy-query kernel, in one shared-memory window
    of ids (1) or in nine windows of 1,024 ids with a ragged last one (1024 = 64 W); with heavy = 2
    the heavy-query kernel also answers the bitmap-mode queries."""
    rng = np.random.default_rng(hlog)
    d, r, n = 64, 3, 9000
    pts = rand_points(rng, n, d)
    pts[1000:6000] = pts[17]                                  # 5,001 equal points: > 4,096 hits
    pts[6000:6600] = pts[23]                                  # 601 equal points
    for i in range(6600, 6900):                               # 300 points near point 29
        pts[i] = pts[29]
        pts[i, 0] ^= np.uint64(1) << np.uint64(int(rng.integers(0, 64)))
    seed = 606
    p = oracle.derive_params(seed, d, r)
    tables = oracle.build_tables(p, pts)
    qs = np.concatenate([pts[[17, 23, 29, 5, 7000]], near(rng, pts, d, r, 40), rand_points(rng, 5, d)])
    qs[5:15] = pts[17]
    idx = F().build(dev(pts), d, r, seed)
    assert idx.tuning()["heavy_kernel"] == 1                  # on by default
    idx.set_tuning(hash_set_log2=hlog, heavy_kernel=heavy)
    res = idx.query(dev(qs), r)
    for i in range(qs.shape[0]):
        ids, ncoll, ncand = oracle.query(p, pts, tables, qs[i], r)
        assert np.array_equal(res.of(i), ids), i
        assert (int(res.collisions[i]), int(res.candidates[i])) == (ncoll, ncand), i
    assert res.of(0).shape[0] > 4096
    again = idx.query(dev(qs), r)                              # the bitmaps were left clear
    assert np.array_equal(again.ids, res.ids) and np.array_equal(again.offs, res.offs)
    idx.free()


@pytest.mark.parametrize("slot_bits", [13, 14, 16, 17, 18, 19, 21, 22, 23])
@pytest.mark.parametrize("skewed", [False, True])
def test_wide_partition_directory_matches_oracle(slot_bits, skewed):
    """Directories with 2^13..2^23 slots per table (partition by the slot's top 1..11 bits;
    below 2^18 slots the entries keep 14 + s id bits) hold the oracle's buckets, through the
    bins and, with many equal keys, through the exact histogram fallback; queries over them
    match the oracle."""
    rng = np.random.default_rng(slot_bits + 100 * skewed)
    d, r, n = 128, 6, 5000
    pts = rand_points(rng, n, d)
    if skewed:
        pts[100:1600] = pts[3]                                   # 1,501 equal points: bins overflow
    seed = 31 + slot_bits
    p = oracle.derive_params(seed, d, r)
    idx = F().build(dev(pts), d, r, seed, slot_bits=slot_bits)
    assert idx.info["slot_bits"] == slot_bits
    for tau in sorted({0, 1, p.T // 2, p.T - 1}):
        keys, ids = idx.export_table(tau)
        sl = keys & np.uint64((1 << slot_bits) - 1)
        assert np.all(np.diff(sl.astype(np.int64)) >= 0)
        order = np.lexsort((ids, keys))
        ok, oi = oracle.table(p, pts, tau)
        assert np.array_equal(keys[order], ok) and np.array_equal(ids[order], oi)
        for key in {int(ok[0]), int(ok[len(ok) // 2]), int(keys[3])}:
            assert np.array_equal(idx.bucket(tau, key), oi[ok == key])
    qs = np.concatenate([near(rng, pts, d, r, 30), pts[[3]]])
    tables = oracle.build_tables(p, pts)
    res = idx.query(dev(qs), r)
    for i in range(qs.shape[0]):
        want, ncoll, ncand = oracle.query(p, pts, tables, qs[i], r)
        assert np.array_equal(res.of(i), want)
        assert (int(res.collisions[i]), int(res.candidates[i])) == (ncoll, ncand)
    idx.free()


@pytest.mark.parametrize("zeros", [1300, 2000, 3000])
def test_empty_sum_bucket_in_bin_zero(zeros):
    """All-zero points have key 0 (the empty sum) in every table, so they all land in slot 0,
    partition bin 0 (2^15 slots: eight bins of ~2,500 entries, capacity 3,276, and bin 0 1,252
    more): with 1,300 of 20,000 it holds ~3,640 entries, which fit only in the larger bin 0 and stay
    below 7/8 of it (every table histogram-free in those bins); with 2,000, ~4,250 fit the trial
    table but pass 7/8, so the other tables get a bin 0 sized from the trial's fill; with 3,000,
    ~5,125 overflow the trial (the exact fallback).  Every directory holds the oracle's buckets, and
    queries over it match the oracle."""
    rng = np.random.default_rng(zeros)
    d, r, n = 128, 6, 20_000
    pts = rand_points(rng, n, d)
    pts[rng.choice(n, size=zeros, replace=False)] = 0
    seed = 321
    p = oracle.derive_params(seed, d, r)
    idx = F().build(dev(pts), d, r, seed, slot_bits=15)
    for tau in sorted({0, 2, p.T - 1}):
        keys, ids = idx.export_table(tau)
        order = np.lexsort((ids, keys))
        ok, oi = oracle.table(p, pts, tau)
        assert np.array_equal(keys[order], ok) and np.array_equal(ids[order], oi)
        assert np.array_equal(idx.bucket(tau, 0), oi[ok == 0]) and (ok == 0).sum() >= zeros
    qs = np.concatenate([near(rng, pts, d, r, 20), np.zeros((2, pts.shape[1]), np.uint64)])
    tables = oracle.build_tables(p, pts)
    res = idx.query(dev(qs), r)
    for i in range(qs.shape[0]):
        want, ncoll, ncand = oracle.query(p, pts, tables, qs[i], r)
        assert np.array_equal(res.of(i), want)
        assert (int(res.collisions[i]), int(res.candidates[i])) == (ncoll, ncand)
    idx.free()


@pytest.mark.parametrize("skewed", [False, True])
def test_long_segments_match_oracle(skewed):
    """Segments longer than one block's 4,608 entries (2^13 slots in two segments of ~15,000
    entries; with skew, 6,000 equal points on one slot of every table, as the empty sum of
    sparse points does): the directory that the long-segment kernel writes holds the oracle's
    buckets, every slot in order, and queries over it match the oracle."""
    rng = np.random.default_rng(4608 + skewed)
    d, r, n = 64, 3, 30_000
    pts = rand_points(rng, n, d)
    if skewed:
        pts[1000:7000] = pts[11]
    seed = 4242
    p = oracle.derive_params(seed, d, r)
    idx = F().build(dev(pts), d, r, seed, slot_bits=13)
    for tau in sorted({0, 3, p.T - 1}):
        keys, ids = idx.export_table(tau)
        sl = keys & np.uint64((1 << 13) - 1)
        assert np.all(np.diff(sl.astype(np.int64)) >= 0)
        order = np.lexsort((ids, keys))
        ok, oi = oracle.table(p, pts, tau)
        assert np.array_equal(keys[order], ok) and np.array_equal(ids[order], oi)
        for key in {int(ok[0]), int(ok[len(ok) // 2]), int(keys[1011])}:
            assert np.array_equal(idx.bucket(tau, key), oi[ok == key])
    qs = np.concatenate([near(rng, pts, d, r, 20), pts[[11, 12]]])
    tables = oracle.build_tables(p, pts)
    res = idx.query(dev(qs), r)
    for i in range(qs.shape[0]):
        want, ncoll, ncand = oracle.query(p, pts, tables, qs[i], r)
        assert np.array_equal(res.of(i), want)
        assert (int(res.collisions[i]), int(res.candidates[i])) == (ncoll, ncand)
    idx.free()


@pytest.mark.parametrize("dup,nq", [(2000, 2200), (20_000, 260)])
def test_result_overflow_reruns_only_the_queries_past_the_buffer(dup, nq):
    """A batch whose hits pass a fresh context's result buffer (2^22 ids): every query reserved
    its run all the same, the buffer grows to the batch's total keeping the runs that fitted,
    and only the queries whose run passed the old end run again.  Queries near a point
    repeated `dup` times have about `dup` hits each (the shared-memory sort below 4,096 hits,
    the bitmap read-out above).  Every answer equals the linear scan, and the same batch on
    the grown context (eager, then replayed as a graph) gives the same ids and counters."""
    rng = np.random.default_rng(dup)
    d, r = 64, 3
    n = dup + 3000
    pts = rand_points(rng, n, d)
    pts[:dup] = pts[0]
    qs = near(rng, pts[:1], d, r, nq)
    idx = F().build(pts, d, r, 31)
    ctx = idx.context()
    ctx.query_async(dev(qs), r)
    first = ctx.fetch()
    assert int(first.offs[-1]) > (1 << 22)                     # the batch did pass the buffer
    for i in range(nq):
        assert np.array_equal(first.of(i), oracle.linear_scan(pts, qs[i], r)), i
    q_dev = dev(qs)
    for _ in range(3):                                         # no overflow now; the third is a graph replay
        ctx.query_async(q_dev, r)
        again = ctx.fetch()
        assert np.array_equal(again.offs, first.offs) and np.array_equal(again.ids, first.ids)
        assert np.array_equal(again.collisions, first.collisions)
        assert np.array_equal(again.candidates, first.candidates)
    ctx.close()
    plain = idx.query_plain(qs[:3], r)
    for i in range(3):
        assert np.array_equal(plain.of(i), first.of(i))
        assert plain.collisions[i] == first.collisions[i] and plain.candidates[i] == first.candidates[i]
    idx.free()


def sparse_points(rng, n, d, density):
    """Bernoulli(density) bits packed LSB-first, with a tenth of the points near-duplicates."""
    bits = rng.random((n, d)) < density
    for i in range(n // 10):
        j = rng.integers(0, n)
        bits[i] = bits[j]
        bits[i, rng.choice(d, size=rng.integers(1, 6), replace=False)] ^= True
    words = (d + 63) // 64
    padded = np.zeros((n, words * 64), np.uint8)
    padded[:, :d] = bits
    return np.packbits(padded, axis=1, bitorder="little").view(np.uint64).reshape(n, words)


# (d, r, n, density): one coordinate per signature block (d < 128), 8, 24 (blocks across word
# boundaries, d not a multiple of 128) and 32 coordinates per block
@pytest.mark.parametrize("d,r,n,density", [(40, 4, 2000, 0.08), (1024, 12, 2500, 0.02), (3000, 12, 1500, 0.01),
                                           (4000, 7, 800, 0.02)])
def test_signature_filter_keeps_ids_and_counters(d, r, n, density):
    """S3's signature pre-filter, on and off, in the batched and plain paths: every query's ids,
    #Collisions and #Candidates equal the oracle's Strategy 2 query at the build radius and at
    half of it (the bound never rejects a point within the radius)."""
    rng = np.random.default_rng(d + n)
    pts = sparse_points(rng, n, d, density)
    qs = np.concatenate([near(rng, pts, d, r, 40), sparse_points(rng, 20, d, density)])
    seed = 900 + d
    idx = F().build(pts, d, r, seed)
    assert idx.tuning()["verify_filter"] == 0                  # off by default
    p = oracle.derive_params(seed, d, r)
    tables = oracle.build_tables(p, pts)
    for radius in (r, r // 2):
        want = [oracle.query(p, pts, tables, q, radius) for q in qs]
        assert sum(len(w[0]) for w in want) > 0
        for vf, hk in ((1, 1), (0, 1), (1, 0), (1, 2)):
            idx.set_tuning(verify_filter=vf, heavy_kernel=hk)
            for res in (idx.query(dev(qs), radius), idx.query_plain(qs, radius)):
                for i, (ids, ncoll, ncand) in enumerate(want):
                    assert np.array_equal(res.of(i), ids), (vf, hk, radius, i)
                    assert int(res.collisions[i]) == ncoll and int(res.candidates[i]) == ncand, (vf, hk, radius, i)
    idx.free()
