"""Parity at the stated workload sizes, in the launch configuration the benchmark times.

For each workload the index is built from device-resident points of the stated size with
the benchmark's kernel shapes (the autotuner's cache, as bench.py uses it).  The oracle
then checks what it can compute at that size:

* the random choices of Algorithms 1 and 2;
* the build's own keys, read back from the directory, for a sample of 10,000 points (all
  points of the small workload) in every table, against the keys of Eq. 1 on g_v AND x;
* complete tables (16, spread over the parts and rows) against the oracle's tables;
* 200 queries against the oracle's Strategy 2 query (Sec. 2.2, S1-S3 of Sec. 4.1), ids and
  #Collisions / #Candidates: with every table where the oracle can hold them all (the
  small and the plain workload), else with the code-row restricted probe at a small
  radius, whose tables the oracle builds in full;
* 200 queries at the full radius against the linear scan (Definition 2), every query
  against the GPU linear scan, and every reported id re-verified on the host.

The small workload (10,000 points, 15 tables, 200 queries) is checked completely: every
key of every point, every table, and all 200 queries one per call through the plain path.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_1602_02620_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

torch = pytest.importorskip("torch")

_POP = np.array([bin(i).count("1") for i in range(256)], dtype=np.uint8)
# oracle calls run in threads (ctypes releases the GIL while the C code runs)
_POOL = ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2))

KEY_SAMPLE = 10_000
FULL_TABLES = 16
QUERY_SAMPLE = 200
# workloads whose every table the oracle builds for the query check; the others use the
# row-restricted probe at this radius (few tables, each complete)
ALL_TABLES = {1, 2}
ROW_RADIUS = {3: 4, 4: 4, 5: 4, 8: 1}


def _popcount_rows(a: np.ndarray) -> np.ndarray:
    return _POP[a.view(np.uint8)].reshape(a.shape[0], -1).sum(axis=1)


def _tables(p, pts, taus):
    return dict(zip(taus, _POOL.map(lambda tau: oracle.table(p, pts, tau), taus)))


@pytest.fixture(scope="module", params=[1, 2, 3, 4, 5, 8])
def full(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02620_gb300 import fclsh

    cfg = request.param
    c = wl.CONFIGS[cfg]
    pts = wl.points(cfg)
    nq = c["nq"] if c["nq"] else 20_000
    qs, _ = wl.queries(cfg, pts, nq)
    seed = c["seed"] + 1000
    bopts = wl.build_options(cfg)                                 # e.g. replication
    p = oracle.derive_params(seed, c["d"], c["r"], rep=bopts.get("replicate", 1))
    pts_dev = torch.from_numpy(pts.view(np.int64)).cuda()
    q_dev = torch.from_numpy(qs.view(np.int64)).cuda()
    cache = os.path.join(ROOT, "paper_1602_02620_gb300", "_build", "autotune.json")
    idx0 = fclsh.build(pts_dev, c["d"], c["r"], seed, **bopts)
    tuned = idx0.autotune(q_dev[: min(nq, 8192)], c["r"], cache)
    idx0.free()
    idx = fclsh.build(pts_dev, c["d"], c["r"], seed, hash_tile=tuned["hash_tile"], **bopts)
    idx.set_tuning(**tuned)
    rng = np.random.default_rng(cfg)
    yield dict(cfg=cfg, c=c, pts=pts, qs=qs, nq=nq, p=p, idx=idx, q_dev=q_dev, rng=rng, fclsh=fclsh)
    idx.free()
    del pts_dev, q_dev
    torch.cuda.empty_cache()


def test_parameters(full):
    idx, p = full["idx"], full["p"]
    assert idx.n == full["c"]["n"] and idx.T == p.T and idx.W == p.W
    perm, part_off, m, b = idx.params()
    assert np.array_equal(perm, p.perm) and np.array_equal(part_off, p.part_off)
    assert np.array_equal(m, p.m) and np.array_equal(b, p.b)


def test_build_keys_of_sampled_points_in_every_table(full):
    """The keys the build stored (read back from the tables) against Eq. 1 on g_v AND x."""
    idx, p, pts, n = full["idx"], full["p"], full["pts"], full["c"]["n"]
    sample = np.arange(n) if n <= KEY_SAMPLE else np.sort(full["rng"].choice(n, size=KEY_SAMPLE, replace=False))
    got = idx.export_keys(sample.astype(np.uint32))
    chunks = np.array_split(sample, max(1, len(sample) // 256))
    want = np.concatenate(list(_POOL.map(lambda ch: oracle.keys_direct(p, pts[ch]), chunks)), axis=1)
    assert got.shape == want.shape == (p.T, len(sample))
    bad = np.argwhere(got != want)
    assert bad.size == 0, ("tables, points", bad[:5].tolist())


def test_complete_tables(full):
    """Whole tables: every (key, id) entry of the build against the oracle's table."""
    idx, p, pts = full["idx"], full["p"], full["pts"]
    taus = sorted({int(x) for x in np.linspace(0, p.T - 1, FULL_TABLES).round()})
    want = _tables(p, pts, taus)
    sb = idx.info["slot_bits"]
    for tau in taus:
        keys, ids = idx.export_table(tau)
        sl = keys & np.uint64((1 << sb) - 1)
        assert np.all(np.diff(sl.astype(np.int64)) >= 0), tau      # grouped by slot, slots ascending
        order = np.lexsort((ids, keys))
        ok, oi = want[tau]
        assert np.array_equal(keys[order], ok) and np.array_equal(ids[order], oi), tau


def test_queries_against_the_oracle_query(full):
    """200 queries against the oracle's Strategy 2 query: ids, #Collisions and #Candidates."""
    cfg, idx, p, pts, qs = full["cfg"], full["idx"], full["p"], full["pts"], full["qs"]
    nq = full["nq"]
    pick = np.sort(full["rng"].choice(nq, size=min(QUERY_SAMPLE, nq), replace=False))
    if cfg in ALL_TABLES:
        radius, rows = p.r, 0
    else:
        radius = ROW_RADIUS[cfg]
        rows = oracle.probe_rows(p, radius)
    if rows == 0:                                   # every table, filled in place ([T][n] each)
        keys = np.empty((p.T, pts.shape[0]), np.uint64)
        ids = np.empty((p.T, pts.shape[0]), np.uint32)

        def fill(tau):
            keys[tau], ids[tau] = oracle.table(p, pts, tau)

        list(_POOL.map(fill, range(p.T)))
        want = list(_POOL.map(lambda i: oracle.query(p, pts, (keys, ids), qs[i], radius), pick))
        del keys, ids
    else:
        tables = _tables(p, pts, oracle.probed_tables(p, rows))
        want = list(_POOL.map(lambda i: oracle.query_listed(p, pts, tables, qs[i], radius, rows=rows), pick))
    idx.set_tuning(probe_rows=1 if rows else 0)
    try:
        res = idx.query(full["q_dev"][torch.from_numpy(pick).cuda()], radius)   # the batched path
        plain = idx.query_plain(qs[pick], radius)                             # one query per call
    finally:
        idx.set_tuning(probe_rows=0)
    for j, (ids, ncoll, ncand) in enumerate(want):
        for r in (res, plain):
            assert np.array_equal(r.of(j), ids), (cfg, int(pick[j]))
            assert int(r.collisions[j]) == ncoll and int(r.candidates[j]) == ncand, (cfg, int(pick[j]))


def test_small_workload_every_query_one_per_call(full):
    """The small workload at its stated form: all 200 queries, one per call, through the plain
    path, against the oracle's query over every table (ids and counters)."""
    if full["cfg"] != 1:
        pytest.skip("the small workload only")
    idx, p, pts, qs = full["idx"], full["p"], full["pts"], full["qs"]
    tables = oracle.build_tables(p, pts)
    for i in range(qs.shape[0]):
        ids, ncoll, ncand = oracle.query(p, pts, tables, qs[i], p.r)
        got = idx.query_plain(qs[i:i + 1], p.r)
        assert np.array_equal(got.of(0), ids), i
        assert int(got.collisions[0]) == ncoll and int(got.candidates[0]) == ncand, i


def test_all_queries_at_the_full_radius(full):
    """Every query of the workload through the batched path (as benchmarked) against the GPU
    linear scan, 200 of them against the oracle's linear scan, and every id re-verified."""
    cfg, idx, pts, qs, nq, r = full["cfg"], full["idx"], full["pts"], full["qs"], full["nq"], full["c"]["r"]
    res = idx.query(full["q_dev"], r)
    if full["c"]["d"] <= 3072:
        brute = idx.bruteforce(full["q_dev"], r)
        assert np.array_equal(res.offs, brute.offs) and np.array_equal(res.ids, brute.ids)
    pick = full["rng"].choice(nq, size=min(QUERY_SAMPLE, nq), replace=False)
    want = list(_POOL.map(lambda i: oracle.linear_scan(pts, qs[i], r), pick))
    for i, w in zip(pick, want):
        assert np.array_equal(res.of(i), w), (cfg, int(i))
    counts = np.diff(res.offs)
    owner = np.repeat(np.arange(nq), counts.astype(np.int64))
    assert np.all(_popcount_rows(pts[res.ids] ^ qs[owner]) <= r)
    assert np.all(res.candidates >= counts) and np.all(res.collisions >= res.candidates)


def test_served_form_on_the_full_index(full):
    """The served workload: requests of mixed radius through the server equal the batched
    answers, and a sampled query of each equals the oracle's linear scan."""
    if full["cfg"] != 5:
        pytest.skip("the served workload only")
    fclsh, idx, pts, qs, nq = full["fclsh"], full["idx"], full["pts"], full["qs"], full["nq"]
    reqs = wl.request_stream(5, 24, rate_per_s=2000.0)
    srv = fclsh.Server(idx, slots=4)
    at, tickets = 0, []
    for _, size, radius in reqs:
        size = min(size, 800)
        blk = qs[at % (nq - size): at % (nq - size) + size]
        tickets.append((srv.submit(blk, radius), blk, radius))
        at += size
    for t, blk, radius in tickets:
        got, _ = srv.wait(t)
        want = idx.query(blk, radius)
        assert np.array_equal(got.offs, want.offs) and np.array_equal(got.ids, want.ids)
        j = blk.shape[0] // 2
        assert np.array_equal(got.of(j), oracle.linear_scan(pts, blk[j], radius))
    srv.close()
