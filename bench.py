"""Benchmark of the fcLSH hot path on one GB300 (or N, one independent problem per GPU).

Workload (default): the batched sparse-fingerprint workload, n = 2,000,000 points of
d = 1,024 bits (bit density 0.02, 20% near-duplicates), build radius r = 20 (two parts
of 512 coordinates, W = 2,048, T = 4,094 tables), 50,000 queries (half near-duplicates at
distance 0..20, half fresh) answered in one batch.  One step = the whole hot path over one
batch: build the index from device-resident points (hash every point into its 4,094 keys,
partition and group every table into its bucket directory) and answer the batch in one
persistent launch sequence (hash, probe, dedup, popcount verify, sorted CSR results).
`value` = queries answered per second of step time, with the build inside the step.
`--workload N` selects another workload (2: n = 1M, d = 128, r = 8, one part, 511 tables).

Printed JSON line: metric, value, unit, sizes and timing fields, plus `breakdown` (points hashed/s,
batched queries/s of the query phase alone, plain one-query-at-a-time GPU
queries/s, GPU brute-force queries/s), `roofline` of the dominant kernel,
`cpu_baseline` (the CPU oracle on a bounded sample), `e2e` (the same job through
the C ABI from pinned host buffers, copies included) and `clocks`.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "queries/s at 100% recall and points hashed/s, batched vs plain on one GB300"
CFG = 4

# DRAM traffic / algorithmic bytes of each stage per workload, from ncu captures of the same
# kernels (profiles/); traffic scales with the algorithmic bytes.  An entry is None (traffic
# reported as null) until it is captured, and is reset to None when its kernel changes.
TRAFFIC_RATIO = {
    2: {   # profiles/launch_list_plain_n1M_d128_r8.md (full size)
        "hash": 0.984,
        "hash_mma": 0.986,
        "scatter": 0.996,
        "finish": 1.057,
        "query": 24.2,
        "hist": None,
    },
    4: {   # profiles/launch_list_sparse_n2M_d1024_r20.md (full size)
        "hash_scatter": 0.998,
        "scatter_wide": 1.136,
        "finish": 1.062,
        "query": 0.362,
    },
}


# Points of at least this many words hashed by the scatter sketch are first listed as their set
# coordinates (one pass per build); every part's hash then reads the list (the library's rule).
CSR_MIN_WORDS = 64


def set_bits(points: np.ndarray) -> int:
    """Total set bits of packed uint64 points."""
    flat = np.ascontiguousarray(points).view(np.uint64).reshape(-1)
    count = getattr(np, "bitwise_count", None)
    if count is not None:
        return int(count(flat).sum(dtype=np.uint64))
    table = np.array([bin(i).count("1") for i in range(256)], np.uint8)
    return int(table[flat.view(np.uint8)].sum(dtype=np.uint64))


def hash_part_bytes(w, L: int, hash_tile: int) -> float:
    """Algorithmic bytes of one hash launch (one part): 8 B per key for its L tables and every
    point, plus what the kernel reads of the points -- the packed words (d/8 B per point), or,
    for long points under the scatter sketch, their list of set coordinates (4 B per set bit and
    12 B of start and length per point).  The listing pass itself reads the packed words once per
    build, before the first part; it is not part of this launch."""
    keys = 8.0 * L * w.n
    words = (w.d + 63) // 64
    if hash_tile == 3 and words >= CSR_MIN_WORDS:
        nnz = set_bits(w.points)
        if nnz <= 2 * w.n * words:   # the list's room; denser points keep the packed words
            return 4.0 * nnz + 12.0 * w.n + keys
    return w.n * w.d / 8.0 + keys


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:   # sampler running before the timed region
                time.sleep(0.01)
            self.lines.clear()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def query_count(cfg: int, nq):
    """Queries of a run: as given, else the workload's own count; the served workload draws
    its requests from a pool of 20,000 queries."""
    from paper_1602_02620_gb300 import workloads

    if nq is None and workloads.CONFIGS[cfg]["nq"] == 0:
        return 20_000
    return nq


_WORKER_CACHE = {}


def _cpu_worker(job):
    """One oracle process: time hashing (direct route) and linear-scan queries on its own
    slice of the job for about budget_s seconds; returns the counts and the seconds taken.
    The workload and its parameters are made once per process (a pool is reused across steps)."""
    cfg, n, nq, k, cores, budget_s = job
    import oracle
    from paper_1602_02620_gb300 import workloads

    key = (cfg, n, nq)
    if key not in _WORKER_CACHE:
        w0 = workloads.make(cfg, n=n, nq=nq)
        p0 = oracle.derive_params(w0.index_seed, w0.d, w0.r,
                                  rep=workloads.build_options(cfg).get("replicate", 1))
        _WORKER_CACHE.clear()
        _WORKER_CACHE[key] = (w0, p0)
    w, p = _WORKER_CACHE[key]
    nqall = w.queries.shape[0]
    h0, q0 = (k * w.n) // cores, (k * nqall) // cores
    t0 = time.perf_counter()
    nh = 0
    while time.perf_counter() - t0 < budget_s * 0.45 and nh < w.n:
        a = (h0 + nh) % w.n
        oracle.keys_direct(p, w.points[a:a + 50])
        nh += min(50, w.n - a)
    th = time.perf_counter() - t0
    t0 = time.perf_counter()                        # the oracle's Algorithm 2 route, for reference
    nf = 0
    while time.perf_counter() - t0 < budget_s * 0.1 and nf < w.n:
        a = (h0 + nf) % w.n
        oracle.keys_fht(p, w.points[a:a + 50])
        nf += min(50, w.n - a)
    tf = time.perf_counter() - t0
    t0 = time.perf_counter()
    nqs = 0
    while time.perf_counter() - t0 < budget_s * 0.45 and nqs < nqall:
        oracle.linear_scan(w.points, w.queries[(q0 + nqs) % nqall], w.r)
        nqs += 1
    tq = time.perf_counter() - t0
    return nh, th, nqs, tq, int(p.T), nf, tf


def cpu_baseline(cfg: int, n, nq, budget_s: float = 12.0, cores: int | None = None, pool=None):
    """The CPU oracle as it stands, on a bounded sample of the same job, on the host's cores.

    Job = hash all n points into their T keys (direct route of the covering
    definition) + answer every query by the oracle's exact answer (linear scan).
    One process per core (spawned: this process may hold a CUDA context) times its
    own slice of both for about budget_s seconds; the summed rates are scaled to the
    whole job.
    """
    import multiprocessing as mp
    from paper_1602_02620_gb300 import workloads

    nq = query_count(cfg, nq)
    w = workloads.make(cfg, n=n, nq=nq)
    cores = cores or os.cpu_count() or 1
    jobs = [(cfg, n, nq, k, cores, budget_s) for k in range(cores)]
    if pool is not None:
        res = pool.map(_cpu_worker, jobs)
    elif cores == 1:
        res = [_cpu_worker(jobs[0])]
    else:
        with mp.get_context("spawn").Pool(cores) as own:
            res = own.map(_cpu_worker, jobs)
    hash_rate = sum(r[0] / r[1] for r in res)
    query_rate = sum(r[2] / r[3] for r in res)
    nqall = w.queries.shape[0]
    job_s = w.n / hash_rate + nqall / query_rate
    one = res[0]
    one_job_s = w.n * one[1] / one[0] + nqall * one[3] / one[2]
    nh, nqs, T = sum(r[0] for r in res), sum(r[2] for r in res), res[0][4]
    return {"value": nqall / job_s, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": "%d points hashed (direct route, all %d tables) + %d queries by linear scan over all %d points "
                      "on %d processes, scaled to the job of %d points + %d queries"
                      % (nh, T, nqs, w.n, cores, w.n, nqall),
            "points_hashed_per_s": hash_rate, "linear_scan_queries_per_s": query_rate,
            "points_hashed_per_s_algorithm2": sum(r[5] / r[6] for r in res if r[6] > 0),
            "single_core_value": nqall / one_job_s}


HASH_ROUTES = ((0, "wht"), (1, "wht_wide_tile"), (3, "wht_scatter_sketch"), (2, "direct_tensor_cores"),
               (4, "direct_cuda_cores"))


def hash_routes(fclsh, idx, pts, reps: int = 3):
    """Points hashed per second into all T keys by every hash kernel that applies to the
    index: Algorithm 2 (sketch + WHT: tiles 0, 1, 3) against the direct O(dL) route of Eq. 1
    (the basic covering construction: tensor cores, tile 2; CUDA cores, tile 4) -- the
    paper's fcLSH / bcLSH comparison of hash computation time (Sec. 4.3)."""
    import torch

    n = min(int(pts.shape[0]), max(4096, (1 << 28) // idx.T))   # at most 2 GB of keys
    pts = pts[:n]
    keys = torch.empty((idx.T, n), dtype=torch.int64, device="cuda")
    saved = idx.tuning()
    out = {}
    for tl, name in HASH_ROUTES:
        try:
            idx.set_tuning(**dict(saved, hash_tile=tl))
        except fclsh.FclshError:
            continue
        idx.hash(pts, out=keys)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            idx.hash(pts, out=keys)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        out[name] = {"ms": ms, "points": n, "points_per_s": n / (ms / 1000.0)}
    idx.set_tuning(**saved)
    del keys
    return out


def hash_ablation(fclsh, n: int = 65_536):
    """The paper's hash-time experiment on synthetic data of n = 64K points (Sec. 4.3):
    d = 128 with r = 3..7, and r = 5 with d = 32..512, every hash route."""
    import torch
    from paper_1602_02620_gb300 import workloads

    rows = []
    for d, r in [(128, 3), (128, 4), (128, 5), (128, 6), (128, 7), (32, 5), (64, 5), (256, 5), (512, 5)]:
        words = (d + 63) // 64
        a = np.zeros((n, words), np.uint64)
        workloads._lib().wl_uniform(workloads._key(100 + d, r), 0, n, d, a.ctypes.data)
        pts = torch.from_numpy(a.view(np.int64)).cuda()
        idx = fclsh.build(pts, d, r, 7)
        routes = hash_routes(fclsh, idx, pts)
        rows.append({"d": d, "r": r, "W": idx.W, "tables": idx.T,
                     "points_per_s": {k: v["points_per_s"] for k, v in routes.items()}})
        idx.free()
    return {"n": n, "data": "uniform bits", "rows": rows}


def served(fclsh, idx, w, n_req: int = 160, load: float = 0.5, batched_qps: float = 1e6, probe_rows: int = 0):
    """Continuous batching on the resident index: a Poisson stream of requests of U{1..4096}
    queries with radii in {r/4, r/2, 3r/4, r} (rounded), offered at `load` times the batched
    throughput, through the server (4 slots, batches of up to 16,384 queries) and, with the
    same arrival times, through a server that runs one request per batch on one slot; then
    each request alone (submitted when the server is idle: its latency without queueing).
    probe_rows = 1 probes only the code rows each request's radius needs (same ids)."""
    import threading

    idx.set_tuning(probe_rows=probe_rows)
    rng = np.random.default_rng(7)
    sizes = rng.integers(1, 4097, size=n_req)
    radii_set = sorted({max(1, round(w.r * f)) for f in (0.25, 0.5, 0.75, 1.0)})
    radii = rng.choice(radii_set, size=n_req)
    rate = load * batched_qps / float(sizes.mean())
    gaps = rng.exponential(1.0 / rate, size=n_req)
    nq = w.queries.shape[0]
    starts = rng.integers(0, max(1, nq - 4096), size=n_req)
    blocks = [w.queries[int(a):int(a) + int(z)] for a, z in zip(starts, sizes)]

    def open_loop(srv):
        tickets = [None] * n_req

        def feed():
            t0 = time.perf_counter()
            at = 0.0
            for i in range(n_req):
                at += gaps[i]
                dt = t0 + at - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                tickets[i] = srv.submit(blocks[i], int(radii[i]))

        th = threading.Thread(target=feed)
        th.start()
        th.join()
        for t in tickets:
            srv.wait(t)
        return srv.stats()

    srv = fclsh.Server(idx, slots=4, max_batch_queries=16384)
    st = open_loop(srv)
    srv.close()
    one = fclsh.Server(idx, slots=1, max_batch_queries=1)
    st1 = open_loop(one)
    one.close()
    alone = fclsh.Server(idx, slots=1, max_batch_queries=1)
    for i in range(n_req):
        alone.wait(alone.submit(blocks[i], int(radii[i])))
    sta = alone.stats()
    alone.close()
    idx.set_tuning(probe_rows=0)
    return {"requests": n_req, "probe_rows": probe_rows, "load": load,
            "offered_queries_per_s": rate * float(sizes.mean()), "radii": radii_set,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "queries_per_s": st["queries_per_s"],
            "mean_batch_queries": st["mean_batch_queries"], "batches": st["batches"],
            "one_at_a_time_queries_per_s": st1["queries_per_s"], "one_at_a_time_p50_ms": st1["p50_ms"],
            "one_at_a_time_p99_ms": st1["p99_ms"],
            "alone_p50_ms": sta["p50_ms"], "alone_p99_ms": sta["p99_ms"]}


def serve_sweep(args):
    """Offered load swept from a quarter to one and a half times the batched throughput on the
    workload's resident index (built once), every query answered both ways (served, one request
    per batch) from the same Poisson arrivals; one JSON line."""
    import torch
    from paper_1602_02620_gb300 import fclsh, workloads

    w = workloads.make(args.workload, n=args.n, nq=query_count(args.workload, args.nq))
    pts = torch.from_numpy(w.points.view(np.int64)).cuda()
    qs = torch.from_numpy(w.queries.view(np.int64)).cuda()
    bopts = workloads.build_options(args.workload)
    cache = os.path.join(ROOT, "paper_1602_02620_gb300", "_build", "autotune.json")
    idx = fclsh.build(pts, w.d, w.r, w.index_seed, **bopts)
    tuned = idx.autotune(qs[: min(qs.shape[0], 8192)], w.r, cache)
    ctx = idx.context()
    for _ in range(3):
        ctx.query_async(qs, w.r)
        ctx.wait()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(5):
        ctx.query_async(qs, w.r)
        ctx.wait()
    b.record()
    torch.cuda.synchronize()
    ctx.close()
    batched_qps = qs.shape[0] * 5 / (a.elapsed_time(b) / 1000.0)
    rows = []
    for probe_rows in (0, 1):
        for load in (0.25, 0.5, 1.0, 1.5):
            rows.append(served(fclsh, idx, w, n_req=args.serve_requests, load=load, batched_qps=batched_qps,
                               probe_rows=probe_rows))
    idx.free()
    print(json.dumps({"serve_sweep": {"workload": w.name, "batched_queries_per_s": batched_qps, "tuning": tuned,
                                      "rows": rows}}))


def classic_lsh(fclsh, w, pts, qs, truth, seed: int, delta: float = 0.1) -> dict:
    """Classic bit-sampling LSH (Sec. 2.2) with the covering index's table count and k by the rule
    of Sec. 4.1 for false-negative ratio delta, on the same points and batch: its recall against
    the exact answers (it reports only verified neighbours, so recall = its hits / the exact hits),
    its counters, and its build + batch time, beside covering LSH's recall of 1."""
    import torch

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    idx = fclsh.build(pts, w.d, w.r, seed, classic_delta=delta)
    ev[1].record()
    res = idx.query(qs, w.r)
    ev[2].record()
    torch.cuda.synchronize()
    samples, _ = idx.classic_params()
    L, k = idx.T, int(samples.shape[1])
    idx.free()
    got, want = np.diff(res.offs).astype(np.int64), np.diff(truth.offs).astype(np.int64)
    has = want > 0
    return {"delta": delta, "tables": L, "k": k, "recall": float(got.sum() / max(want.sum(), 1)),
            "mean_query_recall": float((got[has] / want[has]).mean()) if has.any() else 1.0,
            "queries_fully_answered": float((got[has] == want[has]).mean()) if has.any() else 1.0,
            "collisions_per_query": float(res.collisions.mean()), "candidates_per_query": float(res.candidates.mean()),
            "build_ms": ev[0].elapsed_time(ev[1]), "batch_ms": ev[1].elapsed_time(ev[2]),
            "queries_per_s": qs.shape[0] / (ev[0].elapsed_time(ev[2]) / 1000.0)}


def workload_config(w, tables: int, nq: int, name: str) -> dict:
    """The `config` object of a JSON line (the same for both arms)."""
    sb = 13
    while sb < 32 and (1 << sb) < w.n:
        sb += 1
    pts_b = w.points.nbytes
    index_b = tables * w.n * 8 + tables * ((1 << sb) + 4) * 4
    return {"workload": name, "n": w.n, "d": w.d, "r": w.r, "tables": tables, "queries": nq,
            "step": "build index from device-resident points + one batch of all queries",
            "l2": "inputs and index %s than L2 (129 MB): %.3g MB of points -> %.3g GB of keys, %.3g GB index"
                  % ("larger" if index_b > 129e6 else "smaller", pts_b / 1e6, w.n * tables * 8 / 1e9, index_b / 1e9)}


def run_reference(args, rank: int):
    """The CPU oracle timed on the host's cores on the same workload (one pool of spawned
    processes for all steps; each step a bounded sample, the whole run a few minutes)."""
    if rank != 0:
        return
    import multiprocessing as mp

    import oracle
    from paper_1602_02620_gb300 import workloads

    w = workloads.make(args.workload, n=args.n, nq=query_count(args.workload, args.nq))
    T = oracle.derive_params(w.index_seed, w.d, w.r,
                             rep=workloads.build_options(args.workload).get("replicate", 1)).T
    total = args.warmup + args.steps
    budget = max(0.5, min(4.0, 150.0 / max(total, 1)))   # seconds of oracle work per step
    cores = os.cpu_count() or 1
    steps = []
    with mp.get_context("spawn").Pool(cores) as pool:
        for i in range(total):
            cb = cpu_baseline(args.workload, args.n, args.nq, budget_s=budget, cores=cores, pool=pool)
            if i >= args.warmup:
                steps.append(cb)
    v = statistics.median(s["value"] for s in steps)
    cb = dict(steps[-1])
    cb["value"] = v
    nq = int(w.queries.shape[0])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * nq / v,
            "ms_per_step_kind": "extrapolated from a bounded sample (see cpu_baseline.sample)",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": workload_config(w, T, nq, w.name),
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_sharded(args, w, seed, rank: int, world: int, local: int, dist):
    """Strong scaling over points (the sharding of the index by point ids): rank k builds its
    contiguous id range with the same seed and Algorithm 1's shape of the whole set, answers
    the whole batch, and the per-shard answers (sorted, offset to global ids) are gathered and
    merged on every rank.  One step = the build of every shard + the batch + the gather."""
    import torch
    from paper_1602_02620_gb300 import fclsh, shard

    nq = int(w.queries.shape[0])
    lo, hi = shard.shard_range(w.n, rank, world)
    pts = torch.from_numpy(w.points[lo:hi].view(np.int64)).cuda()
    qs = torch.from_numpy(w.queries.view(np.int64)).cuda()
    bopts = workloads_build_options(args.workload)

    tables = []

    def step():
        sh = shard.ShardedIndex(pts, w.n, w.d, w.r, seed, rank, world, **bopts)
        if sh.index is not None and not tables:
            tables.append(sh.index.T)
        res = sh.query(qs, w.r)
        sh.free()
        return res

    for _ in range(max(args.warmup, 1)):
        res = step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = fclsh.kernel_launches()
    ev0.record()
    for _ in range(args.steps):
        res = step()
    ev1.record()
    torch.cuda.synchronize()
    launches = fclsh.kernel_launches() - l0
    if dist:
        dist.barrier()
    elapsed = ev0.elapsed_time(ev1) / 1000.0
    if dist:
        tt = torch.tensor([elapsed], dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed = float(tt.item())
    value = nq * args.steps / elapsed
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": dict(workload_config(w, tables[0] if tables else 0, nq, w.name + " (sharded by points)"),
                           parallelism="points sharded over %d GPUs, answers gathered" % world),
            "results_per_step": int(res.offs[-1]), "gpu_launches": int(launches),
        }))
    if dist:
        dist.destroy_process_group()


def workloads_build_options(cfg: int) -> dict:
    from paper_1602_02620_gb300 import workloads

    return workloads.build_options(cfg)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fclsh")
    ap.add_argument("--plain-sample", type=int, default=300)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=None, help="fewer points of the same workload (profiling)")
    ap.add_argument("--nq", type=int, default=None, help="fewer queries of the same workload (profiling)")
    ap.add_argument("--hash-tile", type=int, default=None, choices=(0, 1, 2, 3, 4),
                    help="force the hash kernel (0/1: WHT tiles, 2: tensor-core contraction) instead of the tuned one")
    ap.add_argument("--slot-bits", type=int, default=None,
                    help="directory slot bits (to profile a smaller instance in the full-size directory layout)")
    ap.add_argument("--serve-sweep", action="store_true",
                    help="only the served form: offered load 0.25x..1.5x the batched throughput, one JSON line")
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--shard", action="store_true",
                    help="with N > 1: shard the points (each rank indexes a contiguous id range with the same seed, "
                         "answers the whole batch, and the answers are gathered); strong scaling")
    ap.add_argument("--workload", type=int, default=CFG, choices=[1, 2, 3, 4, 5, 6, 7, 8],
                    help="workload id (default: 4, the n=2M d=1024 r=20 batched sparse workload)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.serve_sweep:
        serve_sweep(args)
        return

    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    from paper_1602_02620_gb300 import fclsh, workloads

    w = workloads.make(args.workload, n=args.n, nq=query_count(args.workload, args.nq))
    # every rank builds with the same seed: without --shard each GPU holds its own replica of the
    # index and answers its own batch (weak scaling); with --shard it holds one contiguous id range
    seed = w.index_seed
    nq = int(w.queries.shape[0])
    if args.shard:
        run_sharded(args, w, seed, rank, world, local, dist)
        return
    pts = torch.from_numpy(w.points.view(np.int64)).cuda()
    qs = torch.from_numpy(w.queries.view(np.int64)).cuda()

    # kernel shapes for this workload: autotuned once on a sample batch (cached)
    cache = os.path.join(ROOT, "paper_1602_02620_gb300", "_build", "autotune.json")
    bopts = workloads.build_options(args.workload)   # e.g. replication
    if args.slot_bits:
        bopts["slot_bits"] = args.slot_bits
    idx0 = fclsh.build(pts, w.d, w.r, seed, **bopts)
    tuned = idx0.autotune(qs[: min(nq, 8192)], w.r, cache)
    idx0.free()
    if args.hash_tile is not None:
        tuned["hash_tile"] = args.hash_tile

    def step(timing: bool):
        """One step: build + the batch on a fresh context (its first batch runs eagerly, so
        per-phase timing costs it nothing); CUDA events on the legacy stream mark the build,
        the batch and the teardown (the library's streams are blocking, so they order)."""
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record()
        idx = fclsh.build(pts, w.d, w.r, seed, timing=timing, hash_tile=tuned["hash_tile"], **bopts)
        ev[1].record()
        idx.set_tuning(**tuned)
        ctx = idx.context()
        ctx.query_async(qs, w.r)
        dr = ctx.wait()
        ev[2].record()
        t = idx.timing_read()
        ctx.close()
        info = dict(idx.info)
        idx.free()
        ev[3].record()
        return t, int(dr.total), info, ev

    for _ in range(args.warmup):
        step(True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = fclsh.kernel_launches()
    torch.cuda.synchronize()
    ev0.record()
    acc = {}
    marks = []
    total = 0
    for _ in range(args.steps):
        t, total, info, ev = step(True)
        marks.append(ev)
        for k in ("build_hash", "build_sort", "build_partition", "build_finish", "build_partition_hist",
                  "query_kernel", "query_csr", "query_heavy"):
            a = acc.setdefault(k, [0.0, 0])
            a[0] += t[k][0]
            a[1] += t[k][1]
    hash_ms, hash_n = acc["build_hash"]
    sort_ms = acc["build_sort"][0]
    ev1.record()
    torch.cuda.synchronize()
    launches = fclsh.kernel_launches() - l0
    # where a step's time goes (averages over the timed steps)
    per = lambda k: acc[k][0] / args.steps
    build_ms = sum(e[0].elapsed_time(e[1]) for e in marks) / args.steps
    batch_ms = sum(e[1].elapsed_time(e[2]) for e in marks) / args.steps
    teardown_ms = sum(e[2].elapsed_time(e[3]) for e in marks) / args.steps
    step_breakdown = {
        "build_ms": build_ms, "build_hash_kernels_ms": per("build_hash"),
        "build_sort_kernels_ms": per("build_sort"),
        "build_other_ms": build_ms - per("build_hash") - per("build_sort"),
        "batch_ms": batch_ms, "batch_query_kernel_ms": per("query_kernel"),
        "batch_query_heavy_kernel_ms": per("query_heavy"), "batch_csr_ms": per("query_csr"),
        "batch_other_ms": batch_ms - per("query_kernel") - per("query_csr"),
        "teardown_ms": teardown_ms,
        "note": "build_other: allocations, parameter copies, memsets and the status read of the build; "
                "batch_other: context set-up and the result-size read; teardown: freeing the context and index",
    }
    if dist:
        dist.barrier()
    clk = clocks.stop()
    elapsed = ev0.elapsed_time(ev1) / 1000.0
    if dist:
        tt = torch.tensor([elapsed], dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed = float(tt.item())
    ms_step = 1000.0 * elapsed / args.steps
    value = world * nq * args.steps / elapsed

    # ---- query phase alone (index resident), batched vs plain vs brute force
    idx = fclsh.build(pts, w.d, w.r, seed, hash_tile=tuned["hash_tile"], **bopts)
    idx.set_tuning(**tuned)
    ctx = idx.context()
    for _ in range(3):
        ctx.query_async(qs, w.r)
        ctx.wait()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    a.record()
    for _ in range(reps):
        ctx.query_async(qs, w.r)
        ctx.wait()
    b.record()
    torch.cuda.synchronize()
    batched_qps = nq * reps / (a.elapsed_time(b) / 1000.0)
    idx.timing_enable(True)
    for _ in range(reps):
        ctx.query_async(qs, w.r)
        ctx.wait()
    tq = idx.timing_read(reset=True)
    idx.timing_enable(False)
    res = ctx.fetch()
    ctx.close()
    # verify (query) kernel: algorithmic bytes per query = the T directory words it reads
    # (2 x 4 B per table) + 8 B per colliding bucket entry + d/8 per distinct candidate + its d/8 bits
    qk_bytes = float(nq * (idx.T * 8 + w.d / 8) + 8 * res.collisions.sum() + (w.d / 8) * res.candidates.sum())
    ns = min(args.plain_sample, nq)
    if args.n is not None or args.nq is not None or args.workload != CFG:
        line_name = "%s%s" % (w.name, " (reduced: n=%d, queries=%d)" % (w.n, nq) if args.n or args.nq else "")
    else:
        line_name = w.name
    t0 = time.perf_counter()
    plain = idx.query_plain(w.queries[:ns], w.r)
    plain_qps = ns / (time.perf_counter() - t0)
    assert np.array_equal(plain.ids, res.ids[: int(res.offs[ns])]), "plain and batched answers differ"
    torch.cuda.synchronize()
    brute_qps = None
    if w.d <= 3072:                       # the GPU linear scan keeps queries of up to 48 words in shared memory
        t0 = time.perf_counter()
        brute = idx.bruteforce(qs, w.r)
        brute_qps = nq / (time.perf_counter() - t0)
        assert np.array_equal(brute.ids, res.ids) and np.array_equal(brute.offs, res.offs), "brute force differs"
    T = idx.T
    serve = served(fclsh, idx, w, batched_qps=batched_qps)
    serve_rows = served(fclsh, idx, w, batched_qps=batched_qps, probe_rows=1)
    routes = hash_routes(fclsh, idx, pts)
    idx.free()
    classic = classic_lsh(fclsh, w, pts, qs, res, seed) if 0 < w.r < w.d <= 4096 else None

    # ---- e2e through the C ABI from pinned host buffers
    hp = torch.from_numpy(w.points.view(np.int64)).pin_memory()
    hq = torch.from_numpy(w.queries.view(np.int64)).pin_memory()
    e2e_t = []
    d2h = 0
    e2e_reps = max(2, min(args.steps, 5))
    for i in range(e2e_reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        idx2 = fclsh.build(hp, w.d, w.r, seed, hash_tile=tuned["hash_tile"], **bopts)
        idx2.set_tuning(**tuned)
        r2 = idx2.query(hq, w.r)
        e2e_t.append(time.perf_counter() - t0)
        d2h = r2.offs.nbytes + r2.ids.nbytes + r2.collisions.nbytes + r2.candidates.nbytes
        assert np.array_equal(r2.ids, res.ids)
        idx2.free()
    e2e = {"value": nq / statistics.median(e2e_t), "unit": "queries/s",
           "h2d_bytes_per_step": int(w.points.nbytes + w.queries.nbytes), "d2h_bytes_per_step": int(d2h)}
    if workloads.CONFIGS[args.workload]["kind"] == "sparse_skewed":
        # sparse data the way a user holds it: CSR rows of set coordinates, packed on the device
        def csr(a):
            bits = np.unpackbits(a.view(np.uint8).reshape(a.shape[0], -1), axis=1, bitorder="little")[:, : w.d]
            rows, cols = np.nonzero(bits)
            ptr = np.zeros(a.shape[0] + 1, np.uint64)
            np.add.at(ptr, rows + 1, 1)
            return (torch.from_numpy(np.cumsum(ptr).astype(np.uint64).view(np.int64)).pin_memory(),
                    torch.from_numpy(cols.astype(np.uint32).view(np.int32)).pin_memory())
        pi, pc = csr(w.points)
        qi, qc = csr(w.queries)
        qdev = torch.empty((nq, w.words), dtype=torch.int64, device="cuda")
        e2e_s = []
        for i in range(e2e_reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            idx2 = fclsh.build_sparse(pi, pc, w.d, w.r, seed, hash_tile=tuned["hash_tile"], **bopts)
            idx2.set_tuning(**tuned)
            fclsh.pack_sparse(qi, qc, w.d, out=qdev)
            r2 = idx2.query(qdev, w.r)
            e2e_s.append(time.perf_counter() - t0)
            assert np.array_equal(r2.ids, res.ids)
            idx2.free()
        e2e["sparse_input"] = {"value": nq / statistics.median(e2e_s), "unit": "queries/s",
                               "h2d_bytes_per_step": int(pi.numel() * 8 + pc.numel() * 4 + qi.numel() * 8 +
                                                         qc.numel() * 4),
                               "d2h_bytes_per_step": int(d2h)}

    # ---- rooflines (HBM) of the build's kernels, from the CUDA events of the timed steps.
    # Algorithmic bytes per launch:
    #   hash (Algorithm 2, one part): hash_part_bytes (points read + 8 B per key for its W-1 tables)
    #   partition scatter (partition_scatter_kernel): per entry 8 B read + 8 B packed write
    #   partition histogram (radix_hist_kernel + scan): per entry 8 B read
    #   segment finish: per entry 8 B read + 8 B written, plus 4 B per directory slot
    peak, peak_kind = peaks()
    hash_avg = hash_ms / max(hash_n, 1)
    L = info["W"] - 1
    entries = w.n * L
    slots = L * ((1 << info["slot_bits"]) + 1)
    hash_bytes = hash_part_bytes(w, L, tuned["hash_tile"])
    hash_stage = {2: ("hash_mma_kernel (tensor-core contraction, all W-1 keys per point)", "hash_mma"),
                  3: ("hash_tile_kernel (Algorithm 2, sketch scattered from set bits)", "hash_scatter")}.get(
        tuned["hash_tile"], ("hash_tile_kernel (Algorithm 2, all W-1 keys per point)", "hash"))
    dbits = info["slot_bits"] - 12   # partition digit bits: a segment spans 4,096 slots
    part_name = ("partition_scatter_kernel (partition by the top 8 slot bits into bins, packed output)" if dbits == 8
                 else "partition_wide_kernel<%d> (partition by the top %d slot bits into bins, packed output)"
                 % (dbits, dbits))
    stages = {
        hash_stage[0]: (acc["build_hash"], hash_bytes, hash_stage[1]),
        part_name: (acc["build_partition"], 16 * entries, "scatter" if dbits == 8 else "scatter_wide"),
        "partition histogram + scan (exact fallback)": (acc["build_partition_hist"], 8 * entries, "hist"),
        "segment finish (segment_one_kernel + segment_finish_kernel)":
            (acc["build_finish"], 16 * entries + 4 * slots, "finish"),
    }
    # traffic ratios apply to the full-size workload they were captured on
    ratios = TRAFFIC_RATIO.get(args.workload, {}) if args.n is None and args.nq is None else {}
    kernels = []
    parts_timed = info["t"] * args.steps      # every part of every timed step
    for name, ((ms, cnt), part_bytes, tag) in stages.items():
        if cnt == 0:
            continue
        avg = ms / cnt
        if tag == "hist":    # runs only on the chunks whose bins overflowed: their entries are not counted here
            kernels.append({"kernel": name, "total_ms": ms, "launches": cnt, "avg_ms": avg, "bytes_per_launch": None,
                            "achieved_gbs": None, "frac": None, "traffic": None})
            continue
        # a part's tables may be processed in several chunks (launches): bytes per launch on average
        nbytes = part_bytes * parts_timed / cnt
        gbs = nbytes / (avg / 1000.0) / 1e9
        ratio = ratios.get(tag)
        kernels.append({"kernel": name, "total_ms": ms, "launches": cnt, "avg_ms": avg, "bytes_per_launch": nbytes,
                        "achieved_gbs": gbs, "frac": gbs / peak,
                        "traffic": int(ratio * nbytes) if ratio else None})
    # the batch's query kernel inside the timed steps (one launch per step, plus a second
    # pass for a step whose results passed the context's buffer)
    qk_ms, qk_n = acc["query_kernel"]
    qk_avg = qk_ms / max(qk_n, 1)
    qk_bytes_launch = qk_bytes * args.steps / max(qk_n, 1)
    qk_gbs = qk_bytes_launch / (qk_avg / 1000.0) / 1e9
    qratio = ratios.get("query")
    qk = {"kernel": "query_batch_kernel + query_heavy_kernel (S1-S3 for the %s-query batch)" % format(nq, ","),
          "total_ms": qk_ms,
          "launches": qk_n, "avg_ms": qk_avg, "bytes_per_launch": qk_bytes_launch, "achieved_gbs": qk_gbs,
          "frac": qk_gbs / peak, "traffic": int(qratio * qk_bytes_launch) if qratio else None,
          "note": "random 32 B sectors: a directory read and a bucket run per (query, table), a point per candidate; "
                  "a launch here is one timed window: the batch kernel, then the heavy-query kernel"}
    if qratio:   # as DRAM sees it: the measured traffic over the live launch time
        qk["dram_gbs"] = qratio * qk_bytes_launch / (qk_avg / 1000.0) / 1e9
        qk["dram_frac"] = qk["dram_gbs"] / peak
    kernels.append(qk)
    csr_ms, csr_n = acc["query_csr"]
    kernels.append({"kernel": "result CSR (scan + gather_runs_kernel)", "total_ms": csr_ms, "launches": csr_n,
                    "avg_ms": csr_ms / max(csr_n, 1), "bytes_per_launch": None, "achieved_gbs": None,
                    "frac": None, "traffic": None})
    dom = max((k for k in kernels if k["frac"] is not None), key=lambda k: k["total_ms"])
    kernels_ms = sum(k["total_ms"] for k in kernels) / args.steps
    step_breakdown["kernels_ms"] = kernels_ms
    step_breakdown["kernels_share_of_step"] = kernels_ms / ms_step
    ach = hash_bytes / (hash_avg / 1000.0) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": workload_config(w, T, nq, line_name),
        "breakdown": {
            "build_hash_ms": hash_avg, "build_sort_ms": sort_ms / args.steps,
            "hash_roofline_frac": ach / peak,
            "points_hashed_per_s": w.n / (hash_avg / 1000.0),
            "batched_query_queries_per_s": batched_qps,
            "batched_query_kernel_ms": tq["query_kernel"][0] / max(tq["query_kernel"][1], 1),
            "batched_query_csr_ms": tq["query_csr"][0] / max(tq["query_csr"][1], 1),
            "collisions_per_query": float(res.collisions.mean()), "candidates_per_query": float(res.candidates.mean()),
            "results_per_query": float(np.diff(res.offs).mean()),
            "plain_queries_per_s": plain_qps, "plain_sample": ns,
            "bruteforce_queries_per_s": brute_qps,
            "results_per_step": total,
            "tuning": tuned,
        },
        "classic_lsh": classic,
        "served": serve,
        "served_row_probe": serve_rows,
        "hash_routes": routes,
        "hash_ablation": hash_ablation(fclsh) if not args.n and not args.nq else None,
        "roofline": {"kernel": dom["kernel"], "bound": "hbm", "achieved": dom["achieved_gbs"], "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": dom["frac"], "traffic": dom["traffic"],
                     "bytes_per_launch": dom["bytes_per_launch"], "avg_launch_ms": dom["avg_ms"]},
        "kernels": kernels,
        "step_breakdown": step_breakdown,
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": e2e,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.n, args.nq)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
