"""ctypes binding of libfclsh.so (the C ABI in include/fclsh.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Arrays may be numpy arrays (host memory) or torch tensors (host
or CUDA); their data pointers are passed through unchanged, so device tensors
stay on the device.  There is no fallback: if the library has not been built,
every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FCLSH_CHECKED=1 selects the checked build (bounds-checked kernels; built by build(checked=True))
LIB_PATH = os.path.join(_HERE, "_build_checked" if os.environ.get("FCLSH_CHECKED") == "1" else "_build", "libfclsh.so")

OK, EINVAL, ENOMEM, ECUDA, ERADIUS, ETIMEOUT, EOVERFLOW = range(7)
_STATUS = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ERADIUS", 5: "ETIMEOUT", 6: "EOVERFLOW"}


class FclshError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, str(status)), msg))
        self.status = status


class BuildOpts(ctypes.Structure):
    _fields_ = [("t", ctypes.c_uint32), ("slot_bits", ctypes.c_uint32), ("mem_budget", ctypes.c_uint64),
                ("perm", ctypes.c_void_p), ("part_off", ctypes.c_void_p), ("m", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("timing", ctypes.c_uint32), ("hash_tile", ctypes.c_uint32), ("replicate", ctypes.c_uint32),
                ("approx_c", ctypes.c_double), ("classic_tables", ctypes.c_uint32), ("classic_k", ctypes.c_uint32),
                ("classic_delta", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("d", ctypes.c_uint32), ("words", ctypes.c_uint32), ("r", ctypes.c_uint32),
                ("t", ctypes.c_uint32), ("rp", ctypes.c_uint32), ("W", ctypes.c_uint32), ("T", ctypes.c_uint32),
                ("slot_bits", ctypes.c_uint32), ("P", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("device", ctypes.c_int), ("rep", ctypes.c_uint32)]


class Result(ctypes.Structure):
    _fields_ = [("nq", ctypes.c_uint64), ("offs", ctypes.POINTER(ctypes.c_uint64)), ("ids", ctypes.POINTER(ctypes.c_uint32)),
                ("collisions", ctypes.POINTER(ctypes.c_uint64)), ("candidates", ctypes.POINTER(ctypes.c_uint64))]


class DeviceResult(ctypes.Structure):
    _fields_ = [("nq", ctypes.c_uint64), ("total", ctypes.c_uint64), ("offs", ctypes.c_void_p), ("ids", ctypes.c_void_p),
                ("collisions", ctypes.c_void_p), ("candidates", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    _fields_ = [("query_block", ctypes.c_uint32), ("query_ctas_per_sm", ctypes.c_uint32),
                ("hash_set_log2", ctypes.c_uint32), ("inline_probe", ctypes.c_uint32), ("use_graph", ctypes.c_uint32),
                ("hash_tile", ctypes.c_uint32), ("probe_rows", ctypes.c_uint32), ("verify_filter", ctypes.c_uint32),
                ("heavy_kernel", ctypes.c_uint32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class ServerOpts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint32), ("max_batch_queries", ctypes.c_uint32), ("mem_reserve", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_uint64), ("queries", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("deferred_for_memory", ctypes.c_uint64), ("mean_batch_queries", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("queries_per_s", ctypes.c_double)]


#: Every entry point of include/fclsh.h: name -> (restype, argtypes).
_vp, _u32, _u64, _i = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
SIGNATURES = {
    "fclsh_build": (_i, [_vp, _u64, _u32, _u32, _u64, _vp, _vp]),
    "fclsh_free": (None, [_vp]),
    "fclsh_get_info": (_i, [_vp, _vp]),
    "fclsh_get_params": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "fclsh_get_classic_params": (_i, [_vp, _vp, _vp, _vp]),
    "fclsh_derive_params": (_i, [_u64, _u32, _u32, _u64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "fclsh_hash": (_i, [_vp, _vp, _u64, _vp, _vp]),
    "fclsh_bucket": (_i, [_vp, _u32, _u64, _vp, _u64, _vp]),
    "fclsh_export_table": (_i, [_vp, _u32, _vp, _vp]),
    "fclsh_export_keys": (_i, [_vp, _vp, _u64, _vp]),
    "fclsh_query": (_i, [_vp, _vp, _u64, _u32, _vp, _vp, _vp]),
    "fclsh_query_plain": (_i, [_vp, _vp, _u64, _u32, _vp, _vp]),
    "fclsh_bruteforce": (_i, [_vp, _vp, _u64, _u32, _vp, _vp]),
    "fclsh_query_plain_noalloc": (_i, [_vp, _vp, _u32, _vp, _u64, _vp, _vp]),
    "fclsh_result_free": (None, [_vp]),
    "fclsh_qctx_create": (_i, [_vp, _vp]),
    "fclsh_qctx_free": (None, [_vp]),
    "fclsh_query_async": (_i, [_vp, _vp, _u64, _u32, _vp, _vp]),
    "fclsh_qctx_wait": (_i, [_vp, _vp]),
    "fclsh_qctx_fetch": (_i, [_vp, _vp]),
    "fclsh_get_tuning": (_i, [_vp, _vp]),
    "fclsh_set_tuning": (_i, [_vp, _vp]),
    "fclsh_autotune": (_i, [_vp, _vp, _u64, _u32, ctypes.c_char_p, _vp]),
    "fclsh_timing_enable": (_i, [_vp, _i]),
    "fclsh_timing_read": (_i, [_vp, _vp, _vp, _i]),
    "fclsh_server_create": (_i, [_vp, _vp, _vp]),
    "fclsh_server_submit": (_i, [_vp, _vp, _u64, _u32, _vp]),
    "fclsh_server_wait": (_i, [_vp, _u64, _i, _vp, _vp]),
    "fclsh_server_stats": (_i, [_vp, _vp, _i]),
    "fclsh_server_free": (None, [_vp]),
    "fclsh_kernel_launches": (_u64, []),
    "fclsh_save": (_i, [_vp, ctypes.c_char_p]),
    "fclsh_pack_sparse": (_i, [_vp, _vp, _u64, _u64, _u32, _vp, _vp]),
    "fclsh_build_sparse": (_i, [_vp, _vp, _u64, _u64, _u32, _u32, _u64, _vp, _vp]),
    "fclsh_load": (_i, [ctypes.c_char_p, _vp]),
    "fclsh_debug_fail_alloc": (_i, [ctypes.c_int64]),
    "fclsh_debug_pool_used": (_i, [_vp]),
    "fclsh_debug_withhold_hash_loads": (_i, [ctypes.c_int]),
    "fclsh_debug_check_status": (_i, [_vp, _vp]),
    "fclsh_last_error": (ctypes.c_char_p, []),
    "fclsh_version": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfclsh.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st: int):
    if st != OK:
        raise FclshError(st, lib().fclsh_last_error().decode())


def _ptr(a) -> int:
    """Data pointer of a numpy array or torch tensor (must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    raise TypeError(type(a))


def _stream(stream) -> int:
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def _rows(a) -> int:
    return a.shape[0] if len(a.shape) > 1 else 1


@dataclass
class QueryResult:
    offs: np.ndarray        # uint64[nq+1]
    ids: np.ndarray         # uint32[offs[-1]]
    collisions: np.ndarray  # uint64[nq]
    candidates: np.ndarray  # uint64[nq]

    def __len__(self):
        return len(self.offs) - 1

    def of(self, i: int) -> np.ndarray:
        return self.ids[int(self.offs[i]):int(self.offs[i + 1])]


def _take_result(rp: ctypes.POINTER(Result)) -> QueryResult:
    r = rp.contents
    nq = int(r.nq)
    offs = np.ctypeslib.as_array(r.offs, shape=(nq + 1,)).copy()
    total = int(offs[-1])
    ids = np.ctypeslib.as_array(r.ids, shape=(max(total, 1),))[:total].copy()
    coll = np.ctypeslib.as_array(r.collisions, shape=(max(nq, 1),))[:nq].copy()
    cand = np.ctypeslib.as_array(r.candidates, shape=(max(nq, 1),))[:nq].copy()
    lib().fclsh_result_free(rp)
    return QueryResult(offs, ids, coll, cand)


class QueryContext:
    """Per-stream query scratch (fclsh_qctx)."""

    def __init__(self, index: "Index"):
        self.index = index
        h = ctypes.c_void_p()
        _check(lib().fclsh_qctx_create(index.handle, ctypes.byref(h)))
        self.handle = h

    def query_async(self, queries, radius: int, radii=None, stream=None):
        _check(lib().fclsh_query_async(self.handle, _ptr(queries), _rows(queries), radius, _ptr(radii), _stream(stream)))

    def wait(self) -> DeviceResult:
        dr = DeviceResult()
        _check(lib().fclsh_qctx_wait(self.handle, ctypes.byref(dr)))
        return dr

    def fetch(self) -> QueryResult:
        rp = ctypes.POINTER(Result)()
        _check(lib().fclsh_qctx_fetch(self.handle, ctypes.byref(rp)))
        return _take_result(rp)

    def close(self):
        if self.handle:
            lib().fclsh_qctx_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Index:
    """An fcLSH index on the current CUDA device (fclsh_index)."""

    def __init__(self, handle):
        self.handle = handle
        info = Info()
        _check(lib().fclsh_get_info(handle, ctypes.byref(info)))
        self.info = {f: int(getattr(info, f)) for f, _ in Info._fields_}
        for k, v in self.info.items():
            setattr(self, k, v)

    # -- checkpoint
    def save(self, path: str) -> None:
        """fclsh_save: parameters, tuning and points to `path` (load() rebuilds the tables)."""
        _check(lib().fclsh_save(self.handle, os.fsencode(path)))

    # -- parameters / diagnostics
    def params(self):
        """(perm, part_off, m, b) over the D = d * rep positions of the (replicated) vector."""
        D, t = self.d * self.rep, self.t
        perm = np.zeros(D, np.uint32)
        part_off = np.zeros(t + 1, np.uint32)
        m = np.zeros(D, np.uint32)
        b = np.zeros(D, np.uint64)
        _check(lib().fclsh_get_params(self.handle, _ptr(perm), _ptr(part_off), _ptr(m), _ptr(b)))
        return perm, part_off, m, b

    def classic_params(self):
        """(samples [T][k], b [k]) of a classic LSH index."""
        k = ctypes.c_uint32()
        _check(lib().fclsh_get_classic_params(self.handle, ctypes.byref(k), None, None))
        samples = np.zeros((self.T, int(k.value)), np.uint32)
        b = np.zeros(int(k.value), np.uint64)
        _check(lib().fclsh_get_classic_params(self.handle, ctypes.byref(k), _ptr(samples), _ptr(b)))
        return samples, b

    def hash(self, pts, out=None, stream=None):
        """Keys [T][cnt] of the given points (numpy in -> numpy out unless `out` is given)."""
        cnt = _rows(pts)
        if out is None:
            out = np.zeros((self.T, cnt), np.uint64)
        _check(lib().fclsh_hash(self.handle, _ptr(pts), cnt, _ptr(out), _stream(stream)))
        return out

    def bucket(self, table: int, key: int) -> np.ndarray:
        cnt = ctypes.c_uint64()
        _check(lib().fclsh_bucket(self.handle, table, key, None, 0, ctypes.byref(cnt)))
        ids = np.zeros(max(int(cnt.value), 1), np.uint32)
        _check(lib().fclsh_bucket(self.handle, table, key, _ptr(ids), ids.shape[0], ctypes.byref(cnt)))
        return ids[:int(cnt.value)]

    def export_table(self, table: int):
        keys = np.zeros(self.n, np.uint64)
        ids = np.zeros(self.n, np.uint32)
        _check(lib().fclsh_export_table(self.handle, table, _ptr(keys), _ptr(ids)))
        return keys, ids

    def export_keys(self, ids) -> np.ndarray:
        """Keys [T][len(ids)] the build stored for the given point ids, read back from the tables."""
        ids = np.ascontiguousarray(ids, np.uint32)
        out = np.zeros((self.T, ids.shape[0]), np.uint64)
        _check(lib().fclsh_export_keys(self.handle, _ptr(ids), ids.shape[0], _ptr(out)))
        return out

    # -- queries
    def query(self, queries, radius: int, radii=None, stream=None) -> QueryResult:
        rp = ctypes.POINTER(Result)()
        _check(lib().fclsh_query(self.handle, _ptr(queries), _rows(queries), radius, _ptr(radii), _stream(stream),
                                 ctypes.byref(rp)))
        return _take_result(rp)

    def query_plain(self, queries, radius: int, stream=None) -> QueryResult:
        rp = ctypes.POINTER(Result)()
        _check(lib().fclsh_query_plain(self.handle, _ptr(queries), _rows(queries), radius, _stream(stream),
                                       ctypes.byref(rp)))
        return _take_result(rp)

    def query_plain_noalloc(self, query, radius: int, ids_out, counts_out, stream=None):
        """One query without allocating (device query, device outputs); asynchronous on `stream`.

        query: CUDA tensor of at least `words` 64-bit words; ids_out: CUDA int32/uint32 tensor
        (its length is the capacity); counts_out: CUDA int64 tensor of at least 3 elements."""
        def bad(why):
            raise FclshError(EINVAL, "query_plain_noalloc: " + why)

        for name, a in (("query", query), ("ids_out", ids_out), ("counts_out", counts_out)):
            if not getattr(a, "is_cuda", False):
                bad("%s must be a CUDA tensor" % name)
            if not a.is_contiguous():
                bad("%s must be contiguous" % name)
        if query.numel() * query.element_size() < 8 * self.words:
            bad("query holds fewer than %d 64-bit words" % self.words)
        if str(ids_out.dtype) not in ("torch.int32", "torch.uint32"):
            bad("ids_out must be int32 or uint32 (got %s)" % ids_out.dtype)
        if str(counts_out.dtype) != "torch.int64" or counts_out.numel() < 3:
            bad("counts_out must be int64 with at least 3 elements")
        _check(lib().fclsh_query_plain_noalloc(self.handle, _ptr(query), radius, _ptr(ids_out), ids_out.numel(),
                                               _ptr(counts_out), _stream(stream)))

    def bruteforce(self, queries, radius: int, stream=None) -> QueryResult:
        rp = ctypes.POINTER(Result)()
        _check(lib().fclsh_bruteforce(self.handle, _ptr(queries), _rows(queries), radius, _stream(stream),
                                      ctypes.byref(rp)))
        return _take_result(rp)

    def context(self) -> QueryContext:
        return QueryContext(self)

    # -- tuning / timing
    def tuning(self) -> dict:
        t = Tuning()
        _check(lib().fclsh_get_tuning(self.handle, ctypes.byref(t)))
        return t.as_dict()

    def set_tuning(self, **kw):
        t = Tuning()
        _check(lib().fclsh_get_tuning(self.handle, ctypes.byref(t)))
        for k, v in kw.items():
            setattr(t, k, v)
        _check(lib().fclsh_set_tuning(self.handle, ctypes.byref(t)))

    def autotune(self, queries, radius: int, cache_path: str | None = None) -> dict:
        t = Tuning()
        _check(lib().fclsh_autotune(self.handle, _ptr(queries), _rows(queries), radius,
                                    cache_path.encode() if cache_path else None, ctypes.byref(t)))
        return t.as_dict()

    def timing_enable(self, on: bool = True):
        _check(lib().fclsh_timing_enable(self.handle, 1 if on else 0))

    def timing_read(self, reset: bool = False):
        ms = (ctypes.c_double * 9)()
        cnt = (ctypes.c_uint64 * 9)()
        _check(lib().fclsh_timing_read(self.handle, ms, cnt, 1 if reset else 0))
        names = ["build_hash", "build_sort", "query_kernel", "query_csr", "hash", "build_partition", "build_finish",
                 "build_partition_hist", "query_heavy"]
        return {nm: (float(ms[i]), int(cnt[i])) for i, nm in enumerate(names)}

    def free(self):
        if self.handle:
            lib().fclsh_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """Continuous-batching request server over a resident index (fclsh_server)."""

    def __init__(self, index: "Index", slots: int = 4, max_batch_queries: int = 16384, mem_reserve: int = 0):
        self.index = index
        o = ServerOpts(slots, max_batch_queries, mem_reserve)
        h = ctypes.c_void_p()
        _check(lib().fclsh_server_create(index.handle, ctypes.byref(o), ctypes.byref(h)))
        self.handle = h

    def submit(self, queries: np.ndarray, radius: int) -> int:
        q = np.ascontiguousarray(queries, dtype=np.uint64)
        t = ctypes.c_uint64()
        _check(lib().fclsh_server_submit(self.handle, _ptr(q), _rows(q), radius, ctypes.byref(t)))
        return int(t.value)

    def wait(self, ticket: int, timeout_ms: int = -1):
        rp = ctypes.POINTER(Result)()
        lat = ctypes.c_double()
        _check(lib().fclsh_server_wait(self.handle, ticket, timeout_ms, ctypes.byref(rp), ctypes.byref(lat)))
        return _take_result(rp), float(lat.value)

    def stats(self, reset: bool = False) -> dict:
        s = ServerStats()
        _check(lib().fclsh_server_stats(self.handle, ctypes.byref(s), 1 if reset else 0))
        return {f: (float(getattr(s, f)) if t is ctypes.c_double else int(getattr(s, f))) for f, t in ServerStats._fields_}

    def close(self):
        if self.handle:
            lib().fclsh_server_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build(points, d: int, r: int, seed: int, t: int | None = None, slot_bits: int | None = None,
          mem_budget: int | None = None, perm=None, part_off=None, m=None, b=None, timing: bool = False,
          hash_tile: int = 0, replicate: int = 0, approx_c: float = 0.0, classic_tables: int = 0,
          classic_k: int = 0, classic_delta: float = 0.0) -> Index:
    """fclsh_build on host (numpy) or device (torch CUDA) points [n][ceil(d/64)] uint64.

    hash_tile selects the hash kernel (0 default WHT tile, 1 twice as many points, 2 the
    tensor-core contraction, 3 the scatter sketch over set bits, 4 the direct O(dL) route on
    CUDA cores); fclsh_autotune reports the fastest of 0..3 as tuning()["hash_tile"], and a
    build whose column lists do not fit takes 3.
    replicate repeats every vector that many times (Algorithm 1, cr < log n); approx_c > 0
    with neither t nor replicate set chooses both by Algorithm 1.
    classic_k > 0 or classic_delta > 0 builds classic bit-sampling LSH instead (the paper's
    baseline with false negatives): classic_tables tables (0 = the covering table count) of
    classic_k sampled coordinates (0 = the rule of Sec. 4.1 for classic_delta)."""
    keep = []
    o = _build_opts(t=t, slot_bits=slot_bits, mem_budget=mem_budget, perm=perm, part_off=part_off, m=m, b=b,
                    timing=timing, hash_tile=hash_tile, replicate=replicate, approx_c=approx_c, keep=keep,
                    classic_tables=classic_tables, classic_k=classic_k, classic_delta=classic_delta)
    h = ctypes.c_void_p()
    _check(lib().fclsh_build(_ptr(points), _rows(points), d, r, seed, ctypes.byref(o), ctypes.byref(h)))
    return Index(h)


def derive_params(n: int, d: int, r: int, seed: int, t: int | None = None, replicate: int = 0,
                  approx_c: float = 0.0) -> dict:
    """fclsh_derive_params: the shape (t, rep, W) and the random choices (perm, part_off, m, b over
    the D = d * rep positions) that fclsh_build would use for n points, computed on the host."""
    o = _build_opts(t=t, replicate=replicate, approx_c=approx_c)
    shape = np.zeros(3, np.uint32)
    _check(lib().fclsh_derive_params(n, d, r, seed, ctypes.byref(o), _ptr(shape), None, None, None, None))
    t_, rep, W = (int(v) for v in shape)
    perm = np.zeros(d * rep, np.uint32)
    part_off = np.zeros(t_ + 1, np.uint32)
    m = np.zeros(d * rep, np.uint32)
    b = np.zeros(d * rep, np.uint64)
    _check(lib().fclsh_derive_params(n, d, r, seed, ctypes.byref(o), _ptr(shape), _ptr(perm), _ptr(part_off),
                                     _ptr(m), _ptr(b)))
    return {"t": t_, "rep": rep, "W": W, "perm": perm, "part_off": part_off, "m": m, "b": b}


def _build_opts(t=None, slot_bits=None, mem_budget=None, perm=None, part_off=None, m=None, b=None,
                timing=False, hash_tile=0, replicate=0, approx_c=0.0, keep=None, classic_tables=0, classic_k=0,
                classic_delta=0.0) -> BuildOpts:
    o = BuildOpts()
    o.classic_tables = classic_tables or 0
    o.classic_k = classic_k or 0
    o.classic_delta = float(classic_delta)
    o.t = t or 0
    o.replicate = replicate or 0
    o.approx_c = float(approx_c)
    o.slot_bits = slot_bits or 0
    o.mem_budget = mem_budget or 0
    o.timing = 1 if timing else 0
    o.hash_tile = hash_tile
    if perm is not None:
        arrs = [np.ascontiguousarray(perm, np.uint32), np.ascontiguousarray(part_off, np.uint32),
                np.ascontiguousarray(m, np.uint32), np.ascontiguousarray(b, np.uint64)]
        if keep is not None:
            keep += arrs
        o.perm, o.part_off, o.m, o.b = (a.ctypes.data for a in arrs)
    return o


def debug_fail_alloc(after: int) -> None:
    """Make the after-th device allocation of the library fail as out of memory (< 0: off)."""
    _check(lib().fclsh_debug_fail_alloc(after))


def debug_withhold_hash_loads(on, chunk: int = 0) -> None:
    """Make the tensor-core hash kernel's bounded waits run out (tests of ETIMEOUT): while on,
    its operand chunk `chunk` is never requested (chunk 0: before any MMA is issued)."""
    _check(lib().fclsh_debug_withhold_hash_loads(chunk + 1 if on else 0))


def debug_check_status():
    """(checked build?, the first failed bounds check's code since the last call, 0 if none)."""
    checked = ctypes.c_int()
    first = ctypes.c_uint32()
    _check(lib().fclsh_debug_check_status(ctypes.byref(checked), ctypes.byref(first)))
    return bool(checked.value), int(first.value)


def debug_pool_used() -> int:
    """Bytes of the library's device memory pool in use (after a device synchronisation)."""
    v = ctypes.c_uint64()
    _check(lib().fclsh_debug_pool_used(ctypes.byref(v)))
    return int(v.value)


def pack_sparse(indptr, indices, d: int, out=None, stream=None):
    """fclsh_pack_sparse: CSR rows (numpy or torch CUDA) -> bit vectors [n][ceil(d/64)] uint64
    (numpy unless `out` is given)."""
    n = int(indptr.shape[0]) - 1
    nnz = int(indices.shape[0])
    if out is None:
        out = np.zeros((max(n, 0), (d + 63) // 64), np.uint64)
    _check(lib().fclsh_pack_sparse(_ptr(indptr), _ptr(indices), max(n, 0), nnz, d, _ptr(out), _stream(stream)))
    return out


def build_sparse(indptr, indices, d: int, r: int, seed: int, **kw) -> Index:
    """fclsh_build_sparse: an index of CSR rows (indptr [n+1] uint64, indices [nnz] uint32);
    keyword options as for build() (t, replicate, approx_c, slot_bits, hash_tile, timing)."""
    keep = []
    o = _build_opts(keep=keep, **kw)
    h = ctypes.c_void_p()
    n = int(indptr.shape[0]) - 1
    _check(lib().fclsh_build_sparse(_ptr(indptr), _ptr(indices), n, int(indices.shape[0]), d, r, seed,
                                    ctypes.byref(o), ctypes.byref(h)))
    return Index(h)


def load(path: str) -> Index:
    """fclsh_load: rebuild an index saved by Index.save on the current device."""
    h = ctypes.c_void_p()
    _check(lib().fclsh_load(os.fsencode(path), ctypes.byref(h)))
    return Index(h)


def kernel_launches() -> int:
    """Kernels the library has enqueued in this process."""
    return int(lib().fclsh_kernel_launches())


def version() -> str:
    return lib().fclsh_version().decode()
