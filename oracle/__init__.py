"""Plain CPU oracle for Fast CoveringLSH (Pham & Pagh, arXiv 1602.02620).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library and never calls it.

The arithmetic lives in ``fclsh_oracle.c`` (plain C, compiled here with gcc on
first use); this module only marshals numpy arrays:

* ``derive_params``  -- the random choices of Algorithm 1 (permutation, parts)
  and Algorithm 2 (prime P, seed vector b, map or permutation m).
* ``keys_direct``    -- keys from the covering definition (Eq. 2/4) hashed by
  Eq. (1), the O(dL) way.
* ``keys_fht``       -- the same keys by Algorithm 2 (sketch + fast Hadamard
  transform); Lemma 3 says the two agree for every b and P.
* ``build_tables`` / ``query`` -- bucket tables and the Strategy 2 query with the
  S1/S2/S3 steps of Sec. 4.1, including #Collisions and #Candidates;
  ``query_listed`` runs the same query given only the tables it probes.
* ``linear_scan``    -- the plain definition of the answer (Definition 2).
* ``classic_*``      -- classic bit-sampling LSH (Sec. 2.2), the baseline with false
  negatives that the paper compares against (Sec. 4.1): parameters, keys, query.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fclsh_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

#: The prime of Eq. (1).  The paper only asks for a prime larger than n^2
#: (Sec. 2.2); 2^50 - 27 is the largest prime below 2^50.
P_DEFAULT = (1 << 50) - 27

_lib_handle = None


def build(force: bool = False) -> str:
    """Compile the oracle's C source into ``_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [
        ("P", ctypes.c_uint64),
        ("d", ctypes.c_uint32),
        ("t", ctypes.c_uint32),
        ("W", ctypes.c_uint32),
        ("words", ctypes.c_uint32),
        ("perm", ctypes.c_void_p),
        ("part_off", ctypes.c_void_p),
        ("m", ctypes.c_void_p),
        ("b", ctypes.c_void_p),
    ]


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        u64, u32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
        lib.oracle_derive_params.argtypes = [u64, u32, u32, u32, u32, u64, vp, vp, vp, vp]
        lib.oracle_derive_params.restype = ctypes.c_int
        lib.oracle_key_direct.argtypes = [vp, vp, u32]
        lib.oracle_key_direct.restype = u64
        lib.oracle_keys_direct.argtypes = [vp, vp, u64, vp]
        lib.oracle_keys_direct.restype = None
        lib.oracle_keys_fht.argtypes = [vp, vp, u64, vp]
        lib.oracle_keys_fht.restype = None
        lib.oracle_table.argtypes = [vp, vp, u64, u32, vp, vp]
        lib.oracle_table.restype = None
        lib.oracle_query.argtypes = [vp, vp, u64, vp, vp, vp, u32, vp, u64, vp]
        lib.oracle_query.restype = u64
        lib.oracle_query_rows.argtypes = [vp, vp, u64, vp, vp, vp, u32, u32, vp, u64, vp]
        lib.oracle_query_rows.restype = u64
        lib.oracle_query_listed.argtypes = [vp, vp, u64, vp, vp, vp, vp, u32, u32, vp, u64, vp]
        lib.oracle_query_listed.restype = u64
        lib.oracle_linear_scan.argtypes = [vp, u64, u32, vp, u32, vp, u64]
        lib.oracle_linear_scan.restype = u64
        lib.oracle_splitmix64.argtypes = [u64, u64, vp]
        lib.oracle_splitmix64.restype = None
        lib.oracle_hamming.argtypes = [vp, vp, u32]
        lib.oracle_hamming.restype = ctypes.c_int
        _lib_handle = lib
    return _lib_handle


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def default_parts(r: int) -> int:
    """Number of parts t for build radius r.

    The paper's experimental setting (Sec. 4.4): one part for r < 10 and two
    parts for r >= 10 (it goes up to r = 20).  Beyond that the rule keeps the
    per-part radius floor(r/t) at most 10 by taking the smallest such t.
    """
    if r < 10:
        return 1
    t = 2
    while r // t > 10:
        t += 1
    return t


@dataclass
class Params:
    """All choices that define one index (names follow the paper)."""

    P: int
    d: int
    r: int          # build radius
    t: int          # parts (Algorithm 1)
    rp: int         # per-part radius r' = floor(r * rep / t)
    W: int          # code length 2^(r'+1)
    perm: np.ndarray      # uint32[D]: position i of the pre-processed vector holds coordinate perm[i]
    part_off: np.ndarray  # uint32[t+1]
    m: np.ndarray         # uint32[D]: code column of position i
    b: np.ndarray         # uint64[D]: seed-vector entry of position i
    rep: int = 1          # replication factor of Algorithm 1 (D = d * rep positions)

    @property
    def words(self) -> int:
        return (self.d + 63) // 64

    @property
    def L(self) -> int:
        """Tables per part, 2^(r'+1) - 1."""
        return self.W - 1

    @property
    def T(self) -> int:
        """Total tables t * (2^(r'+1) - 1)."""
        return self.t * (self.W - 1)

    def _c(self) -> _Params:
        for a, dt in ((self.perm, np.uint32), (self.part_off, np.uint32), (self.m, np.uint32), (self.b, np.uint64)):
            assert a.dtype == dt and a.flags.c_contiguous
        return _Params(self.P, self.d, self.t, self.W, self.words,
                       _ptr(self.perm), _ptr(self.part_off), _ptr(self.m), _ptr(self.b))


def derive_params(seed: int, d: int, r: int, t: int | None = None, P: int = P_DEFAULT, rep: int = 1) -> Params:
    """Draw the index's random choices from ``seed`` (see fclsh_oracle.c for the order).

    rep > 1 replicates every vector rep times first (Algorithm 1 for cr < log n); the
    index then covers radius r * rep of the replicated vectors."""
    if t is None:
        t = 1 if rep > 1 else default_parts(r)
    rp = r * rep // t
    W = 2 << rp
    D = d * rep
    perm = np.zeros(D, np.uint32)
    part_off = np.zeros(t + 1, np.uint32)
    m = np.zeros(D, np.uint32)
    b = np.zeros(D, np.uint64)
    rc = _lib().oracle_derive_params(seed, d, t, rep, W, P, _ptr(perm), _ptr(part_off), _ptr(m), _ptr(b))
    if rc != 0:
        raise ValueError("bad parameters d=%d r=%d t=%d rep=%d" % (d, r, t, rep))
    return Params(P, d, r, t, rp, W, perm, part_off, m, b, rep)


def make_params(d: int, r: int, m, b, P: int = P_DEFAULT, t: int = 1, perm=None, part_off=None,
                rep: int = 1) -> Params:
    """Explicit parameters (e.g. the worked examples of Sec. 2.3 and 3.1); m and b have
    d * rep entries, and without a perm position i reads coordinate i mod d."""
    rp = r * rep // t
    W = 2 << rp
    D = d * rep
    perm = (np.arange(D, dtype=np.uint32) % d) if perm is None else np.ascontiguousarray(perm, np.uint32)
    if part_off is None:
        blk = D // t
        part_off = [k * blk for k in range(t)] + [D]
    return Params(P, d, r, t, rp, W, perm, np.ascontiguousarray(part_off, np.uint32),
                  np.ascontiguousarray(m, np.uint32), np.ascontiguousarray(b, np.uint64), rep)


def _pts(pts, words: int) -> np.ndarray:
    a = np.ascontiguousarray(pts, dtype=np.uint64)
    if a.ndim == 1:
        a = a.reshape(-1, words)
    assert a.shape[1] == words
    return a


def key_direct(p: Params, x, tau: int) -> int:
    x = _pts(x, p.words)
    return int(_lib().oracle_key_direct(ctypes.byref(p._c()), _ptr(x), tau))


def keys_direct(p: Params, pts) -> np.ndarray:
    """uint64[T][n] keys by the covering definition and Eq. (1)."""
    pts = _pts(pts, p.words)
    out = np.zeros((p.T, pts.shape[0]), np.uint64)
    _lib().oracle_keys_direct(ctypes.byref(p._c()), _ptr(pts), pts.shape[0], _ptr(out))
    return out


def keys_fht(p: Params, pts) -> np.ndarray:
    """uint64[T][n] keys by Algorithm 2 (sketch + fast Hadamard transform)."""
    pts = _pts(pts, p.words)
    out = np.zeros((p.T, pts.shape[0]), np.uint64)
    _lib().oracle_keys_fht(ctypes.byref(p._c()), _ptr(pts), pts.shape[0], _ptr(out))
    return out


def table(p: Params, pts, tau: int):
    """(keys, ids) of table tau sorted by (key, id)."""
    pts = _pts(pts, p.words)
    n = pts.shape[0]
    keys = np.zeros(n, np.uint64)
    ids = np.zeros(n, np.uint32)
    _lib().oracle_table(ctypes.byref(p._c()), _ptr(pts), n, tau, _ptr(keys), _ptr(ids))
    return keys, ids


def build_tables(p: Params, pts):
    """All T tables as two [T][n] arrays sorted by (key, id) within each row."""
    pts = _pts(pts, p.words)
    n = pts.shape[0]
    keys = np.zeros((p.T, n), np.uint64)
    ids = np.zeros((p.T, n), np.uint32)
    for tau in range(p.T):
        keys[tau], ids[tau] = table(p, pts, tau)
    return keys, ids


def query(p: Params, pts, tables, q, radius: int, rows: int = 0):
    """Strategy 2 query.  Returns (sorted ids, #Collisions, #Candidates).

    rows = 0 probes every table; rows > 0 probes only the code rows v = 1..rows of
    each part (see probe_rows()), and the counters count those tables only.
    """
    pts = _pts(pts, p.words)
    q = _pts(q, p.words)
    keys, ids = tables
    n = pts.shape[0]
    cap = max(n, 1)
    out = np.zeros(cap, np.uint32)
    counters = np.zeros(2, np.uint64)
    cnt = _lib().oracle_query_rows(ctypes.byref(p._c()), _ptr(pts), n, _ptr(keys), _ptr(ids),
                                   _ptr(q), radius, rows, _ptr(out), cap, _ptr(counters))
    return out[:cnt].copy(), int(counters[0]), int(counters[1])


def probed_tables(p: Params, rows: int) -> list:
    """Tables a query probes with ``rows`` code rows per part (0 = all T)."""
    L = p.W - 1
    if rows == 0 or rows >= L:
        return list(range(p.T))
    return [k * L + v - 1 for k in range(p.t) for v in range(1, rows + 1)]


def query_listed(p: Params, pts, tables: dict, q, radius: int, rows: int = 0):
    """Strategy 2 query like ``query`` with only some tables given: ``tables`` maps a
    table index to its (keys, ids) from ``table``; every probed table must be present.
    Returns (sorted ids, #Collisions, #Candidates)."""
    pts = _pts(pts, p.words)
    q = _pts(q, p.words)
    n = pts.shape[0]
    taus = sorted(tables)
    missing = set(probed_tables(p, rows)) - set(taus)
    if missing:
        raise ValueError("probed tables not given: %s" % sorted(missing)[:8])
    keys = np.stack([np.ascontiguousarray(tables[t][0], np.uint64) for t in taus])
    ids = np.stack([np.ascontiguousarray(tables[t][1], np.uint32) for t in taus])
    row = np.full(p.T, 0xFFFFFFFF, np.uint32)
    row[taus] = np.arange(len(taus), dtype=np.uint32)
    cap = max(n, 1)
    out = np.zeros(cap, np.uint32)
    counters = np.zeros(2, np.uint64)
    cnt = _lib().oracle_query_listed(ctypes.byref(p._c()), _ptr(pts), n, _ptr(keys), _ptr(ids), _ptr(row),
                                     _ptr(q), radius, rows, _ptr(out), cap, _ptr(counters))
    if cnt == (1 << 64) - 1:
        raise ValueError("a probed table was not given")
    return out[:cnt].copy(), int(counters[0]), int(counters[1])


def probe_rows(p: Params, radius: int) -> int:
    """Code rows per part that a query of this radius must probe: 2^(floor(radius*rep/t)+1) - 1,
    at most W - 1 (pigeonhole over the t parts, or distance radius*rep between the replicated
    vectors, then Theorem 1 on the map m mod 2^(floor(radius*rep/t)+1))."""
    e = radius * p.rep // p.t + 1
    return min(p.W - 1, (1 << e) - 1) if e < 63 else p.W - 1


def linear_scan(pts, q, radius: int, words: int | None = None) -> np.ndarray:
    """Every id within Hamming distance ``radius`` of q, ascending (Definition 2)."""
    q = np.ascontiguousarray(q, dtype=np.uint64).reshape(-1)
    words = q.shape[0] if words is None else words
    pts = _pts(pts, words)
    n = pts.shape[0]
    cap = max(n, 1)
    out = np.zeros(cap, np.uint32)
    cnt = _lib().oracle_linear_scan(_ptr(pts), n, words, _ptr(q), radius, _ptr(out), cap)
    return out[:cnt].copy()


# ---------------------------------------------------------------- classic bit-sampling LSH

def classic_rule_k(L: int, r: int, d: int, delta: float) -> int:
    """Bit samples per table of classic LSH by the rule of Sec. 4.1:
    k = ceil(log(1 - delta^(1/L)) / log(1 - r/d)) -- the k at which a point at distance r
    escapes all L tables with probability about delta."""
    import math

    return max(1, math.ceil(math.log1p(-(delta ** (1.0 / L))) / math.log1p(-r / d)))


@dataclass
class ClassicParams:
    """Classic LSH (Sec. 2.2): table j samples coordinates samples[j] (k of them, with
    replacement); its key is Eq. 1 on the sampled bits with the seed vector b."""

    P: int
    d: int
    samples: np.ndarray   # uint32[L][k]
    b: np.ndarray         # uint64[k]

    @property
    def L(self) -> int:
        return self.samples.shape[0]


def classic_params(seed: int, d: int, L: int, k: int, P: int = P_DEFAULT) -> ClassicParams:
    """Draws from SplitMix64 started at seed: every table's k samples next() mod d, table by
    table, then the k entries of b uniform below P (the top bits of a draw, rejected if >= P)."""
    bits = (P - 1).bit_length()
    need = L * k + k + 64
    out = splitmix64(seed, need)
    samples = (out[: L * k] % np.uint64(d)).astype(np.uint32).reshape(L, k)
    b, at = [], L * k
    while len(b) < k:
        if at == len(out):
            out = splitmix64(seed, 2 * len(out))
        u = int(out[at]) >> (64 - bits)
        at += 1
        if u < P:
            b.append(u)
    return ClassicParams(P, d, samples, np.array(b, np.uint64))


def _bits(pts, d: int) -> np.ndarray:
    a = np.ascontiguousarray(pts, dtype=np.uint64)
    a = a.reshape(-1, (d + 63) // 64)
    return np.unpackbits(a.view(np.uint8).reshape(a.shape[0], -1), axis=1, bitorder="little")[:, :d]


def classic_keys(cp: ClassicParams, pts) -> np.ndarray:
    """uint64[L][n]: key_j(x) = (sum_i b_i x_{samples[j][i]}) mod P (Eq. 1 on the sampled bits;
    the sum of k < 2^13 values below 2^50 is exact in 64 bits)."""
    assert cp.samples.shape[1] < (1 << 13)
    x = _bits(pts, cp.d).astype(np.uint64)
    keys = np.zeros((cp.L, x.shape[0]), np.uint64)
    for j in range(cp.L):
        keys[j] = (x[:, cp.samples[j]] @ cp.b) % np.uint64(cp.P)
    return keys


def classic_query(cp: ClassicParams, pts, keys: np.ndarray, q, radius: int):
    """Strategy 2 over the classic tables (Sec. 2.2): the points whose key equals the query's
    in some table are the candidates; those within `radius` are reported.  Returns (sorted ids,
    #Collisions, #Candidates) as the covering query does."""
    qk = classic_keys(cp, q)[:, 0]
    hit = keys == qk[:, None]
    cand = hit.any(axis=0)
    x = _bits(pts, cp.d)
    dist = (x != _bits(q, cp.d)[0]).sum(axis=1)
    ids = np.nonzero(cand & (dist <= radius))[0].astype(np.uint32)
    return ids, int(hit.sum()), int(cand.sum())


def hamming(a, b) -> int:
    a = np.ascontiguousarray(a, dtype=np.uint64).reshape(-1)
    b = np.ascontiguousarray(b, dtype=np.uint64).reshape(-1)
    return int(_lib().oracle_hamming(_ptr(a), _ptr(b), a.shape[0]))


def splitmix64(seed: int, n: int) -> np.ndarray:
    """First n outputs of the oracle's SplitMix64 generator started at seed."""
    out = np.zeros(n, np.uint64)
    _lib().oracle_splitmix64(seed, n, _ptr(out))
    return out
