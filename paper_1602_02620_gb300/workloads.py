"""Seeded synthetic workloads shaped like the paper's data (Sec. 4.2, Table 2).

The paper's data sets (ANN_SIFT1M, Webspam, Enron, MovieLens) are not
available, so every input here is synthetic and seeded; the recipes mirror
their shapes: uniform 128-bit image codes (SIFT-like), clustered 256-bit codes
(image-code clusters), and sparse 1024-bit fingerprints with near-duplicates
(text-like).  This module holds none of the index's arithmetic; the C part
(``csrc/workloads.c``) only generates bits.

Eight workloads (sizes as named):

====  ==========  =====  ==  =========  ==========================================
name  n           d      r   queries    data / queries
====  ==========  =====  ==  =========  ==========================================
1     10,000      64     3   200        Bernoulli(1/2); 100 planted at k in 0..3, 100 uniform
2     1,000,000   128    8   10,000     Bernoulli(1/2); 50% planted at k in 0..8, 50% uniform
3     4,000,000   256    16  100,000    4,096 centres, flip p=0.05; queries centre + flip p~U[0.02,0.08]
4     2,000,000   1,024  20  50,000     density 0.02, 20% near-dups at 1..20; 50% near-dup queries, 50% random
5     8,000,000   256    16  stream     as 3; requests of U{1..4096} queries, radius in {4,8,12,16}
6     40,000      28,102 29  1,000      sparse, skewed popularity, ~150 set bits (Enron-like); 10% near-dups
7     234,834     140,214 13 2,000      sparse, skewed popularity, ~85 set bits (MovieLens-like); 10% near-dups
8     1,000,000   128    2   10,000     as 2 with k in 0..2, indexed with 4 copies of each vector (Algorithm 1)
====  ==========  =====  ==  =========  ==========================================
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "workloads.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libfclsh_workloads.so")
_lib_handle = None


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        u64, u32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
        lib.wl_stream_key.argtypes = [u64, u64]
        lib.wl_stream_key.restype = u64
        lib.wl_uniform.argtypes = [u64, u64, u64, u32, vp]
        lib.wl_bernoulli.argtypes = [u64, u64, u64, u32, u32, vp]
        lib.wl_clustered.argtypes = [u64, u64, u64, u64, u64, u32, vp, u32, u32, u32, vp, vp]
        lib.wl_planted.argtypes = [u64, u64, u64, vp, u64, u32, u32, u32, vp, vp, vp]
        lib.wl_near_duplicates.argtypes = [u64, vp, u64, u32, u32, u32, u32]
        lib.wl_near_duplicates.restype = u64
        lib.wl_raw.argtypes = [u64, u64, u64, vp]
        lib.wl_sparse_skewed.argtypes = [u64, u64, u64, u32, u32, u32, vp]
        lib.wl_sparse_skewed.restype = None
        for f in ("wl_uniform", "wl_bernoulli", "wl_clustered", "wl_planted", "wl_raw"):
            getattr(lib, f).restype = None
        _lib_handle = lib
    return _lib_handle


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def thr16(p: float) -> int:
    """16-bit threshold of a Bernoulli(p) bit."""
    return int(round(p * 65536))


# Stream ids (one independent counter-based stream each).
S_DATA, S_CENTRES, S_CHOICE, S_NOISE, S_NOISE_LVL = 1, 2, 3, 4, 5
S_Q_UNIFORM, S_Q_PLANT, S_NEARDUP = 6, 7, 8
S_Q_CHOICE, S_Q_NOISE, S_Q_NOISE_LVL, S_REQUESTS = 9, 10, 11, 12

CONFIGS = {
    1: dict(name="plain-small n=10000 d=64 r=3", n=10_000, d=64, r=3, nq=200, seed=1, kind="uniform", plant=(0, 3)),
    2: dict(name="plain n=1000000 d=128 r=8", n=1_000_000, d=128, r=8, nq=10_000, seed=2, kind="uniform", plant=(0, 8)),
    3: dict(name="batched-clustered n=4000000 d=256 r=16", n=4_000_000, d=256, r=16, nq=100_000, seed=3,
            kind="clustered", centres=4096, p_data=0.05, p_query=(0.02, 0.08)),
    4: dict(name="batched-sparse n=2000000 d=1024 r=20", n=2_000_000, d=1024, r=20, nq=50_000, seed=4,
            kind="sparse", density=0.02, dup_frac=0.2, dup_k=(1, 20), plant=(0, 20)),
    5: dict(name="served-clustered n=8000000 d=256 r=16", n=8_000_000, d=256, r=16, nq=0, seed=5,
            kind="clustered", centres=4096, p_data=0.05, p_query=(0.02, 0.08),
            req_size=(1, 4096), req_radii=(4, 8, 12, 16)),
    # very high-dimensional sparse sets of the shapes of Enron and MovieLens (Table 2)
    6: dict(name="highd-enron n=40000 d=28102 r=29", n=40_000, d=28_102, r=29, nq=1_000, seed=6,
            kind="sparse_skewed", lmin=20, lmean=130, dup_frac=0.1, dup_k=(1, 29), plant=(0, 29)),
    7: dict(name="highd-movielens n=234834 d=140214 r=13", n=234_834, d=140_214, r=13, nq=2_000, seed=7,
            kind="sparse_skewed", lmin=15, lmean=70, dup_frac=0.1, dup_k=(1, 13), plant=(0, 13)),
    # Algorithm 1's replication for a small radius: the bench workload's points at r = 2, four copies
    # (the paper's synthetic setting for r = 2), 511 tables as at r = 8 without replication
    8: dict(name="replicated n=1000000 d=128 r=2 (4 copies)", n=1_000_000, d=128, r=2, nq=10_000, seed=8,
            kind="uniform", plant=(0, 2), build={"replicate": 4}),
}


def build_options(cfg_id: int) -> dict:
    """Index options a workload is defined with (e.g. replication), as keyword arguments."""
    return dict(CONFIGS[cfg_id].get("build", {}))


@dataclass
class Workload:
    cfg: int
    name: str
    n: int
    d: int
    r: int
    seed: int
    points: np.ndarray                     # uint64[n][words]
    queries: np.ndarray                    # uint64[nq][words]
    meta: dict = field(default_factory=dict)

    @property
    def words(self) -> int:
        return (self.d + 63) // 64

    @property
    def index_seed(self) -> int:
        """Seed of the index's random choices: data seed + 1000."""
        return self.seed + 1000


def _key(seed: int, s: int) -> int:
    return int(_lib().wl_stream_key(seed, s))


def centres(cfg: dict) -> np.ndarray:
    d, nc = cfg["d"], cfg["centres"]
    out = np.zeros((nc, (d + 63) // 64), np.uint64)
    _lib().wl_uniform(_key(cfg["seed"], S_CENTRES), 0, nc, d, _p(out))
    return out


def points(cfg_id: int, n: int | None = None) -> np.ndarray:
    """The first n data points of workload cfg_id (prefix-stable)."""
    cfg = CONFIGS[cfg_id]
    n = cfg["n"] if n is None else n
    d, seed = cfg["d"], cfg["seed"]
    words = (d + 63) // 64
    out = np.zeros((n, words), np.uint64)
    lib = _lib()
    if cfg["kind"] == "uniform":
        lib.wl_uniform(_key(seed, S_DATA), 0, n, d, _p(out))
    elif cfg["kind"] == "clustered":
        c = centres(cfg)
        t = thr16(cfg["p_data"])
        lib.wl_clustered(_key(seed, S_CHOICE), _key(seed, S_NOISE), _key(seed, S_NOISE_LVL), 0, n, d,
                         _p(c), c.shape[0], t, t, _p(out), None)
    elif cfg["kind"] == "sparse":
        lib.wl_bernoulli(_key(seed, S_DATA), 0, n, d, thr16(cfg["density"]), _p(out))
        lo, hi = cfg["dup_k"]
        lib.wl_near_duplicates(_key(seed, S_NEARDUP), _p(out), n, d, thr16(cfg["dup_frac"]), lo, hi)
    elif cfg["kind"] == "sparse_skewed":
        lib.wl_sparse_skewed(_key(seed, S_DATA), 0, n, d, cfg["lmin"], cfg["lmean"], _p(out))
        lo, hi = cfg["dup_k"]
        lib.wl_near_duplicates(_key(seed, S_NEARDUP), _p(out), n, d, thr16(cfg["dup_frac"]), lo, hi)
    else:
        raise ValueError(cfg["kind"])
    return out


def queries(cfg_id: int, pts: np.ndarray, nq: int | None = None, first: int = 0):
    """nq queries of workload cfg_id (query indices first..first+nq) and their metadata."""
    cfg = CONFIGS[cfg_id]
    nq = cfg["nq"] if nq is None else nq
    d, seed = cfg["d"], cfg["seed"]
    words = (d + 63) // 64
    out = np.zeros((nq, words), np.uint64)
    meta = {}
    lib = _lib()
    n = pts.shape[0]
    if cfg["kind"] in ("uniform", "sparse", "sparse_skewed"):
        # even global query index -> planted near a data point, odd -> fresh random
        idx = np.arange(first, first + nq)
        planted = (idx % 2) == 0
        src = np.full(nq, 0xFFFFFFFF, np.uint32)
        kk = np.zeros(nq, np.uint32)
        kmin, kmax = cfg["plant"]
        for i in range(nq):
            g = first + i
            if planted[i]:
                s = np.zeros(1, np.uint32)
                k = np.zeros(1, np.uint32)
                lib.wl_planted(_key(seed, S_Q_PLANT), g // 2, 1, _p(pts), n, d, kmin, kmax,
                               _p(out[i:i + 1]), _p(s), _p(k))
                src[i], kk[i] = s[0], k[0]
            elif cfg["kind"] == "uniform":
                lib.wl_uniform(_key(seed, S_Q_UNIFORM), g // 2, 1, d, _p(out[i:i + 1]))
            elif cfg["kind"] == "sparse_skewed":
                lib.wl_sparse_skewed(_key(seed, S_Q_UNIFORM), g // 2, 1, d, cfg["lmin"], cfg["lmean"],
                                     _p(out[i:i + 1]))
            else:
                lib.wl_bernoulli(_key(seed, S_Q_UNIFORM), g // 2, 1, d, thr16(cfg["density"]), _p(out[i:i + 1]))
        meta.update(planted=planted, src=src, k=kk)
    elif cfg["kind"] == "clustered":
        c = centres(cfg)
        lo, hi = cfg["p_query"]
        cid = np.zeros(nq, np.uint32)
        lib.wl_clustered(_key(seed, S_Q_CHOICE), _key(seed, S_Q_NOISE), _key(seed, S_Q_NOISE_LVL), first, nq, d,
                         _p(c), c.shape[0], thr16(lo), thr16(hi), _p(out), _p(cid))
        meta.update(centre=cid)
    return out, meta


def make(cfg_id: int, n: int | None = None, nq: int | None = None) -> Workload:
    cfg = CONFIGS[cfg_id]
    pts = points(cfg_id, n)
    qn = cfg["nq"] if nq is None else nq
    q, meta = queries(cfg_id, pts, qn)
    return Workload(cfg_id, cfg["name"], pts.shape[0], cfg["d"], cfg["r"], cfg["seed"], pts, q, meta)


def request_stream(cfg_id: int, count: int, rate_per_s: float, first: int = 0):
    """Poisson request stream: list of (arrival_s, size, radius) for requests first..first+count.

    Inter-arrival times are exponential with the given rate, sizes uniform in
    the workload's request-size range and radii uniform over its radius set.
    """
    cfg = CONFIGS[cfg_id]
    raw = np.zeros(3 * count, np.uint64)
    _lib().wl_raw(_key(cfg["seed"], S_REQUESTS), 3 * first, 3 * count, _p(raw))
    raw = raw.reshape(count, 3)
    smin, smax = cfg["req_size"]
    radii = cfg["req_radii"]
    out = []
    t = 0.0
    for j in range(count):
        u = (int(raw[j, 0]) >> 11) * (1.0 / (1 << 53))
        t += -math.log(1.0 - u) / rate_per_s
        size = smin + int(raw[j, 1]) % (smax - smin + 1)
        radius = radii[int(raw[j, 2]) % len(radii)]
        out.append((t, size, radius))
    return out
