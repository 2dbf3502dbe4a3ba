"""Build libfclsh.so (CUDA for sm_103a) and the workload generator library in-tree.

Every translation unit is compiled in parallel with nvcc
(``-gencode arch=compute_103a,code=sm_103a -lineinfo -O3``) and linked into
``_build/libfclsh.so``.  Usage: ``python -m paper_1602_02620_gb300.build``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(BUILD, "libfclsh.so")

SOURCES = ["api.cu", "hash.cu", "hash_mma.cu", "sort.cu", "query.cu", "params.cpp", "server.cpp", "noalloc.cu"]
HEADERS = ["common.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _newer(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra=(), build_dir=None) -> str:
    obj = os.path.join(build_dir or BUILD, os.path.basename(src) + ".o")
    deps = [os.path.join(CSRC, src)] + [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "fclsh.h")]
    if _newer(obj, deps):
        cmd = [nvcc()] + NVCC_FLAGS + list(extra) + ["-c", os.path.join(CSRC, src), "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    """Compile (if stale) and link libfclsh.so; returns its path.  checked=True builds the
    bounds-checked variant (-DFCLSH_CHECKED) into _build_checked/."""
    bdir = os.path.join(HERE, "_build_checked") if checked else BUILD
    lib = os.path.join(bdir, "libfclsh.so")
    extra = list(extra) + (["-DFCLSH_CHECKED"] if checked else [])
    os.makedirs(bdir, exist_ok=True)
    if force:
        for f in os.listdir(bdir):
            if f.endswith(".o"):
                os.remove(os.path.join(bdir, f))
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, bdir), SOURCES))
    if _newer(lib, objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-o", lib + ".tmp"] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
        os.replace(lib + ".tmp", lib)
    if verbose:
        print(lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv)
