"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import os
import re

from tests.conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "fclsh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fclsh_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1602_02620_gb300 import build as B
    from paper_1602_02620_gb300 import fclsh

    B.build()
    lib = fclsh.lib()
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(fclsh.SIGNATURES), set(names) ^ set(fclsh.SIGNATURES)
    assert "sm_103a" in fclsh.version()


def test_every_declaration_cites_its_passage():
    """Each entry point's comment in include/fclsh.h names the passage of the paper that
    defines it (section, algorithm, equation, definition, lemma, theorem, strategy, example,
    table) or says that it has no counterpart in the paper."""
    src = open(os.path.join(ROOT, "include", "fclsh.h")).read()
    cite = re.compile(r"Sec\.|Algorithm|Eq\.|Definition|Lemma|Theorem|Strategy|Example|Table|no\s+counterpart",
                      re.I)
    last, missing = None, []
    for m in re.finditer(r"/\*.*?\*/|\b(?:fclsh_status|void|const char \*|uint64_t)\s*\*?\s*(fclsh_[a-z0-9_]+)\s*\(",
                         src, re.S):
        if m.group(0).startswith("/*"):
            last = re.sub(r"\s*\n\s*\*?\s*", " ", m.group(0))
            continue
        if not (last and cite.search(last)):
            missing.append(m.group(1))
    assert not missing, missing


def test_errors_without_touching_the_gpu():
    """Argument checks fail cleanly before any device call."""
    import ctypes
    from paper_1602_02620_gb300 import fclsh

    lib = fclsh.lib()
    h = ctypes.c_void_p()
    assert lib.fclsh_build(None, 10, 64, 3, 1, None, ctypes.byref(h)) == fclsh.EINVAL
    assert b"NULL" in lib.fclsh_last_error()
    assert lib.fclsh_get_info(None, None) == fclsh.EINVAL
    lib.fclsh_free(None)
    lib.fclsh_result_free(None)


def _fnv64(data: bytes) -> int:
    h = 0xCBF29CE484222325
    for c in data:
        h = ((h ^ c) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def _index_file(d=64, r=3, n=5, words=1, checksum_ok=True, version=1):
    """An index file in the documented layout (identity parameters, all-zero points)."""
    import struct

    t, rep, sb, tile, W = 1, 1, 18, 0, 2 << r
    body = b"FCLSHIX1"
    body += struct.pack("<8I", d, r, t, rep, sb, tile, W, version)
    body += struct.pack("<2Q", n, (1 << 50) - 27)
    body += struct.pack("<7I", 256, 4, 12, 4, 1, tile, 0)
    body += struct.pack("<%dI" % d, *range(d))
    body += struct.pack("<2I", 0, d)
    body += struct.pack("<%dI" % d, *[i % W for i in range(d)])
    body += struct.pack("<%dQ" % d, *range(1, d + 1))
    body += bytes(8 * n * words)
    return body + struct.pack("<Q", _fnv64(body) ^ (0 if checksum_ok else 1))


def test_load_rejects_bad_files_without_a_gpu(tmp_path):
    """fclsh_load checks the file (magic, version, sizes, checksum) before any device call."""
    import ctypes
    from paper_1602_02620_gb300 import fclsh

    lib = fclsh.lib()
    h = ctypes.c_void_p()
    missing = str(tmp_path / "missing.idx").encode()
    assert lib.fclsh_load(missing, ctypes.byref(h)) == fclsh.EINVAL
    cases = {
        "magic.idx": b"NOTANIDX" + _index_file()[8:],
        "version.idx": _index_file(version=7),
        "truncated.idx": _index_file()[:100],
        "checksum.idx": _index_file(checksum_ok=False),
    }
    for name, data in cases.items():
        p = tmp_path / name
        p.write_bytes(data)
        assert lib.fclsh_load(str(p).encode(), ctypes.byref(h)) == fclsh.EINVAL, name
        assert not h.value
    good = tmp_path / "good.idx"
    good.write_bytes(_index_file())
    st = lib.fclsh_load(str(good).encode(), ctypes.byref(h))
    import torch

    if not torch.cuda.is_available():   # the file passes every check; the rebuild needs a device
        assert st == fclsh.ECUDA, lib.fclsh_last_error()
    else:
        assert st == fclsh.OK
        lib.fclsh_free(h)


def test_sparse_argument_errors_without_a_gpu():
    import ctypes
    from paper_1602_02620_gb300 import fclsh

    lib = fclsh.lib()
    h = ctypes.c_void_p()
    assert lib.fclsh_pack_sparse(None, None, 3, 0, 64, None, None) == fclsh.EINVAL      # NULL rows
    buf = (ctypes.c_uint64 * 4)()
    assert lib.fclsh_pack_sparse(buf, buf, 1, 0, 0, buf, None) == fclsh.EINVAL           # d = 0
    assert lib.fclsh_build_sparse(buf, buf, 0, 0, 64, 3, 1, None, ctypes.byref(h)) == fclsh.EINVAL   # n = 0
    assert lib.fclsh_build_sparse(buf, buf, 1, 0, 300_000, 3, 1, None, ctypes.byref(h)) == fclsh.EINVAL


def _algorithm1_rule(n, r, c):
    """The reading of Algorithm 1's rule the library states (log = log2; copies capped at
    floor(10 / r); parts raised until floor(r / t) <= 10), written out for the test."""
    import math

    if r == 0:
        return 1, 1
    lg = math.log2(max(n, 2))
    rep, parts = 1, 1
    if c * r < lg:
        rep = max(1, min(math.floor(lg / (c * r)), 10 // r))
    elif c * r > lg:
        parts = math.ceil(c * r / lg)
    if rep > 1:
        return 1, rep
    while r // parts > 10:
        parts += 1
    return parts, 1


def test_host_parameters_match_the_oracle_without_a_gpu():
    """fclsh_derive_params, the host half of fclsh_build, draws the same shape, permutation,
    parts, map and seed vector as the oracle's independent derivation."""
    import numpy as np

    import oracle
    from paper_1602_02620_gb300 import fclsh

    cases = [(64, 3, None, 0), (128, 8, None, 0), (256, 16, None, 0), (1024, 20, None, 0), (300, 7, 3, 0),
             (100, 2, 1, 3), (17, 4, None, 2), (28_102, 29, None, 0), (140_214, 13, None, 0), (96, 32, None, 0),
             (5, 0, None, 0), (70, 6, None, 0), (128, 2, None, 4)]
    for i, (d, r, t, rep) in enumerate(cases):
        seed = 1000 + 7 * i
        got = fclsh.derive_params(10_000, d, r, seed, t=t, replicate=rep)
        want = oracle.derive_params(seed, d, r, t=t, rep=rep or 1)
        assert (got["t"], got["rep"], got["W"]) == (want.t, want.rep, want.W), (d, r, t, rep)
        for k in ("perm", "part_off", "m", "b"):
            assert np.array_equal(got[k], getattr(want, k)), (d, r, t, rep, k)


def test_algorithm1_rule_and_rejections_without_a_gpu():
    """approx_c picks copies or parts by the stated rule; the shapes fclsh_build rejects on the
    host are rejected the same way by fclsh_derive_params, and accepted ones pass both."""
    import ctypes

    import numpy as np
    import torch

    from paper_1602_02620_gb300 import fclsh

    for n in (1_000, 1_000_000, 100_000_000):
        for r in (0, 1, 2, 3, 5, 8, 13, 20, 40):
            for c in (0.5, 1.0, 1.5, 2.0, 3.0):
                got = fclsh.derive_params(n, 256, r, 1, approx_c=c)
                assert (got["t"], got["rep"]) == _algorithm1_rule(n, r, c), (n, r, c)
    lib = fclsh.lib()
    pts = np.zeros(64, np.uint64)
    h = ctypes.c_void_p()
    shape = np.zeros(3, np.uint32)
    for d, r, kw, ok in [(64, 3, {}, True), (64, 3, {"t": 2, "replicate": 2}, False), (8, 3, {"t": 9}, False),
                         (256, 25, {"t": 2}, False), (64, 2, {"replicate": 33}, False), (64, 11, {"t": 1}, False),
                         (64, 3, {"approx_c": -1.0}, False), (0, 3, {}, False), (300_000, 3, {}, False)]:
        o = fclsh._build_opts(**kw)
        st = lib.fclsh_derive_params(100, d, r, 5, ctypes.byref(o), shape.ctypes.data, None, None, None, None)
        assert (st == fclsh.OK) == ok, (d, r, kw, fclsh.last_error() if hasattr(fclsh, "last_error") else st)
        sb = lib.fclsh_build(pts.ctypes.data, 1, d, r, 5, ctypes.byref(o), ctypes.byref(h))
        if not ok:
            assert sb == fclsh.EINVAL, (d, r, kw)
        elif not torch.cuda.is_available():
            assert sb == fclsh.ECUDA, (d, r, kw)     # past the host checks, the build needs a device
        elif sb == fclsh.OK:
            lib.fclsh_free(h)


def _struct_fields(header: str, name: str) -> list:
    """Field names of `typedef struct { ... } name;` in the header, in order."""
    import re

    text = re.sub(r"/\*.*?\*/", "", header, flags=re.S)
    end = re.search(r"\}\s*" + name + r"\s*;", text)
    assert end, name
    body = text[text.rindex("typedef struct {", 0, end.start()) + len("typedef struct {"):end.start()]
    return [f.split()[-1].split("[")[0] for f in body.split(";") if f.strip()]


def test_python_structs_mirror_the_header():
    """The binding's ctypes structs have the header's fields in the header's order (a field added
    to one and not the other would shift every later field)."""
    from paper_1602_02620_gb300 import fclsh

    header = open(os.path.join(ROOT, "include", "fclsh.h")).read()
    for cname, pycls in (("fclsh_tuning", fclsh.Tuning), ("fclsh_server_opts", fclsh.ServerOpts)):
        assert _struct_fields(header, cname) == [f for f, _ in pycls._fields_], cname


def test_timing_read_names_every_phase():
    """fclsh_timing_read fills as many phases as the header declares, and the binding names each."""
    import re

    from paper_1602_02620_gb300 import fclsh

    header = open(os.path.join(ROOT, "include", "fclsh.h")).read()
    m = re.search(r"fclsh_timing_read\(fclsh_index \*idx, double ms\[(\d+)\], uint64_t counts\[(\d+)\]", header)
    assert m and m.group(1) == m.group(2)
    src = open(os.path.join(ROOT, "paper_1602_02620_gb300", "fclsh.py")).read()
    assert "(ctypes.c_double * %s)()" % m.group(1) in src and "(ctypes.c_uint64 * %s)()" % m.group(1) in src
