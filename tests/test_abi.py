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
