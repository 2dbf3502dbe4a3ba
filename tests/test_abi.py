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
