import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libfclsh.so")
    config.addinivalue_line("markers", "slow: full-size workloads")


def read_golden(name: str) -> dict:
    """key -> list of whitespace-separated tokens, comments dropped."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, *v = line.split()
            out[k] = v
    return out


def bits_to_words(s: str):
    """A bit string (coordinate 0 first) packed LSB-first into uint64 words."""
    import numpy as np

    words = (len(s) + 63) // 64
    w = np.zeros(words, np.uint64)
    for i, ch in enumerate(s):
        if ch == "1":
            w[i >> 6] |= np.uint64(1) << np.uint64(i & 63)
    return w


def bits_to_int(s: str) -> int:
    """Bit string (coordinate 0 first) as the integer sum 2^i over set coordinates."""
    return sum(1 << i for i, ch in enumerate(s) if ch == "1")


@pytest.fixture(autouse=True)
def _checked_build_guard(request):
    """With FCLSH_CHECKED=1 the GPU tests run against the bounds-checked build of the library
    (python -m paper_1602_02620_gb300.build --checked): after each one, no check may have fired."""
    yield
    if os.environ.get("FCLSH_CHECKED") != "1" or request.node.get_closest_marker("gpu") is None:
        return
    try:
        import torch
    except ImportError:
        return
    if not torch.cuda.is_available():
        return
    from paper_1602_02620_gb300 import fclsh

    checked, first = fclsh.debug_check_status()
    assert checked, "FCLSH_CHECKED=1 but the loaded library is not the checked build"
    assert first == 0, "bounds check 0x%04x failed in %s" % (first, request.node.nodeid)
