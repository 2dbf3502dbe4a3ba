"""Host-side accounting of bench.py: the algorithmic bytes a hash launch is credited with."""
from types import SimpleNamespace

import numpy as np

import bench


def test_set_bits_counts_every_word():
    rng = np.random.default_rng(0)
    pts = rng.integers(0, 2**63, size=(37, 5), dtype=np.uint64) | np.uint64(1 << 63)
    want = int(np.unpackbits(pts.view(np.uint8)).sum())
    assert bench.set_bits(pts) == want


def test_hash_bytes_follow_what_the_kernel_reads():
    rng = np.random.default_rng(1)
    # dense short points: the packed words of every point, plus 8 B per key
    w = SimpleNamespace(n=100, d=128, points=rng.integers(0, 2**63, size=(100, 2), dtype=np.uint64))
    assert bench.hash_part_bytes(w, 511, 2) == 100 * (16 + 8 * 511)
    # long sparse points under the scatter sketch: their list of set coordinates instead
    d = 64 * bench.CSR_MIN_WORDS
    pts = np.zeros((50, d // 64), np.uint64)
    for i in range(50):
        for c in rng.choice(d, size=20, replace=False):
            pts[i, c >> 6] |= np.uint64(1) << np.uint64(c & 63)
    w = SimpleNamespace(n=50, d=d, points=pts)
    assert bench.hash_part_bytes(w, 127, 3) == 4 * 50 * 20 + 12 * 50 + 8 * 127 * 50
    # the same points by a gather kernel, or too short for the list, are read as packed words
    assert bench.hash_part_bytes(w, 127, 0) == 50 * d / 8 + 8 * 127 * 50
    short = SimpleNamespace(n=50, d=d // 2, points=pts[:, : d // 128])
    assert bench.hash_part_bytes(short, 127, 3) == 50 * (d // 2) / 8 + 8 * 127 * 50
