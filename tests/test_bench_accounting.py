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


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the oracle on the host cores, no GPU) prints one JSON line with the
    fields the benchmark contract names: its own value repeated in cpu_baseline and e2e, no
    host-device traffic, and a ms_per_step that says it is extrapolated from a sample."""
    import json
    import os
    import subprocess
    import sys

    from tests.conftest import ROOT

    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "1",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, r.stdout[-2000:]
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["higher_is_better"] is True and line["steps"] == 1
    assert line["value"] > 0 and line["unit"] == "queries/s"
    assert "extrapolated" in line["ms_per_step_kind"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "queries/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("plain-small")
