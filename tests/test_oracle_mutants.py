"""The oracle's pins catch plausible mistakes.

Each mutant below plants one mistake in a copy of the oracle -- a flipped sign, a dropped
term, a wrong index, a transposed operand, an off-by-one, a missing reduction -- and at
least one pin of ``tests/test_oracle.py`` must fail on that copy, while the unchanged copy
passes them all.  The mistakes are planted in copies of the oracle only, on the CPU; each
copy is compiled and run in a subprocess of its own, so the real oracle is never touched.
Every mutant keeps all memory accesses in bounds (where a mistake would let a buffer
overflow, the mutant also enlarges that buffer).
"""
import json
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

from tests.conftest import ROOT

P = (1 << 50) - 27
C, PY = "fclsh_oracle.c", "__init__.py"

# name -> (the pin that must catch it, [(file, original text, planted text), ...]); each
# original text occurs exactly once in its file.
MUTANTS = {
    # Walsh-Hadamard transform and the finish of Algorithm 2
    "butterfly operands transposed": ("test_lemma3_fht_equals_direct", [
        (C, "t[j + h] = a - c;", "t[j + h] = c - a;")]),
    "transform misses its last stage": ("test_lemma3_fht_equals_direct", [
        (C, "for (uint32_t h = 1; h < W; h <<= 1)", "for (uint32_t h = 1; h < W / 2; h <<= 1)")]),
    "finish adds the transform": ("test_lemma3_fht_equals_direct", [
        (C, "i128 twice = l1 - t[v];", "i128 twice = l1 + t[v];")]),
    "finish drops the halving": ("test_lemma3_fht_equals_direct", [
        (C, "i128 half = twice / 2;", "i128 half = twice;")]),
    "finish skips mod P": ("test_fht_route_against_dense_hadamard", [
        (C, "out[v - 1] = (uint64_t)(half % (i128)p->P);", "out[v - 1] = (uint64_t)half;")]),
    "sketch into the wrong column": ("test_lemma3_fht_equals_direct", [
        (C, "t[p->m[i]] += qt;", "t[p->m[i] ^ 1u] += qt;")]),
    "l1 norm keeps only the last term": ("test_lemma3_fht_equals_direct", [
        (C, "l1 += qt;", "l1 = qt;")]),
    # covering vectors and Eq. (1)
    "code entry by OR": ("test_code_rows_match_sylvester_hadamard", [
        (C, "return parity32(v & j);", "return parity32(v | j);")]),
    "column index is the position": ("test_example1_covering_vectors", [
        (C, "int g = had(v, p->m[i]);", "int g = had(v, i - p->part_off[k]);")]),
    "covering vector ORed with the point": ("test_example1_covering_vectors", [
        (C, "int y = g & xi;", "int y = g | xi;")]),
    "permutation ignored": ("test_example3_partition", [
        (C, "int xi = get_bit(x, p->perm[i]);", "int xi = get_bit(x, i % p->d);")]),
    "first term of Eq. (1) dropped": ("test_example1_covering_vectors", [
        (C, "sum += (u128)p->b[i] * (u128)y;", "if (i > p->part_off[k]) sum += (u128)p->b[i] * (u128)y;")]),
    "Eq. (1) skips mod P": ("test_r0_special_case_is_plain_universal_hash", [
        (C, "return (uint64_t)(sum % p->P);", "return (uint64_t)sum;")]),
    # parameters (Algorithm 1 pre-processing, choices of m and b)
    "general map may take column 0": ("test_prime_and_params_ranges", [
        (C, "m[lo + i] = 1 + (uint32_t)(sm64_next(&state) % (uint64_t)(W - 1));",
         "m[lo + i] = (uint32_t)(sm64_next(&state) % (uint64_t)W);")]),
    "replication repeats each coordinate": ("test_example3_replication", [
        (C, "perm[copy * d + c] = c;", "perm[copy * d + c] = (copy * d + c) / rep;")]),
    "SplitMix64 multiplier typo": ("test_splitmix64_published_vector", [
        (C, "0xBF58476D1CE4E5B9ULL", "0xBF58476D1CE4E5B8ULL")]),
    "per-part radius ignores replication": ("test_example3_replication", [
        (PY, "    rp = r * rep // t\n    W = 2 << rp\n    D = d * rep\n    perm = np.zeros(D",
         "    rp = r // t\n    W = 2 << rp\n    D = d * rep\n    perm = np.zeros(D")]),
    # tables and the query (Strategy 2, S1-S3)
    "tables not sorted by key": ("test_tables_group_equal_keys", [
        (C, "if (x->key != y->key) return x->key < y->key ? -1 : 1;", "if (0) return 0;")]),
    "bucket search finds the end of the bucket": ("test_strategy2_equals_linear_scan", [
        (C, "if (keys[mid] < key) lo = mid + 1; else hi = mid;", "if (keys[mid] <= key) lo = mid + 1; else hi = mid;")]),
    "query keys taken from the wrong table": ("test_strategy2_equals_linear_scan", [
        (C, "qkeys[tau] = oracle_key_direct(p, q, tau);", "qkeys[tau] = oracle_key_direct(p, q, tau ? tau - 1 : 0);")]),
    "candidates not deduplicated": ("test_strategy2_equals_linear_scan", [
        (C, "if (!(bitmap[id >> 3] & (1u << (id & 7)))) {", "if (1) {"),
        (C, "uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));",
         "uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1) * T);")]),
    "verify excludes distance == radius": ("test_strategy2_equals_linear_scan", [
        (C, "if (hamming(q, pts + (uint64_t)id * p->words, p->words) <= (int)radius) {",
         "if (hamming(q, pts + (uint64_t)id * p->words, p->words) < (int)radius) {")]),
    "restricted probe skips its last row": ("test_counters_follow_their_definitions", [
        (C, "if (rows && v > rows) continue;", "if (rows && v >= rows) continue;")]),
    "probe rule one row bit short": ("test_row_restricted_probe_covers_exhaustively", [
        (PY, "e = radius * p.rep // p.t + 1", "e = radius * p.rep // p.t")]),
    # the plain definition of the answer
    "distance misses the last word": ("test_linear_scan_bruteforce", [
        (C, "for (uint32_t w = 0; w < words; w++) {\n        uint64_t z",
         "for (uint32_t w = 0; w + 1 < words; w++) {\n        uint64_t z")]),
    "linear scan excludes distance == radius": ("test_linear_scan_bruteforce", [
        (C, "if (hamming(q, pts + i * words, words) <= (int)radius) {",
         "if (hamming(q, pts + i * words, words) < (int)radius) {")]),
}

# Pins run on every copy: (test function of tests/test_oracle.py, arguments).
BATTERY = [
    ("test_example1_covering_vectors", []),
    ("test_example2_code_matrix_and_collisions", []),
    ("test_example3_partition", []),
    ("test_example3_replication", []),
    ("test_code_rows_match_sylvester_hadamard", [16]),
    ("test_fht_route_against_dense_hadamard", [64, 101]),
    ("test_lemma3_fht_equals_direct", [64, 3, 1, P]),
    ("test_lemma3_fht_equals_direct", [100, 2, 1, 97]),
    ("test_lemma3_fht_equals_direct", [256, 16, 2, P]),
    ("test_r0_special_case_is_plain_universal_hash", []),
    ("test_theorem1_every_map_covers", [10, 3]),
    ("test_near_pairs_always_collide", [64, 10, 2]),
    ("test_splitmix64_published_vector", []),
    ("test_prime_and_params_ranges", []),
    ("test_partition_rule", []),
    ("test_linear_scan_bruteforce", []),
    ("test_strategy2_equals_linear_scan", [64, 3, 1]),
    ("test_tables_group_equal_keys", []),
    ("test_replication_equals_index_of_repeated_vectors", [10, 1, 4]),
    ("test_row_restricted_probe_covers_exhaustively", [8, 2]),
    ("test_counters_follow_their_definitions", [64, 3, 1, 1]),
]

# Runs the battery against the oracle package found first on sys.path (the copy) and
# prints the names of the pins that failed.
_RUNNER = r"""
import json, sys
copy_dir, root, battery = sys.argv[1], sys.argv[2], json.loads(sys.argv[3])
sys.path.insert(0, copy_dir)
import oracle
assert oracle.__file__.startswith(copy_dir), oracle.__file__
sys.path.append(root)
import tests.test_oracle as pins
failed = []
for name, args in battery:
    try:
        getattr(pins, name)(*args)
    except Exception:
        failed.append(name)
print(json.dumps(failed))
"""


def _run_copy(base, num, name, edits):
    """Copy the oracle, plant `edits`, run the battery on it; returns the failed pins."""
    copy_dir = os.path.join(base, "copy%02d" % num)
    pkg = os.path.join(copy_dir, "oracle")
    os.makedirs(pkg)
    for f in (C, PY):
        shutil.copy(os.path.join(ROOT, "oracle", f), os.path.join(pkg, f))
    for f, old, new in edits:
        path = os.path.join(pkg, f)
        src = open(path).read()
        assert src.count(old) == 1, (name, old)
        open(path, "w").write(src.replace(old, new))
    out = subprocess.run([sys.executable, "-c", _RUNNER, copy_dir, ROOT, json.dumps(BATTERY)],
                         cwd=copy_dir, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, (name, out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    base = str(tmp_path_factory.mktemp("oracle_mutants"))
    jobs = {"unchanged": []}
    jobs.update({k: v[1] for k, v in MUTANTS.items()})
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        futs = {k: ex.submit(_run_copy, base, i, k, e) for i, (k, e) in enumerate(jobs.items())}
        return {k: f.result() for k, f in futs.items()}


def test_unchanged_copy_passes_every_pin(results):
    assert results["unchanged"] == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_the_mutant(results, name):
    failed = results[name]
    assert failed, "no pin caught: " + name
    assert MUTANTS[name][0] in failed, (name, failed)
