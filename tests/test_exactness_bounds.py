"""The integer bounds the kernels' exactness rests on, checked with Python integers from the
constants in the library's shared header (no GPU).

* mod P by folding 2^50 == 27: one conditional subtraction for every 64-bit value;
* Algorithm 2 in 64-bit integers: |y_v| <= W (P - 1) < 2^61 for W <= 2^11, and S - y_v < 2^62;
* the scatter sketch adds up to kScatterMaxPop seed values (< P) without reducing;
* the tensor-core route: five 11-bit limbs cover b < 2^50, sums of <= 128 limb products stay
  exact in fp32 (< 2^24), and the recombined value stays below 2^63;
* a directory entry holds the key's top 50 - s bits and the id in 64 bits;
* S3's signature bound (kSigBlocks blocks, the query's occupancy levels) never exceeds the
  Hamming distance, so the pre-filter drops no point within the radius.
"""
import os
import re

import sympy

from tests.conftest import ROOT


def _const(name):
    src = open(os.path.join(ROOT, "paper_1602_02620_gb300", "csrc", "common.cuh")).read()
    m = re.search(r"constexpr\s+\w+\s+%s\s*=\s*([^;]+);" % name, src)
    assert m, name
    expr = m.group(1).replace("ULL", "").replace("1ULL", "1")
    return int(eval(expr, {}))


def _mod_p(x, P):
    r = (x & ((1 << 50) - 1)) + (x >> 50) * 27
    assert r < 2 * P
    return r - P if r >= P else r


def test_prime_and_fold():
    P = _const("kP")
    assert P == 2**50 - 27 and sympy.isprime(P)
    for x in [0, 1, P - 1, P, P + 1, 2**50, 2**63 - 1, 2**63, 2**64 - 1, 16383 * (P - 1),
              *(pow(7, k, 2**64) for k in range(200))]:
        assert _mod_p(x, P) == x % P


def test_algorithm2_stays_in_64_bits():
    P = _const("kP")
    W = 2 ** _const("kMaxLogW")
    assert W * (P - 1) < 2**61                      # |y_v| after the transform of reduced t_j
    assert 2 * W * (P - 1) < 2**62                  # S - y_v = 2 sum over C(v, j) = 1 of t_j


def test_scatter_sketch_sums_fit():
    P = _const("kP")
    pop = _const("kScatterMaxPop")
    assert pop * (P - 1) < 2**64


def test_tensor_core_limbs_are_exact():
    P = _const("kP")
    limb_bits, limbs, K = 11, 5, 128
    assert limb_bits * limbs >= (P - 1).bit_length()
    acc_max = K * (2**limb_bits - 1)                # a sum of K products of 0/1 and one limb
    assert acc_max < 2**18 < 2**24                  # exact in fp32
    assert sum(acc_max << (limb_bits * l) for l in range(limbs)) < 2**63
    # fp16 holds every limb value exactly (11-bit significand)
    assert 2**limb_bits - 1 <= 2**11


def test_directory_entry_fits_64_bits():
    for s in range(13, 33):
        id_bits = 32 if s >= 18 else 14 + s
        assert (50 - s) + id_bits <= 64, s


def _block_counts(bits, B, blocks):
    """Set coordinates of a 0/1 vector in each of `blocks` blocks of B coordinates."""
    padded = list(bits) + [0] * (blocks * B - len(bits))
    return [sum(padded[j * B:(j + 1) * B]) for j in range(blocks)]


def _sig_bound(x, q, d, blocks, levels):
    """S3's pre-filter bound as the kernels compute it from the two block-occupancy signatures and
    the query's occupancy levels: one per block only x occupies, plus min(q's count, levels) per
    block only q occupies."""
    B = -(-d // blocks)
    cx, cq = _block_counts(x, B, blocks), _block_counts(q, B, blocks)
    only_x = sum(1 for a, b in zip(cx, cq) if a and not b)
    only_q = sum(min(b, levels) for a, b in zip(cx, cq) if b and not a)
    return only_x + only_q


def test_signature_bound_never_exceeds_the_distance():
    """A candidate is rejected unread when the bound passes the radius, so the bound must be a lower
    bound on the Hamming distance for every pair (blocks across word boundaries, counts above the
    number of levels), and exact when a block is one coordinate (d <= kSigBlocks)."""
    import numpy as np
    blocks, levels = _const("kSigBlocks"), 8
    assert blocks == 128
    src = open(os.path.join(ROOT, "paper_1602_02620_gb300", "csrc", "common.cuh")).read()
    assert re.search(r"constexpr\s+int\s+kSigLevels\s*=\s*%d\s*;" % levels, src)
    rng = np.random.default_rng(11)
    for d, dens in ((40, 0.3), (128, 0.5), (200, 0.1), (1024, 0.02), (1024, 0.5), (3000, 0.01), (4000, 0.6)):
        for _ in range(60):
            x = (rng.random(d) < dens).astype(int)
            q = (rng.random(d) < dens).astype(int)
            if rng.random() < 0.5:   # a near pair: q = x with a few coordinates flipped
                q = x.copy()
                q[rng.choice(d, size=int(rng.integers(0, 8)), replace=False)] ^= 1
            dist = int((x != q).sum())
            lb = _sig_bound(x, q, d, blocks, levels)
            assert lb <= dist, (d, dens, lb, dist)
            if d <= blocks:
                assert lb == dist
