"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a printed
example, an independent construction (scipy's Sylvester Hadamard matrix, Python
big integers, brute force), a theorem of the paper, or a published test vector.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg
import sympy

import oracle
from tests.conftest import bits_to_int, bits_to_words, read_golden

P = oracle.P_DEFAULT


def _pow2_b(d):
    """b_i = 2^i: the Eq. (1) key then equals the bit mask of g_v AND x."""
    return [1 << i for i in range(d)]


# ----------------------------------------------------------------- worked examples

def test_example1_covering_vectors():
    """Example 1 (Sec. 2.3): the seven vectors g_v and the single collision at g_4."""
    g = read_golden("example1_covering.txt")
    d, r = int(g["d"][0]), int(g["r"][0])
    m = [int(s, 2) for s in g["m"]]
    p = oracle.make_params(d, r, m, _pow2_b(d))
    assert p.W == 8 and p.T == 7
    ones = bits_to_words("1" * d)
    x, q = bits_to_words(g["x"][0]), bits_to_words(g["q"][0])
    for v in range(1, 8):
        assert oracle.key_direct(p, ones, v - 1) == bits_to_int(g["g%d" % v][0])
    kx, kq = oracle.keys_direct(p, x)[:, 0], oracle.keys_direct(p, q)[:, 0]
    coll = [v for v in range(1, 8) if kx[v - 1] == kq[v - 1]]
    assert coll == [int(g["collide"][0])]
    assert int(kx[coll[0] - 1]) == bits_to_int(g["value"][0])
    assert oracle.hamming(x, q) == 2


def test_example2_code_matrix_and_collisions():
    """C_{7,8} and Example 2 (Sec. 3.1): x collides with q only under row 3, y never."""
    g = read_golden("example2_c78.txt")
    d, r = int(g["d"][0]), int(g["r"][0])
    p = oracle.make_params(d, r, list(range(d)), _pow2_b(d))
    ones = bits_to_words("1" * d)
    for v in range(1, 8):
        assert oracle.key_direct(p, ones, v - 1) == bits_to_int(g["C%d" % v][0])
    x, y, q = (bits_to_words(g[k][0]) for k in ("x", "y", "q"))
    assert oracle.hamming(x, q) == int(g["dist_xq"][0])
    assert oracle.hamming(y, q) == int(g["dist_yq"][0])
    kx, ky, kq = (oracle.keys_direct(p, a)[:, 0] for a in (x, y, q))
    coll_xq = [v for v in range(1, 8) if kx[v - 1] == kq[v - 1]]
    assert coll_xq == [int(g["collide_xq"][0])]
    assert int(kx[coll_xq[0] - 1]) == bits_to_int(g["value_xq"][0])
    assert g["collide_yq"] == ["none"]
    assert not any(ky[v] == kq[v] for v in range(7))
    # the same keys through Algorithm 2
    pts = np.stack([x, y, q])
    assert np.array_equal(oracle.keys_fht(p, pts), oracle.keys_direct(p, pts))


def test_example3_partition():
    """Example 3 (Sec. 3.1): permuting 0011 into 0110 and splitting gives 01 and 10."""
    g = read_golden("example3_preprocessing.txt")
    q, qp = g["q"][0], g["permuted"][0]
    # a permutation with q'_i = q_{perm[i]} that turns 0011 into 0110
    perm = [0, 2, 3, 1]
    assert "".join(q[j] for j in perm) == qp
    # t = 2 parts, r = 2 -> r' = 1, W = 4.  m = (1, 3) in each part: row v = 1 has
    # Had(1)_1 = Had(1)_3 = 1, so with b = (1, 2) the row-1 key spells the part's bits.
    p = oracle.make_params(4, 2, m=[1, 3, 1, 3], b=[1, 2, 1, 2], t=2, perm=perm)
    assert p.W == 4 and p.T == 6
    keys = oracle.keys_direct(p, bits_to_words(q))[:, 0]
    assert int(keys[0 * 3 + 0]) == bits_to_int(g["part1"][0])
    assert int(keys[1 * 3 + 0]) == bits_to_int(g["part2"][0])


def test_example3_replication():
    """Example 3 (Sec. 3.1): replicating 0011 twice gives 00110011.  The derived positions
    of a replicated index read those bits, and with every position on column 1 and
    b_i = 2^i the row-1 key spells the replicated vector."""
    g = read_golden("example3_preprocessing.txt")
    q, q2 = g["q"][0], g["replicated2"][0]
    p = oracle.derive_params(9, 4, 1, rep=2)
    assert p.rep == 2 and p.t == 1 and p.rp == 2 and p.W == 8 and p.perm.shape == (8,)
    assert "".join(q[int(c)] for c in p.perm) == q2
    p = oracle.make_params(4, 1, m=[1] * 8, b=_pow2_b(8), rep=2)
    assert int(oracle.keys_direct(p, bits_to_words(q))[0, 0]) == bits_to_int(q2)
    assert int(oracle.keys_fht(p, bits_to_words(q))[0, 0]) == bits_to_int(q2)


def _repeat_bits(pts, d, rep):
    """Each packed d-bit row written rep times in a row, repacked (plain numpy bit ops)."""
    words = (d + 63) // 64
    bits = np.unpackbits(pts.view(np.uint8).reshape(-1, words * 8), axis=1, bitorder="little")[:, :d]
    rb = np.concatenate([bits] * rep, axis=1)
    D = d * rep
    W2 = (D + 63) // 64
    padded = np.zeros((rb.shape[0], W2 * 64), np.uint8)
    padded[:, :D] = rb
    return np.packbits(padded, axis=1, bitorder="little").view(np.uint64).reshape(-1, W2)


@pytest.mark.parametrize("d,r,rep", [(10, 1, 4), (40, 2, 3), (24, 3, 2), (100, 2, 2), (70, 1, 5), (17, 4, 2)])
def test_replication_equals_index_of_repeated_vectors(d, r, rep):
    """Algorithm 1, cr < log n: a replicated index gives every point the keys that a plain
    index on the explicitly repeated d*rep-bit vectors gives, with the same m and b and
    radius r*rep (covering both the specific, d*rep <= W, and general construction)."""
    rng = np.random.default_rng(d * 13 + rep)
    p = oracle.derive_params(d + 100 * rep, d, r, rep=rep)
    assert p.rp == r * rep and p.W == 2 << (r * rep)
    pts = rng.integers(0, 2**63, size=(60, (d + 63) // 64), dtype=np.uint64)
    if d % 64:
        pts[:, -1] &= np.uint64((1 << (d % 64)) - 1)
    plain = oracle.make_params(d * rep, r * rep, m=p.m, b=p.b)
    assert plain.W == p.W
    want = oracle.keys_direct(plain, _repeat_bits(pts, d, rep))
    assert np.array_equal(oracle.keys_direct(p, pts), want)
    assert np.array_equal(oracle.keys_fht(p, pts), want)


@pytest.mark.parametrize("d,r,rep", [(6, 1, 3), (5, 2, 2), (8, 1, 4), (7, 2, 2), (12, 1, 2)])
def test_replication_total_recall_exhaustive(d, r, rep):
    """Lemma 4 (1): with replication every z with |z| <= r still collides with 0 in some
    table, for random m and b (the replicated z has rep*|z| <= r' ones, Theorem 1)."""
    zs = list(_ball(d, r))
    Z = np.zeros((len(zs), 1), np.uint64)
    for i, pos in enumerate(zs):
        Z[i, 0] = sum(1 << j for j in pos)
    for trial in range(25):
        p = oracle.derive_params(trial * 7 + d, d, r, rep=rep)
        k = oracle.keys_direct(p, Z)
        assert np.all((k == 0).any(axis=0)), trial


def test_replication_expected_collisions():
    """Lemma 4 (2), replication: a pair at distance D0 collides in fewer than
    2 * 2^(rep r) * 2^(-rep D0) tables on average.  The rep*D0 differing positions have
    independent columns, so the expectation has the closed forms of Theorem 2 with
    rep*D0 in place of the distance; both are pinned (4 standard errors)."""
    from math import comb
    rng = np.random.default_rng(11)
    for d, r, rep, general in ((12, 2, 2, False), (60, 1, 3, True)):
        W = 2 << (r * rep)
        assert (d * rep > W) == general
        for dist in (1, 2, 3):
            k = rep * dist
            counts = []
            for trial in range(300):
                p = oracle.derive_params(7000 + trial, d, r, rep=rep)
                x = rng.integers(0, 2**63, size=(1, 1), dtype=np.uint64)
                x[0, 0] &= np.uint64((1 << d) - 1)
                y = x.copy()
                for pos in rng.choice(d, size=dist, replace=False):
                    y[0, 0] ^= np.uint64(1) << np.uint64(pos)
                counts.append(int((oracle.keys_direct(p, x) == oracle.keys_direct(p, y)).sum()))
            mean, se = np.mean(counts), np.std(counts) / np.sqrt(len(counts))
            if general:
                exact = (W - 1) * ((W / 2 - 1) / (W - 1)) ** k
            else:
                exact = (W - 1) * comb(W // 2, k) / comb(W, k)
            assert exact < 2 * 2.0 ** (rep * r) * 2.0 ** (-rep * dist)
            assert abs(mean - exact) <= 4 * se + 1e-9, (d, rep, dist, mean, exact)


@pytest.mark.parametrize("d,r,rep", [(32, 2, 3), (48, 3, 2), (100, 2, 2), (64, 1, 4)])
def test_replicated_query_equals_linear_scan(d, r, rep):
    """Strategy 2 on a replicated index reports the linear-scan answer for every radius
    rho <= r, probing all tables or only rows v < 2^(rho*rep+1)."""
    rng = np.random.default_rng(d + 3 * rep)
    words = (d + 63) // 64
    n = 250
    pts = rng.integers(0, 2**63, size=(n, words), dtype=np.uint64)
    if d % 64:
        pts[:, -1] &= np.uint64((1 << (d % 64)) - 1)
    pts[5:9] = pts[4]
    p = oracle.derive_params(d * r + rep, d, r, rep=rep)
    tables = oracle.build_tables(p, pts)
    for qi in range(15):
        q = pts[rng.integers(0, n)].copy()
        for pos in rng.choice(d, size=rng.integers(0, r + 2), replace=False):
            q[pos >> 6] ^= np.uint64(1) << np.uint64(pos & 63)
        for rho in range(r + 1):
            rows = oracle.probe_rows(p, rho)
            assert rows == min(p.W - 1, (2 << (rho * rep)) - 1)
            ids, ncoll, ncand = oracle.query(p, pts, tables, q, rho, rows=rows)
            full, fcoll, fcand = oracle.query(p, pts, tables, q, rho)
            assert ids.tolist() == oracle.linear_scan(pts, q, rho).tolist() == full.tolist()
            assert ncoll <= fcoll and ncand <= fcand and ncoll >= ncand >= len(ids)


# ----------------------------------------------------------------- Hadamard code

@pytest.mark.parametrize("W", [2, 4, 8, 16, 32])
def test_code_rows_match_sylvester_hadamard(W):
    """C = (1 - H) / 2 (Eq. 6) with H the Sylvester Hadamard matrix of scipy."""
    H = scipy.linalg.hadamard(W)
    r = W.bit_length() - 2
    p = oracle.make_params(W, r, list(range(W)), _pow2_b(W))
    ones = np.full((W + 63) // 64, ~np.uint64(0), np.uint64)
    if W % 64:
        ones[-1] = np.uint64((1 << (W % 64)) - 1)
    for v in range(1, W):
        want = sum(1 << j for j in range(W) if (1 - H[v, j]) // 2 == 1)
        assert oracle.key_direct(p, ones, v - 1) == want


@pytest.mark.parametrize("W,P_", [(8, 97), (64, 101), (512, 65537), (2048, (1 << 31) - 1), (256, P)])
def test_fht_route_against_dense_hadamard(W, P_):
    """Algorithm 2's finish, h = (||q~||_1 - H t)/2 mod P, with H from scipy, t by hand."""
    rng = np.random.default_rng(W)
    d = W // 2
    r = W.bit_length() - 2
    p = oracle.derive_params(11 + W, d, r, t=1, P=P_)
    assert p.W == W
    H = scipy.linalg.hadamard(W).astype(object)
    pts = rng.integers(0, 2**63, size=(5, (d + 63) // 64), dtype=np.uint64)
    if d % 64:
        pts[:, -1] &= np.uint64((1 << (d % 64)) - 1)
    got = oracle.keys_fht(p, pts)
    for i in range(pts.shape[0]):
        bits = [(int(pts[i, j >> 6]) >> (j & 63)) & 1 for j in range(d)]
        t = [0] * W
        for pos in range(d):
            t[int(p.m[pos])] += int(p.b[pos]) * bits[int(p.perm[pos])]
        l1 = sum(t)
        y = H.dot(np.array(t, dtype=object))
        for v in range(1, W):
            assert (l1 - y[v]) % 2 == 0
            assert int(got[v - 1, i]) == ((l1 - y[v]) // 2) % P_


# ----------------------------------------------------------------- Lemma 3

@pytest.mark.parametrize("d,r,t,P_", [
    (64, 3, 1, P),        # general construction (d > W = 16)
    (128, 8, 1, P),       # specific construction (d <= W = 512)
    (100, 2, 1, 97),      # general, small prime: many modular wraps
    (256, 16, 2, P),      # two parts, specific per part
    (1024, 20, 2, 1009),  # two parts, W = 2048, small prime
    (300, 7, 3, 65537),   # three parts, general per part (100 > 16)
    (70, 6, 1, P),        # specific with d not a multiple of 64
    (5, 0, 1, P),         # r = 0: one table, W = 2
])
def test_lemma3_fht_equals_direct(d, r, t, P_):
    """Lemma 3: Algorithm 2 gives the same keys as Eq. (1) on the covering vectors."""
    p = oracle.derive_params(1000 + d + r, d, r, t=t, P=P_)
    rng = np.random.default_rng(d * 31 + r)
    words = (d + 63) // 64
    pts = rng.integers(0, 2**63, size=(40, words), dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=(40, words), dtype=np.uint64)
    if d % 64:
        pts[:, -1] &= np.uint64((1 << (d % 64)) - 1)
    pts[0] = 0
    assert np.array_equal(oracle.keys_fht(p, pts), oracle.keys_direct(p, pts))
    assert not oracle.keys_direct(p, pts)[:, 0].any()   # the zero vector hashes to 0 everywhere


def test_r0_special_case_is_plain_universal_hash():
    """r = 0, general map: W = 2, every coordinate goes to column 1, so the one key
    is Eq. (1) itself, sum_i b_i x_i mod P (checked with Python integers)."""
    d = 200
    p = oracle.derive_params(5, d, 0)
    assert p.W == 2 and p.T == 1 and np.all(p.m == 1)
    rng = np.random.default_rng(0)
    pts = rng.integers(0, 2**63, size=(20, 4), dtype=np.uint64)
    pts[:, -1] &= np.uint64((1 << (d % 64)) - 1)
    keys = oracle.keys_direct(p, pts)
    for i in range(20):
        s = sum(int(p.b[j]) for j in range(d) if (int(pts[i, p.perm[j] >> 6]) >> (int(p.perm[j]) & 63)) & 1)
        assert int(keys[0, i]) == s % P


# ----------------------------------------------------------------- Theorem 1 / 2

def _ball(d, r):
    for k in range(r + 1):
        for pos in itertools.combinations(range(d), k):
            yield pos


@pytest.mark.parametrize("d,r", [(4, 1), (6, 2), (8, 2), (10, 3), (12, 3), (20, 2)])
def test_theorem1_every_map_covers(d, r):
    """Theorem 1: for any m, every z with |z| <= r has a row v with g_v AND z = 0."""
    W = 2 << r
    rng = np.random.default_rng(d * 7 + r)
    zs = list(_ball(d, r))
    Z = np.zeros((len(zs), 1), np.uint64)
    for i, pos in enumerate(zs):
        Z[i, 0] = sum(1 << j for j in pos)
    maps = [rng.integers(0, W, size=d) for _ in range(30)]
    maps.append(np.zeros(d, np.int64))                 # degenerate: every coordinate on column 0
    maps.append(np.full(d, W - 1, np.int64))           # all on one column
    for m in maps:
        p = oracle.make_params(d, r, m, _pow2_b(d))
        k = oracle.keys_direct(p, Z)                   # key == bit mask of g_v AND z
        assert np.all((k == 0).any(axis=0))


@pytest.mark.parametrize("d,r,t", [(64, 3, 1), (128, 6, 1), (64, 10, 2), (96, 12, 2), (90, 21, 3)])
def test_near_pairs_always_collide(d, r, t):
    """Total recall (Theorem 1 with the pigeonhole split of Sec. 3.1): any two points
    at distance <= r share a key in at least one table, for random b, m and pi."""
    rng = np.random.default_rng(d + r)
    words = (d + 63) // 64
    for trial in range(6):
        p = oracle.derive_params(trial * 17 + d, d, r, t=t)
        xs = rng.integers(0, 2**63, size=(50, words), dtype=np.uint64)
        if d % 64:
            xs[:, -1] &= np.uint64((1 << (d % 64)) - 1)
        ys = xs.copy()
        for i in range(50):
            k = rng.integers(0, r + 1)
            for pos in rng.choice(d, size=k, replace=False):
                ys[i, pos >> 6] ^= np.uint64(1) << np.uint64(pos & 63)
        kx, ky = oracle.keys_direct(p, xs), oracle.keys_direct(p, ys)
        assert np.all((kx == ky).any(axis=0))


def test_theorem2_expected_collisions_closed_form():
    """Theorem 2 (2): E[#rows v with g_v(x) = g_v(y)] < 2^(r+1-dist).

    The expectation also has a closed form, pinned here both ways (4 standard
    errors).  A row v != 0 collides iff every differing position lands on a column
    j with <a(j), v> = 0; W/2 columns (column 0 among them) have that property.
      - specific construction (d = W, random permutation): the dist positions land
        on distinct columns, E = (W-1) C(W/2, dist) / C(W, dist);
      - general construction with column 0 left out (Sec. 3.3): columns are uniform
        over 1..W-1, of which W/2-1 qualify, E = (W-1) ((W/2-1)/(W-1))^dist.
    The printed "sharper" bound 2^(r+1) (1/2 - 2^-(r+1))^dist is below this exact
    value for dist >= 2, so only Theorem 2's bound is asserted as a bound.
    """
    from math import comb
    rng = np.random.default_rng(3)
    d, r = 64, 5
    W = 2 << r
    for dist in (3, 6, 9):
        counts = []
        for trial in range(400):
            p = oracle.derive_params(trial, d, r)
            x = rng.integers(0, 2**63, size=(1, 1), dtype=np.uint64)
            y = x.copy()
            for pos in rng.choice(d, size=dist, replace=False):
                y[0, 0] ^= np.uint64(1) << np.uint64(pos)
            counts.append(int((oracle.keys_direct(p, x) == oracle.keys_direct(p, y)).sum()))
        mean, se = np.mean(counts), np.std(counts) / np.sqrt(len(counts))
        exact = (W - 1) * comb(W // 2, dist) / comb(W, dist)
        assert exact < 2.0 ** (r + 1 - dist)
        assert abs(mean - exact) <= 4 * se + 1e-9, (dist, mean, exact)
    d, r = 200, 3
    W = 2 << r
    for dist in (1, 2, 4):
        counts = []
        for trial in range(400):
            p = oracle.derive_params(5000 + trial, d, r)
            x = rng.integers(0, 2**63, size=(1, 4), dtype=np.uint64)
            x[0, 3] &= np.uint64((1 << 8) - 1)
            y = x.copy()
            for pos in rng.choice(d, size=dist, replace=False):
                y[0, pos >> 6] ^= np.uint64(1) << np.uint64(pos & 63)
            counts.append(int((oracle.keys_direct(p, x) == oracle.keys_direct(p, y)).sum()))
        mean, se = np.mean(counts), np.std(counts) / np.sqrt(len(counts))
        exact = (W - 1) * ((W / 2 - 1) / (W - 1)) ** dist
        assert exact < 2.0 ** (r + 1 - dist)
        assert abs(mean - exact) <= 4 * se + 1e-9, (dist, mean, exact)


# ----------------------------------------------------------------- parameters / RNG

def test_splitmix64_published_vector():
    """SplitMix64 from seed 1234567: the generator's published first outputs."""
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    assert [int(v) for v in oracle.splitmix64(1234567, 5)] == want


def test_prime_and_params_ranges():
    assert sympy.isprime(P) and P < 2**50 and not any(sympy.isprime(q) for q in range(P + 1, 2**50))
    for (d, r) in [(64, 3), (128, 8), (256, 16), (1024, 20), (30, 25)]:
        p = oracle.derive_params(42, d, r)
        assert p.t == oracle.default_parts(r) and p.rp == r // p.t and p.W == 2 ** (p.rp + 1)
        assert sorted(p.perm.tolist()) == list(range(d))
        if p.t == 1:
            assert p.perm.tolist() == list(range(d))
        assert p.part_off[0] == 0 and p.part_off[-1] == d
        for k in range(p.t):
            lo, hi = int(p.part_off[k]), int(p.part_off[k + 1])
            mk = p.m[lo:hi]
            if hi - lo <= p.W:
                assert len(set(mk.tolist())) == hi - lo and mk.max() < p.W     # injective: a permutation's prefix
            else:
                assert mk.min() >= 1 and mk.max() < p.W                         # column 0 left out
        assert int(p.b.max()) < P
        q = oracle.derive_params(42, d, r)
        assert np.array_equal(p.b, q.b) and np.array_equal(p.m, q.m)


def test_partition_rule():
    """Sec. 4.4: one part below radius 10, two parts for 10..20 (L = 2(2^(r/2+1) - 1))."""
    assert [oracle.default_parts(r) for r in range(10)] == [1] * 10
    assert all(oracle.default_parts(r) == 2 for r in range(10, 22))
    for r in (10, 12, 14, 16):
        p = oracle.derive_params(1, 256, r)
        assert p.T == 2 * (2 ** (r // 2 + 1) - 1)
    assert oracle.derive_params(1, 256, 16).T == 1022       # the paper's L for r = 16


# ----------------------------------------------------------------- queries

def test_linear_scan_bruteforce():
    rng = np.random.default_rng(9)
    pts = rng.integers(0, 2**63, size=(300, 2), dtype=np.uint64)
    q = pts[17].copy()
    q[0] ^= np.uint64(0b1011)
    for radius in (0, 3, 40, 64, 128):
        want = [i for i in range(300)
                if bin(int(pts[i, 0]) ^ int(q[0])).count("1") + bin(int(pts[i, 1]) ^ int(q[1])).count("1") <= radius]
        assert oracle.linear_scan(pts, q, radius).tolist() == want


@pytest.mark.parametrize("d,r,t", [(32, 4, 1), (64, 3, 1), (100, 6, 1), (128, 2, 1), (64, 12, 2), (200, 9, 1)])
def test_strategy2_equals_linear_scan(d, r, t):
    """Strategy 2 over the covering tables reports exactly the linear-scan answer
    (no false negatives, no false positives), for every radius up to r."""
    rng = np.random.default_rng(d + 100 * r)
    words = (d + 63) // 64
    n = 400
    pts = rng.integers(0, 2**63, size=(n, words), dtype=np.uint64)
    if d % 64:
        pts[:, -1] &= np.uint64((1 << (d % 64)) - 1)
    pts[5] = pts[4]                                    # a duplicate point
    p = oracle.derive_params(d * r + 1, d, r, t=t)
    tables = oracle.build_tables(p, pts)
    for qi in range(25):
        q = pts[rng.integers(0, n)].copy()
        for pos in rng.choice(d, size=rng.integers(0, r + 2), replace=False):
            q[pos >> 6] ^= np.uint64(1) << np.uint64(pos & 63)
        for radius in sorted({0, r // 2, r}):
            ids, ncoll, ncand = oracle.query(p, pts, tables, q, radius)
            want = oracle.linear_scan(pts, q, radius)
            assert ids.tolist() == want.tolist()
            assert ncoll >= ncand >= len(ids)


def test_tables_group_equal_keys():
    rng = np.random.default_rng(1)
    pts = rng.integers(0, 4, size=(200, 1), dtype=np.uint64)   # many duplicates
    p = oracle.derive_params(3, 64, 3)
    keys_all = oracle.keys_direct(p, pts)
    for tau in (0, 7, 14):
        keys, ids = oracle.table(p, pts, tau)
        assert np.all(np.diff(keys.astype(np.float64)) >= 0)
        assert sorted(ids.tolist()) == list(range(200))
        assert np.array_equal(keys, keys_all[tau, ids])


@pytest.mark.parametrize("d,r", [(8, 2), (10, 3), (12, 3)])
def test_row_restricted_probe_covers_exhaustively(d, r):
    """Rows v < 2^(rho+1) of a code built for r >= rho still cover radius rho (Theorem 1
    applied to the map m mod 2^(rho+1)); one row fewer does not, for some z."""
    W = 2 << r
    rng = np.random.default_rng(d * 31 + r)
    for rho in range(r + 1):
        zs = list(_ball(d, rho))
        Z = np.zeros((len(zs), 1), np.uint64)
        for i, pos in enumerate(zs):
            Z[i, 0] = sum(1 << j for j in pos)
        rows = (2 << rho) - 1
        seen_gap = False
        for trial in range(20):
            m = rng.integers(0, W, size=d)
            p = oracle.make_params(d, r, m, _pow2_b(d))
            k = oracle.keys_direct(p, Z)               # key == bit mask of g_v AND z
            assert oracle.probe_rows(p, rho) == rows
            assert np.all((k[:rows] == 0).any(axis=0)), (rho, trial)
            if rho > 0 and not np.all((k[: rows // 2] == 0).any(axis=0)):
                seen_gap = True
        assert rho == 0 or seen_gap                    # the bound is needed: fewer rows miss some z


@pytest.mark.parametrize("d,r,t", [(64, 6, 1), (64, 12, 2), (96, 14, 2), (90, 21, 3)])
def test_row_restricted_query_equals_linear_scan(d, r, t):
    """Strategy 2 probing only rows v <= 2^(floor(rho/t)+1) - 1 of each part still reports
    exactly the linear-scan answer for every radius rho <= r; its counters are those of the
    probed tables and never exceed the full query's."""
    rng = np.random.default_rng(d + 7 * r)
    words = (d + 63) // 64
    n = 300
    pts = rng.integers(0, 2**63, size=(n, words), dtype=np.uint64)
    if d % 64:
        pts[:, -1] &= np.uint64((1 << (d % 64)) - 1)
    p = oracle.derive_params(d * r + 5, d, r, t=t)
    tables = oracle.build_tables(p, pts)
    for qi in range(20):
        q = pts[rng.integers(0, n)].copy()
        for pos in rng.choice(d, size=rng.integers(0, r + 1), replace=False):
            q[pos >> 6] ^= np.uint64(1) << np.uint64(pos & 63)
        for rho in sorted({0, 1, r // 3, r // 2, r}):
            rows = oracle.probe_rows(p, rho)
            ids, ncoll, ncand = oracle.query(p, pts, tables, q, rho, rows=rows)
            full, fcoll, fcand = oracle.query(p, pts, tables, q, rho)
            assert ids.tolist() == oracle.linear_scan(pts, q, rho).tolist() == full.tolist()
            assert ncoll <= fcoll and ncand <= fcand and ncoll >= ncand >= len(ids)
            if rows == p.W - 1:
                assert (ncoll, ncand) == (fcoll, fcand)


@pytest.mark.parametrize("d,r,t,rep", [(64, 3, 1, 1), (96, 12, 2, 1), (32, 2, 1, 3), (128, 6, 1, 1)])
def test_counters_follow_their_definitions(d, r, t, rep):
    """#Collisions and #Candidates of Sec. 4.1, recomputed from their definitions: the number
    of (table, point) pairs whose key equals the query's in that table, and the number of
    distinct points among them -- with the keys from the Algorithm 2 route and plain numpy
    (the oracle's query takes the direct route's tables and its own merge)."""
    rng = np.random.default_rng(d + r + rep)
    words = (d + 63) // 64
    n = 300
    pts = rng.integers(0, 2**63, size=(n, words), dtype=np.uint64)
    if d % 64:
        pts[:, -1] &= np.uint64((1 << (d % 64)) - 1)
    pts[10:20] = pts[3]                                # repeated points collide in every table
    p = oracle.derive_params(d + 7, d, r, t=t, rep=rep)
    tables = oracle.build_tables(p, pts)
    keys = oracle.keys_fht(p, pts)                     # [T][n]
    for qi in range(12):
        q = pts[rng.integers(0, n)].copy()
        for pos in rng.choice(d, size=rng.integers(0, r + 3), replace=False):
            q[pos >> 6] ^= np.uint64(1) << np.uint64(pos & 63)
        qk = oracle.keys_fht(p, q)[:, 0]
        hit = keys == qk[:, None]                      # [T][n]: point collides with q in the table
        for rows in (0, oracle.probe_rows(p, r // 2)):
            sel = hit if rows == 0 else hit.reshape(p.t, p.L, n)[:, :rows, :].reshape(-1, n)
            ids, ncoll, ncand = oracle.query(p, pts, tables, q, r // 2 if rows else r, rows=rows)
            assert ncoll == int(sel.sum())
            assert ncand == int(sel.any(axis=0).sum())


@pytest.mark.parametrize("d,r,t", [(64, 6, 1), (96, 12, 2), (90, 21, 3)])
def test_listed_query_follows_the_definitions(d, r, t):
    """The query given only the tables it probes: its ids are the linear scan's at the query's
    radius (total recall through the probed rows, Theorem 1 and the pigeonhole of Sec. 3.1),
    and #Collisions / #Candidates are recomputed from their definitions (Sec. 4.1) with the
    Algorithm 2 keys and plain numpy.  A probed table that is not given is an error."""
    rng = np.random.default_rng(d * 3 + r)
    words = (d + 63) // 64
    n = 400
    pts = rng.integers(0, 2**63, size=(n, words), dtype=np.uint64)
    if d % 64:
        pts[:, -1] &= np.uint64((1 << (d % 64)) - 1)
    pts[20:40] = pts[7]
    p = oracle.derive_params(d + 11, d, r, t=t)
    keys = oracle.keys_fht(p, pts)
    for radius in (0, 2, r // 2):
        rows = oracle.probe_rows(p, radius)
        taus = oracle.probed_tables(p, rows)
        tables = {tau: oracle.table(p, pts, tau) for tau in taus}
        for qi in range(6):
            q = pts[rng.integers(0, n)].copy()
            for pos in rng.choice(d, size=rng.integers(0, radius + 2), replace=False):
                q[pos >> 6] ^= np.uint64(1) << np.uint64(pos & 63)
            ids, ncoll, ncand = oracle.query_listed(p, pts, tables, q, radius, rows=rows)
            assert np.array_equal(ids, oracle.linear_scan(pts, q, radius))
            hit = keys[taus] == oracle.keys_fht(p, q)[taus, 0][:, None]
            assert ncoll == int(hit.sum()) and ncand == int(hit.any(axis=0).sum())
        if rows < p.W - 1:
            with pytest.raises(ValueError):
                oracle.query_listed(p, pts, {tau: tables[tau] for tau in taus[1:]}, pts[0], radius, rows=rows)


def test_oracle_routes_agree_on_random_parameters():
    """Lemma 3 (direct route == Algorithm 2) and total recall on parameters drawn at random
    (dimension, radius, parts or copies, seed)."""
    hypothesis = pytest.importorskip("hypothesis")
    st = hypothesis.strategies

    @hypothesis.settings(max_examples=40, deadline=None)
    @hypothesis.given(d=st.integers(1, 200), r=st.integers(0, 12), parts=st.integers(1, 3),
                      rep=st.integers(1, 3), seed=st.integers(0, 2**40))
    def check(d, r, parts, rep, seed):
        t = min(parts, d) if rep == 1 else 1
        if (r * rep) // t > 6:                         # keep W <= 128 so that the case stays fast
            return
        p = oracle.derive_params(seed, d, r, t=t, rep=rep)
        rng = np.random.default_rng(seed % 1000)
        words = (d + 63) // 64
        pts = rng.integers(0, 2**63, size=(8, words), dtype=np.uint64)
        if d % 64:
            pts[:, -1] &= np.uint64((1 << (d % 64)) - 1)
        kd, kf = oracle.keys_direct(p, pts), oracle.keys_fht(p, pts)
        assert np.array_equal(kd, kf)
        y = pts[:1].copy()                              # a point within r of pts[0] collides somewhere
        for pos in rng.choice(d, size=min(d, r), replace=False):
            y[0, pos >> 6] ^= np.uint64(1) << np.uint64(pos & 63)
        assert (oracle.keys_direct(p, y)[:, 0] == kd[:, 0]).any()

    check()


# ---------------------------------------------------------------- classic bit-sampling LSH

def test_classic_key_collides_exactly_when_the_sampled_bits_agree():
    """Eq. 1 on the sampled bits (Sec. 2.2): with b_i = 2^i and distinct samples the key is the
    sampled bit string read as an integer, so two points share a table's key exactly when they
    agree on that table's samples; a coordinate drawn twice counts twice."""
    rng = np.random.default_rng(3)
    d, k = 90, 40
    samples = np.stack([rng.choice(d, size=k, replace=False) for _ in range(30)]).astype(np.uint32)
    cp = oracle.ClassicParams(P, d, samples, np.array([1 << i for i in range(k)], np.uint64))
    x = rng.integers(0, 2**63, size=(200, 2), dtype=np.uint64)
    x[:, 1] &= np.uint64((1 << (d - 64)) - 1)
    y = x.copy()                                       # y differs from x in one random coordinate
    for i, c in enumerate(rng.integers(0, d, size=200)):
        y[i, c >> 6] ^= np.uint64(1) << np.uint64(c & 63)
    kx, ky = oracle.classic_keys(cp, x), oracle.classic_keys(cp, y)
    bx, by = oracle._bits(x, d), oracle._bits(y, d)
    agree = np.stack([(bx[:, s] == by[:, s]).all(axis=1) for s in samples])
    assert np.array_equal(kx == ky, agree) and agree.any() and (~agree).any()
    twice = oracle.ClassicParams(P, d, np.array([[5, 5, 7]], np.uint32), np.array([1, 2, 4], np.uint64))
    pt = np.zeros((1, 2), np.uint64)
    pt[0, 0] = np.uint64((1 << 5) | (1 << 7))
    assert int(oracle.classic_keys(twice, pt)[0, 0]) == 1 + 2 + 4


def test_classic_collision_probability_is_sampling_with_replacement():
    """A pair at distance delta shares a table's key with probability (1 - delta/d)^k when the k
    coordinates are drawn independently (with replacement); drawing them without replacement
    would give C(d - delta, k) / C(d, k), which the tolerance tells apart."""
    from math import comb

    d, k, L = 40, 8, 8000
    cp = oracle.classic_params(77, d, L, k)
    rng = np.random.default_rng(5)
    x = rng.integers(0, 2**40, size=(1, 1), dtype=np.uint64)
    for delta in (1, 4, 10):
        y = x.copy()
        for c in rng.choice(d, size=delta, replace=False):
            y[0, 0] ^= np.uint64(1) << np.uint64(c)
        frac = float((oracle.classic_keys(cp, x) == oracle.classic_keys(cp, y)).mean())
        p = (1 - delta / d) ** k
        se = (p * (1 - p) / L) ** 0.5
        assert abs(frac - p) < 3 * se + 1e-9, (delta, frac, p)
        if delta == 10:
            assert abs(frac - comb(d - delta, k) / comb(d, k)) > 3 * se


def test_classic_rule_k_is_the_smallest_k_reaching_the_false_negative_ratio():
    """k = ceil(log(1 - delta^(1/L)) / log(1 - r/d)) (Sec. 4.1): a point at distance r escapes
    all L tables with probability (1 - (1 - r/d)^k)^L, which first reaches delta at this k."""
    for L in (15, 127, 511, 4094):
        for r, d in ((3, 64), (8, 128), (20, 1024), (6, 64)):
            for delta in (0.1, 0.01):
                k = oracle.classic_rule_k(L, r, d, delta)
                p = 1 - r / d
                assert (1 - p ** k) ** L >= delta * (1 - 1e-9)
                assert k == 1 or (1 - p ** (k - 1)) ** L < delta


def test_classic_query_has_false_negatives_at_about_delta():
    """Classic LSH reports only true neighbours (Strategy 2 verifies), counts each candidate
    once, and misses a point planted at distance r with probability about delta -- the recall
    below 1 of Tables 3 and 4 that covering LSH removes."""
    rng = np.random.default_rng(9)
    d, r, n, L, delta = 64, 6, 400, 127, 0.1
    k = oracle.classic_rule_k(L, r, d, delta)
    cp = oracle.classic_params(21, d, L, k)
    pts = rng.integers(0, 2**63, size=(n, 1), dtype=np.uint64) * np.uint64(2)
    keys = oracle.classic_keys(cp, pts)
    misses = 0
    for i in range(n):
        q = pts[i].copy()
        for c in rng.choice(d, size=r, replace=False):
            q[0] ^= np.uint64(1) << np.uint64(c)
        ids, ncoll, ncand = oracle.classic_query(cp, pts, keys, q, r)
        truth = oracle.linear_scan(pts, q, r)
        assert set(ids.tolist()) <= set(truth.tolist()) and ncand <= ncoll
        misses += int(i not in ids.tolist())
    miss_p = (1 - (1 - r / d) ** k) ** L
    assert abs(misses / n - miss_p) < 4 * (miss_p * (1 - miss_p) / n) ** 0.5 + 0.01, (misses, miss_p)
    assert misses > 0
