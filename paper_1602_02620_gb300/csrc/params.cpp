// params.cpp -- the index's random choices (Algorithm 1 permutation and parts,
// Algorithm 2 seed vector b and map/permutation m) and the per-column lists the
// sketch kernels read.
//
// Randomness: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), implemented here
// from its published definition.  Draw order: the permutation pi of [d] when
// t > 1 (Fisher-Yates from the top), then for every part k in turn its map m_k
// followed by its seed vector b_k.  Uniform values below P take the top 50 bits
// of a draw and reject values >= P.
//
// Replication (Algorithm 1, cr < log n): the vector is repeated rep times, so
// there are D = d * rep positions and position i reads coordinate i mod d (copy
// i / d); it takes no draws and needs t = 1.  Positions then play the role that
// coordinates play without replication.
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace fclsh {

namespace {

class SplitMix64 {
  public:
    explicit SplitMix64(uint64_t seed) : s_(seed) {}
    uint64_t next()
    {
        s_ += 0x9E3779B97F4A7C15ULL;
        uint64_t z = s_;
        z ^= z >> 30;
        z *= 0xBF58476D1CE4E5B9ULL;
        z ^= z >> 27;
        z *= 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
    uint64_t below(uint64_t bound) { return next() % bound; }
    uint64_t residue()   // uniform in [0, P)
    {
        for (;;) {
            uint64_t u = next() >> 14;   // P - 1 has 50 bits
            if (u < kP) return u;
        }
    }

  private:
    uint64_t s_;
};

template <typename T>
void shuffle(SplitMix64 &g, std::vector<T> &a)
{
    for (size_t i = a.size(); i > 1; --i) {
        size_t j = (size_t)g.below(i);
        std::swap(a[i - 1], a[j]);
    }
}

}  // namespace

uint32_t default_parts(uint32_t r)
{
    // One part below radius 10 and two from 10 on (the paper's experimental
    // setting); past 21 the smallest t keeping floor(r/t) <= 10.
    if (r < 10) return 1;
    uint32_t t = 2;
    while (r / t > 10) ++t;
    return t;
}

// Algorithm 1's choice for approximation factor c, reading its log as log2 (the
// covering family has 2^(r+1) tables and a far pair collides in a table with
// probability 2^-distance, so c r = log2 n balances them like classic LSH):
// replicate floor(log2 n / (c r)) times when c r < log2 n, partition into
// ceil(c r / log2 n) parts when c r > log2 n.  The kernels cover at most radius
// 10 per part, so replication is capped at floor(10 / r) copies and t is raised
// until floor(r / t) <= 10; both keep every guarantee (any t and rep are exact).
void algorithm1_rule(uint64_t n, uint32_t r, double c, uint32_t *t, uint32_t *rep)
{
    *t = 1;
    *rep = 1;
    if (r == 0) return;
    const double lg = std::log2((double)(n < 2 ? 2 : n));
    const double cr = c * r;
    uint32_t parts = 1;
    if (cr < lg) {
        uint32_t R = (uint32_t)std::floor(lg / cr);
        if (R > 10 / r) R = 10 / r;
        *rep = R < 1 ? 1 : R;
    } else if (cr > lg) {
        parts = (uint32_t)std::ceil(cr / lg);
    }
    if (*rep == 1) {
        while (r / parts > 10) ++parts;
        *t = parts;
    }
}

int derive_params(uint64_t seed, uint32_t d, uint32_t t, uint32_t rep, uint32_t W, std::vector<uint32_t> &perm,
                  std::vector<uint32_t> &part_off, std::vector<uint32_t> &m, std::vector<uint64_t> &b)
{
    if (d == 0 || t == 0 || t > d || rep == 0 || (rep > 1 && t > 1) || W < 2 || (W & (W - 1))) return -1;
    SplitMix64 g(seed);
    const uint32_t D = d * rep;
    perm.resize(D);
    for (uint32_t i = 0; i < D; ++i) perm[i] = i % d;
    if (t > 1) shuffle(g, perm);
    part_off.resize(t + 1);
    for (uint32_t k = 0; k < t; ++k) part_off[k] = k * (D / t);
    part_off[t] = D;
    m.assign(D, 0);
    b.assign(D, 0);
    std::vector<uint32_t> sigma(W);
    for (uint32_t k = 0; k < t; ++k) {
        const uint32_t lo = part_off[k], dk = part_off[k + 1] - lo;
        if (dk <= W) {                       // specific construction: permutation of the padded columns
            for (uint32_t j = 0; j < W; ++j) sigma[j] = j;
            shuffle(g, sigma);
            std::copy(sigma.begin(), sigma.begin() + dk, m.begin() + lo);
        } else {                             // general construction: map into columns 1..W-1
            for (uint32_t i = 0; i < dk; ++i) m[lo + i] = 1 + (uint32_t)g.below(W - 1);
        }
        for (uint32_t i = 0; i < dk; ++i) b[lo + i] = g.residue();
    }
    return 0;
}

void column_lists(uint32_t D, uint32_t t, uint32_t W, const std::vector<uint32_t> &perm,
                  const std::vector<uint32_t> &part_off, const std::vector<uint32_t> &m,
                  const std::vector<uint64_t> &b, std::vector<uint32_t> &col_off,
                  std::vector<uint32_t> &coord, std::vector<uint64_t> &bval)
{
    // Counting sort of the permuted positions of each part by their column m(i);
    // stable, so a column lists its positions in increasing order.
    col_off.assign((size_t)t * (W + 1), 0);
    coord.assign(D, 0);
    bval.assign(D, 0);
    for (uint32_t k = 0; k < t; ++k) {
        uint32_t *off = col_off.data() + (size_t)k * (W + 1);
        const uint32_t lo = part_off[k], hi = part_off[k + 1];
        std::vector<uint32_t> cnt(W, 0);
        for (uint32_t i = lo; i < hi; ++i) cnt[m[i]]++;
        uint32_t run = lo;
        for (uint32_t j = 0; j < W; ++j) {
            off[j] = run;
            run += cnt[j];
        }
        off[W] = run;
        std::vector<uint32_t> fill(off, off + W);
        for (uint32_t i = lo; i < hi; ++i) {
            uint32_t at = fill[m[i]]++;
            coord[at] = perm[i];
            bval[at] = b[i];
        }
    }
}

void coord_lists(uint32_t d, uint32_t t, uint32_t W, const std::vector<uint32_t> &perm,
                 const std::vector<uint32_t> &part_off, const std::vector<uint32_t> &m,
                 const std::vector<uint64_t> &b, std::vector<uint32_t> &off, std::vector<uint32_t> &col,
                 std::vector<uint64_t> &bval, uint32_t *max_pop)
{
    // The same positions as column_lists, grouped by the coordinate they read
    // (counting sort per part, stable), for a sketch that visits a point's set bits.
    const uint32_t D = (uint32_t)perm.size();
    off.assign((size_t)t * (d + 1), 0);
    col.assign(D, 0);
    bval.assign(D, 0);
    uint32_t pop = 0;
    for (uint32_t k = 0; k < t; ++k) {
        uint32_t *o = off.data() + (size_t)k * (d + 1);
        const uint32_t lo = part_off[k], hi = part_off[k + 1];
        std::vector<uint32_t> cnt(d, 0), colpop(W, 0);
        for (uint32_t i = lo; i < hi; ++i) {
            cnt[perm[i]]++;
            pop = std::max(pop, ++colpop[m[i]]);
        }
        uint32_t run = lo;
        for (uint32_t c = 0; c < d; ++c) {
            o[c] = run;
            run += cnt[c];
        }
        o[d] = run;
        std::vector<uint32_t> fill(o, o + d);
        for (uint32_t i = lo; i < hi; ++i) {
            const uint32_t at = fill[perm[i]]++;
            col[at] = m[i];
            bval[at] = b[i];
        }
    }
    *max_pop = pop;
}

// ---------------------------------------------------------------- classic bit-sampling LSH

// Classic LSH for Hamming space (Sec. 2.2): a hash function samples one coordinate, and
// table j concatenates k of them, g_j = (x_{s_j(1)}, ..., x_{s_j(k)}), keyed by Eq. 1:
// key_j(x) = (sum_i b_i x_{s_j(i)}) mod P with one seed vector b of k entries for every
// table.  k follows the rule of Sec. 4.1, k = ceil(log(1 - delta^(1/L)) / log(1 - r/d)),
// which makes a point at distance r a false negative with probability about delta.
uint32_t classic_rule_k(uint32_t L, uint32_t r, uint32_t d, double delta)
{
    if (r == 0 || r >= d || L == 0 || !(delta > 0.0 && delta < 1.0)) return 0;
    const double num = std::log1p(-std::pow(delta, 1.0 / (double)L));
    const double den = std::log1p(-(double)r / (double)d);
    const double k = std::ceil(num / den);
    return k < 1.0 ? 1u : (k > 8192.0 ? 8192u : (uint32_t)k);
}

// Draw order from `seed`: for table j = 0..L-1 in turn, its k samples s_j(i) = next() mod d
// (coordinates with replacement, as independent draws from the bit-sampling family), then the
// k entries of b, uniform below P.
void classic_params(uint64_t seed, uint32_t d, uint32_t L, uint32_t k, std::vector<uint32_t> &samples,
                    std::vector<uint64_t> &b)
{
    SplitMix64 g(seed);
    samples.resize((size_t)L * k);
    for (size_t i = 0; i < samples.size(); ++i) samples[i] = (uint32_t)g.below(d);
    b.resize(k);
    for (uint32_t i = 0; i < k; ++i) b[i] = g.residue();
}

// Per table: the distinct sampled coordinates, ascending, each with the sum of its b entries
// mod P (a coordinate drawn twice counts twice in Eq. 1), so that key_j(x) = sum over the
// list of bsum x_c mod P.
void classic_lists(uint32_t L, uint32_t k, const std::vector<uint32_t> &samples, const std::vector<uint64_t> &b,
                   std::vector<uint32_t> &off, std::vector<uint32_t> &coord, std::vector<uint64_t> &bsum)
{
    off.assign((size_t)L + 1, 0);
    coord.clear();
    bsum.clear();
    std::vector<std::pair<uint32_t, uint64_t>> row(k);
    for (uint32_t j = 0; j < L; ++j) {
        for (uint32_t i = 0; i < k; ++i) row[i] = {samples[(size_t)j * k + i], b[i]};
        std::sort(row.begin(), row.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
        off[j] = (uint32_t)coord.size();
        for (uint32_t i = 0; i < k; ++i) {
            if (!coord.empty() && coord.size() > off[j] && coord.back() == row[i].first) {
                bsum.back() = add_mod_p(bsum.back(), row[i].second);
            } else {
                coord.push_back(row[i].first);
                bsum.push_back(row[i].second);
            }
        }
    }
    off[L] = (uint32_t)coord.size();
}

}  // namespace fclsh
