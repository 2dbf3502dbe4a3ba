// params.cpp -- the index's random choices (Algorithm 1 permutation and parts,
// Algorithm 2 seed vector b and map/permutation m) and the per-column lists the
// sketch kernels read.
//
// Randomness: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), implemented here
// from its published definition.  Draw order: the permutation pi of [d] when
// t > 1 (Fisher-Yates from the top), then for every part k in turn its map m_k
// followed by its seed vector b_k.  Uniform values below P take the top 50 bits
// of a draw and reject values >= P.
#include <stdint.h>

#include <algorithm>
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

int derive_params(uint64_t seed, uint32_t d, uint32_t t, uint32_t W, std::vector<uint32_t> &perm,
                  std::vector<uint32_t> &part_off, std::vector<uint32_t> &m, std::vector<uint64_t> &b)
{
    if (d == 0 || t == 0 || t > d || W < 2 || (W & (W - 1))) return -1;
    SplitMix64 g(seed);
    perm.resize(d);
    for (uint32_t i = 0; i < d; ++i) perm[i] = i;
    if (t > 1) shuffle(g, perm);
    part_off.resize(t + 1);
    for (uint32_t k = 0; k < t; ++k) part_off[k] = k * (d / t);
    part_off[t] = d;
    m.assign(d, 0);
    b.assign(d, 0);
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

void column_lists(uint32_t d, uint32_t t, uint32_t W, const std::vector<uint32_t> &perm,
                  const std::vector<uint32_t> &part_off, const std::vector<uint32_t> &m,
                  const std::vector<uint64_t> &b, std::vector<uint32_t> &col_off,
                  std::vector<uint32_t> &coord, std::vector<uint64_t> &bval)
{
    // Counting sort of the permuted positions of each part by their column m(i);
    // stable, so a column lists its positions in increasing order.
    col_off.assign((size_t)t * (W + 1), 0);
    coord.assign(d, 0);
    bval.assign(d, 0);
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

}  // namespace fclsh
