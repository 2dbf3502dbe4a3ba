/*
 * workloads.c -- seeded synthetic bit-vector generators shared by the tests,
 * the benchmark and the oracle checks.  Holds none of the index's arithmetic:
 * it only produces input points and queries.
 *
 * Randomness: counter-based SplitMix64.  U(key, i) is the i-th output of a
 * SplitMix64 generator whose state starts at `key` (Steele, Lea & Flood,
 * OOPSLA 2014): mix(key + (i+1) * GAMMA).  Every value therefore depends only
 * on (seed, stream, counter), so any slice can be generated on its own.
 *
 * Bernoulli(p) bits use 16-bit thresholds: a 64-bit draw gives four 16-bit
 * uniforms u, and a bit is set iff u < thr, thr = round(p * 65536).
 * Points are packed LSB-first: coordinate j is word j/64, bit j%64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t U(uint64_t key, uint64_t i)
{
    return mix64(key + (i + 1) * GAMMA);
}

/* Key of stream `s` under `seed`. */
uint64_t wl_stream_key(uint64_t seed, uint64_t s)
{
    return U(seed, s);
}

static inline uint32_t words_of(uint32_t d) { return (d + 63) / 64; }

static inline uint64_t last_mask(uint32_t d)
{
    return (d % 64) ? ((1ULL << (d % 64)) - 1) : ~0ULL;
}

/* n points of d i.i.d. Bernoulli(1/2) bits: word w of point i = U(key, i*words + w). */
void wl_uniform(uint64_t key, uint64_t first, uint64_t n, uint32_t d, uint64_t *out)
{
    uint32_t words = words_of(d);
    uint64_t mask = last_mask(d);
    for (uint64_t i = 0; i < n; i++) {
        uint64_t gi = first + i;
        for (uint32_t w = 0; w < words; w++) out[i * words + w] = U(key, gi * words + w);
        out[i * words + words - 1] &= mask;
    }
}

/* d Bernoulli(thr/65536) bits for row `gi` of stream `key`, XORed into `row`. */
static void bernoulli_row(uint64_t key, uint64_t gi, uint32_t d, uint32_t thr, uint64_t *row)
{
    uint32_t groups = (d + 3) / 4;
    for (uint32_t g = 0; g < groups; g++) {
        uint64_t u = U(key, gi * groups + g);
        for (uint32_t s = 0; s < 4; s++) {
            uint32_t j = 4 * g + s;
            if (j >= d) break;
            if (((u >> (16 * s)) & 0xFFFF) < thr) row[j >> 6] ^= 1ULL << (j & 63);
        }
    }
}

/* n points of d i.i.d. Bernoulli(thr/65536) bits. */
void wl_bernoulli(uint64_t key, uint64_t first, uint64_t n, uint32_t d, uint32_t thr, uint64_t *out)
{
    uint32_t words = words_of(d);
    memset(out, 0, sizeof(uint64_t) * n * words);
    for (uint64_t i = 0; i < n; i++) bernoulli_row(key, first + i, d, thr, out + i * words);
}

/*
 * Clustered points: point i = centres[U(ckey, i) % nc] XOR noise, noise bits
 * Bernoulli(thr_i/65536).  thr_i = thr_lo + U(tkey, i) % (thr_hi - thr_lo + 1)
 * (a per-point noise level; thr_lo == thr_hi gives a fixed level).
 * centre_out (may be NULL) receives the centre index of each point.
 */
void wl_clustered(uint64_t ckey, uint64_t nkey, uint64_t tkey, uint64_t first, uint64_t n, uint32_t d,
                  const uint64_t *centres, uint32_t nc, uint32_t thr_lo, uint32_t thr_hi,
                  uint64_t *out, uint32_t *centre_out)
{
    uint32_t words = words_of(d);
    for (uint64_t i = 0; i < n; i++) {
        uint64_t gi = first + i;
        uint32_t c = (uint32_t)(U(ckey, gi) % nc);
        uint32_t thr = thr_lo + (uint32_t)(U(tkey, gi) % (uint64_t)(thr_hi - thr_lo + 1));
        uint64_t *row = out + i * words;
        memcpy(row, centres + (uint64_t)c * words, sizeof(uint64_t) * words);
        bernoulli_row(nkey, gi, d, thr, row);
        if (centre_out) centre_out[i] = c;
    }
}

/* Flip k distinct coordinates of `row`, positions drawn from U(key, base + j) % d with rejection. */
static void flip_distinct(uint64_t key, uint64_t base, uint32_t d, uint32_t k, uint64_t *row)
{
    uint32_t *pos = (uint32_t *)malloc(sizeof(uint32_t) * (k ? k : 1));
    uint32_t got = 0;
    uint64_t j = 0;
    if (k > d) k = d;
    while (got < k) {
        uint32_t p = (uint32_t)(U(key, base + j++) % d);
        int dup = 0;
        for (uint32_t a = 0; a < got; a++) if (pos[a] == p) { dup = 1; break; }
        if (dup) continue;
        pos[got++] = p;
        row[p >> 6] ^= 1ULL << (p & 63);
    }
    free(pos);
}

/*
 * Planted queries: query i copies data point src_i = U(key, 3i) % n and flips
 * k_i = kmin + U(key, 3i+1) % (kmax - kmin + 1) distinct coordinates, drawn
 * from the sub-stream U(U(key, 3i+2), .).  src_out/k_out (may be NULL) record
 * the source and the distance.
 */
void wl_planted(uint64_t key, uint64_t first, uint64_t nq, const uint64_t *pts, uint64_t n, uint32_t d,
                uint32_t kmin, uint32_t kmax, uint64_t *out, uint32_t *src_out, uint32_t *k_out)
{
    uint32_t words = words_of(d);
    for (uint64_t i = 0; i < nq; i++) {
        uint64_t gi = first + i;
        uint32_t src = (uint32_t)(U(key, 3 * gi) % n);
        uint32_t k = kmin + (uint32_t)(U(key, 3 * gi + 1) % (uint64_t)(kmax - kmin + 1));
        uint64_t sub = U(key, 3 * gi + 2);
        memcpy(out + i * words, pts + (uint64_t)src * words, sizeof(uint64_t) * words);
        flip_distinct(sub, 0, d, k, out + i * words);
        if (src_out) src_out[i] = src;
        if (k_out) k_out[i] = k;
    }
}

/*
 * Near-duplicates in place: for i = 1..n-1 in order, with probability
 * thr/65536 (first 16 bits of U(key, 4i)), point i becomes a copy of the
 * earlier point src = U(key, 4i+1) % i with k = kmin + U(key, 4i+2) % (kmax-kmin+1)
 * distinct coordinates flipped (sub-stream U(key, 4i+3)).  Returns the count.
 */
uint64_t wl_near_duplicates(uint64_t key, uint64_t *pts, uint64_t n, uint32_t d, uint32_t thr,
                            uint32_t kmin, uint32_t kmax)
{
    uint32_t words = words_of(d);
    uint64_t cnt = 0;
    for (uint64_t i = 1; i < n; i++) {
        if ((U(key, 4 * i) & 0xFFFF) >= thr) continue;
        uint64_t src = U(key, 4 * i + 1) % i;
        uint32_t k = kmin + (uint32_t)(U(key, 4 * i + 2) % (uint64_t)(kmax - kmin + 1));
        memcpy(pts + i * words, pts + src * words, sizeof(uint64_t) * words);
        flip_distinct(U(key, 4 * i + 3), 0, d, k, pts + i * words);
        cnt++;
    }
    return cnt;
}

/* Uniform double in [0, 1) from the top 53 bits of a draw. */
static inline double unit(uint64_t u) { return (double)(u >> 11) * (1.0 / 9007199254740992.0); }

/*
 * Sparse high-dimensional points with skewed coordinate popularity (the shape of
 * bag-of-words and rating vectors): point gi draws its sub-stream key k = U(key, gi),
 * sets L = min(d/2, lmin + floor(-lmean * ln(1 - u))) coordinates with u = unit(U(k, 0))
 * (a geometric-like length), each c = floor(d * v^2) with v = unit(U(k, j)), j = 1, 2, ...,
 * skipping coordinates already set (low coordinates are the popular ones).
 */
void wl_sparse_skewed(uint64_t key, uint64_t first, uint64_t n, uint32_t d, uint32_t lmin, uint32_t lmean,
                      uint64_t *out)
{
    uint32_t words = words_of(d);
    memset(out, 0, sizeof(uint64_t) * n * words);
    for (uint64_t i = 0; i < n; i++) {
        uint64_t k = U(key, first + i);
        uint64_t *row = out + i * words;
        double len = (double)lmin - (double)lmean * log(1.0 - unit(U(k, 0)));
        uint32_t L = len > (double)(d / 2) ? d / 2 : (uint32_t)len;
        uint32_t got = 0;
        for (uint64_t j = 1; got < L; j++) {
            double v = unit(U(k, j));
            uint32_t c = (uint32_t)((double)d * v * v);
            if (c >= d) c = d - 1;
            if (row[c >> 6] >> (c & 63) & 1ULL) continue;
            row[c >> 6] |= 1ULL << (c & 63);
            got++;
        }
    }
}

/* n draws U(key, first + i) (raw 64-bit values, for request streams). */
void wl_raw(uint64_t key, uint64_t first, uint64_t n, uint64_t *out)
{
    for (uint64_t i = 0; i < n; i++) out[i] = U(key, first + i);
}
