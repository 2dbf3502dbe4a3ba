// hash.cu -- Algorithm 2 on the GPU: all W-1 keys of every point of one part.
//
// For a point q and part k (Sec. 3.2, "Fast computation of hash functions"):
//   sketch   t_j = sum_{i in part k, m(i) = j} b_i q_i  (mod P)
//   transform y = H t (Walsh-Hadamard, Sylvester order)
//   finish   h_v = ((S - y_v) / 2) mod P, S = y_0 = sum_j t_j, v = 1..W-1
// which by Lemma 3 equals p(g_v AND q) of Eq. (1).  Reducing t_j mod P first
// changes no key and keeps |y| <= W P < 2^61, so 64-bit integers are exact.
//
// Kernel shapes:
//   W <= 32   one thread per point; the whole transform in registers.
//   W >= 64   a tile of NP points in shared memory laid out [j][p] (p fastest),
//             W/32 threads per point, 32 values per thread.  The log2(W) butterfly
//             levels are split into 2 or 3 register phases (each at most 5 levels);
//             between phases the values pass through shared memory once.  The first
//             phase gathers the sketch straight into registers (no scatter), the last
//             phase applies the finish and stores keys table-major, coalesced over
//             the NP consecutive points.
#include "common.cuh"

namespace fclsh {

namespace {

// In-register Walsh-Hadamard transform of K values (unnormalised, natural order).
template <int K>
__device__ __forceinline__ void wht_regs(uint64_t *v)
{
#pragma unroll
    for (int h = 1; h < K; h <<= 1)
#pragma unroll
        for (int i = 0; i < K; i += 2 * h)
#pragma unroll
            for (int j = i; j < i + h; ++j) {
                uint64_t a = v[j], c = v[j + h];
                v[j] = a + c;
                v[j + h] = a - c;
            }
}

// Column data of one part staged in shared memory: offsets relative to the part.
struct ColsSmem {
    const uint32_t *off;     // [W+1]
    const uint32_t *coord;   // [dk]
    const uint64_t *bval;    // [dk]
};

// t_j for one point whose words are at x (global, read through L1).
__device__ __forceinline__ uint64_t sketch_column(const ColsSmem &c, uint32_t j, const uint64_t *__restrict__ x)
{
    uint64_t s = 0;
    const uint32_t e1 = c.off[j + 1];
    for (uint32_t e = c.off[j]; e < e1; ++e) {
        const uint32_t bit = c.coord[e];
        const uint64_t w = __ldg(x + (bit >> 6));
        const uint64_t take = 0ULL - ((w >> (bit & 63)) & 1ULL);
        s = add_mod_p(s, c.bval[e] & take);
    }
    return s;
}

// Stage the part's column lists into shared memory (all threads, then a barrier by the caller).
__device__ __forceinline__ ColsSmem stage_cols(const PartCols &pc, uint32_t W, void *smem_base)
{
    const uint32_t base = pc.col_off[0];
    const uint32_t dk = pc.col_off[W] - base;
    uint64_t *bv = reinterpret_cast<uint64_t *>(smem_base);
    uint32_t *off = reinterpret_cast<uint32_t *>(bv + dk);
    uint32_t *coord = off + (W + 1);
    for (uint32_t i = threadIdx.x; i <= W; i += blockDim.x) off[i] = pc.col_off[i] - base;
    for (uint32_t i = threadIdx.x; i < dk; i += blockDim.x) {
        coord[i] = pc.coord[base + i];
        bv[i] = pc.bval[base + i];
    }
    return ColsSmem{off, coord, bv};
}

__host__ __device__ constexpr size_t cols_smem_bytes(uint32_t W, uint32_t dk)
{
    return (size_t)dk * 8 + ((size_t)W + 1 + dk) * 4 + 8;
}

// Gather modes of the sketch.  GENERAL walks a column's list (general
// construction, several coordinates per column).  With the specific construction a
// column holds at most one coordinate, packed with its seed value as
// b | coord << 50 (b = 0 for an empty column): PACKED_REG keeps the point's
// words in registers (d <= 256), PACKED_LDG reads them through L1.
enum GatherMode { GENERAL = 0, PACKED_REG = 1, PACKED_LDG = 2, SCATTER = 3 };

__device__ __forceinline__ const uint64_t *stage_packed(const PartCols &pc, uint32_t W, void *smem_base)
{
    uint64_t *pk = reinterpret_cast<uint64_t *>(smem_base);
    const uint32_t base = pc.col_off[0];
    for (uint32_t j = threadIdx.x; j < W; j += blockDim.x) {
        const uint32_t e0 = pc.col_off[j], e1 = pc.col_off[j + 1];
        pk[j] = e1 > e0 ? (pc.bval[e0] | ((uint64_t)pc.coord[e0] << 50)) : 0ULL;
    }
    (void)base;
    return pk;
}

struct PointRegs {
    uint64_t x0, x1, x2, x3;
    __device__ __forceinline__ uint64_t word(uint32_t c) const
    {
        const uint32_t w = c >> 6;
        return w < 2 ? (w == 0 ? x0 : x1) : (w == 2 ? x2 : x3);
    }
};

__device__ __forceinline__ uint64_t packed_value(uint64_t pk, uint64_t word_of_coord)
{
    const uint32_t c = (uint32_t)(pk >> 50);
    const uint64_t take = 0ULL - ((word_of_coord >> (c & 63)) & 1ULL);
    return pk & kMask50 & take;
}

// ------------------------------------------------------------------ W <= 32

template <int LOGW>
__global__ void __launch_bounds__(128) hash_small_kernel(const uint64_t *__restrict__ pts, uint64_t cnt,
                                                         uint32_t words, PartCols pc, uint64_t *__restrict__ keys,
                                                         uint64_t ld)
{
    constexpr int W = 1 << LOGW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const ColsSmem cols = stage_cols(pc, W, smem_raw);
    __syncthreads();
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const uint64_t *x = pts + i * words;
    uint64_t v[W];
    uint64_t S = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        v[j] = sketch_column(cols, j, x);
        S += v[j];
    }
    wht_regs<W>(v);
#pragma unroll
    for (int j = 1; j < W; ++j) keys[(uint64_t)(j - 1) * ld + i] = finish_key(S, v[j]);
}

// W <= 32 with the scatter sketch (hash_tile 3, or parts too long for staged
// column lists): 128 points per block, sketch [j][p] in shared memory.  Warp w
// walks the words of its 32 points (a lane a word), and each set coordinate adds
// the seed values of its positions to their columns; then thread p transforms its
// point's sketch in registers.  Sums stay below 2^64 while no column of the part
// holds more than 16,383 positions (checked by the host).
template <int LOGW>
__global__ void __launch_bounds__(128, 4) hash_small_scatter_kernel(const uint64_t *__restrict__ pts, uint64_t cnt,
                                                                 uint32_t words, CoordLists cl,
                                                                 uint64_t *__restrict__ keys, uint64_t ld)
{
    constexpr int W = 1 << LOGW, NP = 128;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long *sk = reinterpret_cast<unsigned long long *>(smem_raw);   // [W][NP]
    for (uint32_t i = threadIdx.x; i < (uint32_t)(W * NP); i += NP) sk[i] = 0ULL;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t p0 = blockIdx.x * (uint64_t)NP;
    for (uint32_t pi = 0; pi < 32; ++pi) {
        const uint32_t p = warp * 32 + pi;
        if (p0 + p >= cnt) break;
        if (cl.pidx) {   // the point's set coordinates are listed: a lane per coordinate
            const uint32_t *ci = cl.pidx + cl.pstart[p0 + p];
            const uint32_t len = cl.plen[p0 + p];
            for (uint32_t j = lane; j < len; j += 32) {
                const uint32_t c = ci[j];
                const uint32_t e1 = __ldg(cl.off + c + 1);
                for (uint32_t e = __ldg(cl.off + c); e < e1; ++e)
                    atomicAdd(sk + (size_t)__ldg(cl.col + e) * NP + p, (unsigned long long)__ldg(cl.b + e));
            }
            continue;
        }
        const uint64_t *x = pts + (p0 + p) * words;
        for (uint32_t w0 = lane; w0 < words; w0 += 128) {   // four words in flight per lane
            uint64_t wv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) wv[u] = w0 + 32 * u < words ? __ldg(x + w0 + 32 * u) : 0ULL;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t w = w0 + 32 * u;
                uint64_t bits = wv[u];
                if (w == words - 1 && (cl.d & 63)) bits &= (1ULL << (cl.d & 63)) - 1;   // coordinates < d only
                while (bits) {
                    const uint32_t c = w * 64 + (uint32_t)(__ffsll((long long)bits) - 1);
                    bits &= bits - 1;
                    const uint32_t e1 = __ldg(cl.off + c + 1);
                    for (uint32_t e = __ldg(cl.off + c); e < e1; ++e)
                        atomicAdd(sk + (size_t)__ldg(cl.col + e) * NP + p, (unsigned long long)__ldg(cl.b + e));
                }
            }
        }
    }
    __syncwarp();
    const uint64_t i = p0 + threadIdx.x;
    if (i >= cnt) return;
    uint64_t v[W];
    uint64_t S = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        v[j] = mod_p(sk[(size_t)j * NP + threadIdx.x]);
        S += v[j];
    }
    wht_regs<W>(v);
#pragma unroll
    for (int j = 1; j < W; ++j) keys[(uint64_t)(j - 1) * ld + i] = finish_key(S, v[j]);
}

// ------------------------------------------------------------------ direct route (bcLSH)

// The O(d'L) route of Eq. (1) on CUDA cores, without the transform: key v of a point
// is sum over its set positions i of b_i * <a(m(i)), v> mod P, i.e. Eq. (1) applied to
// g_v AND x (the basic covering construction; Lemma 3's other side).  A block takes
// kDirectPoints points: it lists every point's set positions (column, seed value)
// in shared memory through the coordinate lists, then each thread computes keys
// (table v, point p) with p fastest, so that a warp's stores cover consecutive points.
constexpr int kDirectPoints = 4;
constexpr int kDirectThreads = 256;

__global__ void __launch_bounds__(kDirectThreads) hash_direct_kernel(const uint64_t *__restrict__ pts, uint64_t cnt,
                                                                     uint32_t words, CoordLists cl, uint32_t W,
                                                                     uint32_t maxpos, uint64_t *__restrict__ keys,
                                                                     uint64_t ld)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *lb = reinterpret_cast<uint64_t *>(smem_raw);                       // [kDirectPoints][maxpos]
    uint16_t *lc = reinterpret_cast<uint16_t *>(lb + (size_t)kDirectPoints * maxpos);
    __shared__ uint32_t len[kDirectPoints];
    const uint64_t p0 = blockIdx.x * (uint64_t)kDirectPoints;
    if (threadIdx.x < kDirectPoints) len[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t real = (uint32_t)(cnt - p0 < (uint64_t)kDirectPoints ? cnt - p0 : (uint64_t)kDirectPoints);
    for (uint32_t it = threadIdx.x; it < real * words; it += blockDim.x) {
        const uint32_t p = it / words, w = it - p * words;
        uint64_t bits = __ldg(pts + p0 * words + it);
        if (w == words - 1 && (cl.d & 63)) bits &= (1ULL << (cl.d & 63)) - 1;   // coordinates < d only
        while (bits) {
            const uint32_t c = w * 64 + (uint32_t)(__ffsll((long long)bits) - 1);
            bits &= bits - 1;
            const uint32_t e1 = __ldg(cl.off + c + 1);
            for (uint32_t e = __ldg(cl.off + c); e < e1; ++e) {
                const uint32_t at = atomicAdd(&len[p], 1u);   // < maxpos: a point has at most the part's positions
                if (!FCLSH_CHECK(at < maxpos, 0x0204)) continue;
                lb[(size_t)p * maxpos + at] = __ldg(cl.b + e);
                lc[(size_t)p * maxpos + at] = (uint16_t)__ldg(cl.col + e);
            }
        }
    }
    __syncthreads();
    const uint32_t pairs = (W - 1) * (uint32_t)kDirectPoints;
    for (uint32_t j = threadIdx.x; j < pairs; j += blockDim.x) {
        const uint32_t p = j % kDirectPoints, v = j / kDirectPoints + 1;
        if (p >= real) continue;
        const uint64_t *b = lb + (size_t)p * maxpos;
        const uint16_t *col = lc + (size_t)p * maxpos;
        uint64_t key = 0;
        for (uint32_t e = 0, n = len[p]; e < n; ++e)
            if (__popc(v & col[e]) & 1) key = add_mod_p(key, b[e]);   // (g_v AND x)_i = <a(m(i)), v> x_i
        keys[(uint64_t)(v - 1) * ld + p0 + p] = key;
    }
}

// ------------------------------------------------------------------ classic bit-sampling LSH

// Keys of classic LSH (Sec. 2.2, Eq. 1 on k sampled coordinates): a block takes 128 points,
// stages their words in shared memory (rows padded by one word) when they fit, and thread p
// computes point p's key in every table of [tau0, tau0 + nt) from the table's list of
// distinct sampled coordinates and summed seed values: sum of bsum over the set ones, mod P
// (the sum of at most 8,192 values below 2^50 stays below 2^63).  A warp's stores cover 32
// consecutive points of one table.
constexpr int kClassicPoints = 128;
constexpr uint32_t kClassicSmemWords = 64;   // points of up to 64 words are staged

__global__ void __launch_bounds__(kClassicPoints) classic_hash_kernel(const uint64_t *__restrict__ pts, uint64_t cnt,
                                                                      uint32_t words, const uint32_t *__restrict__ off,
                                                                      const uint32_t *__restrict__ coord,
                                                                      const uint64_t *__restrict__ bsum, uint32_t tau0,
                                                                      uint32_t nt, uint64_t *__restrict__ keys,
                                                                      uint64_t ld)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *xs = reinterpret_cast<uint64_t *>(smem_raw);   // [kClassicPoints][words + 1] when staged
    const uint64_t p0 = blockIdx.x * (uint64_t)kClassicPoints;
    const uint32_t real = (uint32_t)(cnt - p0 < (uint64_t)kClassicPoints ? cnt - p0 : (uint64_t)kClassicPoints);
    const bool staged = words <= kClassicSmemWords;
    const uint32_t stride = words + 1;
    if (staged) {
        for (uint32_t it = threadIdx.x; it < real * words; it += blockDim.x) {
            const uint32_t p = it / words, w = it - p * words;
            xs[(size_t)p * stride + w] = __ldg(pts + p0 * words + it);
        }
        __syncthreads();
    }
    const uint32_t p = threadIdx.x;
    if (p >= real) return;
    const uint64_t *xg = pts + (p0 + p) * words;
    const uint64_t *xsm = xs + (size_t)p * stride;
    for (uint32_t j = 0; j < nt; ++j) {
        const uint32_t e0 = __ldg(off + tau0 + j), e1 = __ldg(off + tau0 + j + 1);
        uint64_t s = 0;
        for (uint32_t e = e0; e < e1; ++e) {
            const uint32_t c = __ldg(coord + e);
            if (!FCLSH_CHECK((c >> 6) < words, 0x0203)) continue;
            const uint64_t w = staged ? xsm[c >> 6] : __ldg(xg + (c >> 6));
            s += __ldg(bsum + e) & (0ULL - ((w >> (c & 63)) & 1ULL));
        }
        keys[(uint64_t)j * ld + p0 + p] = mod_p(s);
    }
}

// ------------------------------------------------------------------ W >= 64

template <int LOGW> struct TileCfg;
//                      points/tile  phases: butterfly levels per register phase   smem swizzle mask
template <> struct TileCfg<6>  { static constexpr int NP = 128, NPH = 2, B0 = 3, B1 = 3, B2 = 0; static constexpr uint32_t M = 0; };
template <> struct TileCfg<7>  { static constexpr int NP = 64,  NPH = 2, B0 = 3, B1 = 4, B2 = 0; static constexpr uint32_t M = 0; };
template <> struct TileCfg<8>  { static constexpr int NP = 32,  NPH = 2, B0 = 4, B1 = 4, B2 = 0; static constexpr uint32_t M = 0; };
template <> struct TileCfg<9>  { static constexpr int NP = 16,  NPH = 2, B0 = 4, B1 = 5, B2 = 0; static constexpr uint32_t M = 0; };
template <> struct TileCfg<10> { static constexpr int NP = 8,   NPH = 2, B0 = 5, B1 = 5, B2 = 0; static constexpr uint32_t M = 0x20; };
template <> struct TileCfg<11> { static constexpr int NP = 8,   NPH = 3, B0 = 5, B1 = 3, B2 = 3; static constexpr uint32_t M = 0x24; };

// A tile of NP_ points: TileCfg's NP (the default) or twice that (a wider tile).
template <int LOGW, int NP_ = TileCfg<LOGW>::NP>
struct Tile {
    using C = TileCfg<LOGW>;
    static constexpr int W = 1 << LOGW;
    static constexpr int NP = NP_;
    static constexpr int NT = NP * W / 32;            // threads per block
    static constexpr size_t VALUES_BYTES = (size_t)W * NP * 8;
    // blocks per SM the register budget is sized for (forcing 3 spills at 80 registers)
    static constexpr int MINB = VALUES_BYTES <= 64 * 1024 ? 2 : 1;
    // the row swizzle matters only when a half-warp spans two rows (NP = 8)
    static constexpr uint32_t M = NP == 8 ? C::M : 0u;
};

// Points per tile for the tile choice (0: default, 1: twice that where it fits).
template <int LOGW>
constexpr int tile_points(uint32_t choice)
{
    constexpr int np = TileCfg<LOGW>::NP;
    return (choice == 1 && (size_t)(1 << LOGW) * 2 * np * 8 <= 128 * 1024) ? 2 * np : np;
}

// Shared-memory slot of value j of point p.  With NP = 8 a half-warp touches two
// rows; flipping bit 0 of the row by the parity of (j & M) puts those two rows in
// opposite halves of the 32 banks in every phase (a bijection: it swaps row pairs).
template <int NP, uint32_t M>
__device__ __forceinline__ uint32_t slot(uint32_t j, uint32_t p)
{
    uint32_t a = j * NP + p;
    if (M) a ^= (uint32_t)(__popc(j & M) & 1) * NP;
    return a;
}

// j of the k-th value along butterfly levels [LO, LO+B) in the group `other`
// (the index over the remaining LOGW-B bits of j).
template <int LO, int B>
__device__ __forceinline__ uint32_t jidx(uint32_t other, uint32_t k)
{
    return ((other >> LO) << (LO + B)) | (k << LO) | (other & ((1u << LO) - 1u));
}

// MODE 0: gather the sketch, transform, write to smem.  1: smem -> transform -> smem.
// 2: smem -> transform -> finish -> global keys.
template <int LOGW, int NP, int LO, int B, int MODE, int GM>
__device__ __forceinline__ void phase(uint64_t *sm, const uint64_t *S_sm, unsigned long long *S_acc, uint32_t p,
                                      uint32_t tp, const ColsSmem &cols, const uint64_t *pk, const PointRegs &xr,
                                      const uint64_t *__restrict__ x, bool valid, uint64_t *__restrict__ keys,
                                      uint64_t ld, uint64_t gp)
{
    using T = Tile<LOGW, NP>;
    constexpr int K = 1 << B, G = 32 / K;
    uint64_t v[32];
    uint64_t part = 0;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const uint32_t other = tp * G + g;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const uint32_t j = jidx<LO, B>(other, k);
            if (MODE == 0) {
                uint64_t tj;
                if (GM == SCATTER) {
                    tj = mod_p(sm[slot<T::NP, T::M>(j, p)]);
                } else if (GM == GENERAL) {
                    tj = valid ? sketch_column(cols, j, x) : 0;
                } else {
                    const uint64_t pj = pk[j];
                    const uint32_t c = (uint32_t)(pj >> 50);
                    tj = packed_value(pj, GM == PACKED_REG ? xr.word(c) : (valid ? __ldg(x + (c >> 6)) : 0ULL));
                }
                v[g * K + k] = tj;
                part += tj;
            } else {
                v[g * K + k] = sm[slot<T::NP, T::M>(j, p)];
            }
        }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) wht_regs<K>(v + g * K);
    if (MODE == 0) atomicAdd(S_acc + p, (unsigned long long)part);
    if (MODE == 2) {
        const uint64_t S = S_sm[p];
        if (valid) {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const uint32_t other = tp * G + g;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const uint32_t j = jidx<LO, B>(other, k);
                    if (j != 0 && FCLSH_CHECK(gp < ld, 0x0201)) keys[(uint64_t)(j - 1) * ld + gp] = finish_key(S, v[g * K + k]);
                }
            }
        }
    } else {
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const uint32_t other = tp * G + g;
#pragma unroll
            for (int k = 0; k < K; ++k) sm[slot<T::NP, T::M>(jidx<LO, B>(other, k), p)] = v[g * K + k];
        }
    }
}

// The tile's sketch by scattering (SCATTER mode): zero the values, then every
// thread takes (point, word) items, p-major so that a warp reads consecutive words
// of one point, and adds the seed values of each set coordinate's positions to
// their columns with shared-memory atomics.
template <int NP, uint32_t M>
__device__ __forceinline__ void scatter_sketch(uint64_t *sm, uint32_t W, const uint64_t *__restrict__ pts,
                                               uint64_t cnt, uint32_t words, uint64_t p0, CoordLists cl,
                                               unsigned char *stage)
{
    for (uint32_t i = threadIdx.x; i < W * (uint32_t)NP; i += blockDim.x) sm[i] = 0ULL;
    if (cl.stage) {   // the part's lists into shared memory: the set bits' lookups stay on chip
        uint64_t *s_b = reinterpret_cast<uint64_t *>(stage);
        uint32_t *s_col = reinterpret_cast<uint32_t *>(stage + (((size_t)cl.npos * 8 + 15) & ~(size_t)15));
        uint32_t *s_off = s_col + ((cl.npos + 3) & ~3u);
        for (uint32_t i = threadIdx.x; i < cl.npos; i += blockDim.x) {
            s_b[i] = __ldg(cl.b + cl.pos0 + i);
            s_col[i] = __ldg(cl.col + cl.pos0 + i);
        }
        for (uint32_t i = threadIdx.x; i <= cl.d; i += blockDim.x) s_off[i] = __ldg(cl.off + i) - cl.pos0;
        cl.b = s_b;
        cl.col = s_col;
        cl.off = s_off;
    }
    __syncthreads();
    const uint64_t real = cnt - p0 < (uint64_t)NP ? cnt - p0 : (uint64_t)NP;
    if (cl.pidx) {   // the points' set coordinates are listed: threads take (point, coordinate)
        // items of the whole tile at once, so that their dependent loads overlap
        __shared__ uint32_t s_first[NP + 1];   // item of the tile where point p's coordinates start
        __shared__ uint64_t s_start[NP];
        if (threadIdx.x < (uint32_t)real) {
            s_start[threadIdx.x] = cl.pstart[p0 + threadIdx.x];
            s_first[threadIdx.x + 1] = cl.plen[p0 + threadIdx.x];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_first[0] = 0;
            for (uint32_t p = 1; p <= (uint32_t)real; ++p) s_first[p] += s_first[p - 1];
        }
        __syncthreads();
        const uint32_t total = s_first[real];
        for (uint32_t it = threadIdx.x; it < total; it += blockDim.x) {
            uint32_t lo = 0, hi = (uint32_t)real;   // the last point p with s_first[p] <= it
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (s_first[mid] <= it) lo = mid;
                else hi = mid;
            }
            const uint32_t p = lo;
            const uint32_t c = cl.pidx[s_start[p] + (it - s_first[p])];
            const uint32_t e1 = cl.off[c + 1];
            for (uint32_t e = cl.off[c]; e < e1; ++e) {
                const uint32_t col = cl.col[e];
                if (FCLSH_CHECK(col < W, 0x0202))
                    atomicAdd(reinterpret_cast<unsigned long long *>(sm + slot<NP, M>(col, p)),
                              (unsigned long long)cl.b[e]);
            }
        }
        return;
    }
    // items of the tile's real points only; eight words in flight per thread
    const uint32_t items = (uint32_t)real * words;
    constexpr int U = 8;
    for (uint32_t it0 = threadIdx.x; it0 < items; it0 += U * blockDim.x) {
        uint64_t wv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t it = it0 + u * blockDim.x;
            wv[u] = it < items ? __ldg(pts + p0 * words + it) : 0ULL;   // the tile's rows are contiguous
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t it = it0 + u * blockDim.x;
            uint64_t bits = wv[u];
            if (!bits) continue;
            const uint32_t p = it / words, w = it - p * words;
            if (w == words - 1 && (cl.d & 63)) bits &= (1ULL << (cl.d & 63)) - 1;   // coordinates < d only
            while (bits) {
                const uint32_t c = w * 64 + (uint32_t)(__ffsll((long long)bits) - 1);
                bits &= bits - 1;
                const uint32_t e1 = cl.off[c + 1];
                for (uint32_t e = cl.off[c]; e < e1; ++e)
                    atomicAdd(reinterpret_cast<unsigned long long *>(sm + slot<NP, M>(cl.col[e], p)),
                              (unsigned long long)cl.b[e]);
            }
        }
    }
}

template <int LOGW, int NP, int GM>
__global__ void __launch_bounds__(Tile<LOGW, NP>::NT, Tile<LOGW, NP>::MINB) hash_tile_kernel(const uint64_t *__restrict__ pts, uint64_t cnt,
                                                                    uint32_t words, PartCols pc, CoordLists cl,
                                                                    uint64_t *__restrict__ keys, uint64_t ld)
{
    using T = Tile<LOGW, NP>;
    using C = typename T::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *sm = reinterpret_cast<uint64_t *>(smem_raw);
    unsigned long long *S_acc = reinterpret_cast<unsigned long long *>(sm + (size_t)T::W * T::NP);
    ColsSmem cols{};
    const uint64_t *pk = nullptr;
    if (GM == SCATTER)
        scatter_sketch<T::NP, T::M>(sm, T::W, pts, cnt, words, blockIdx.x * (uint64_t)T::NP, cl,
                                    reinterpret_cast<unsigned char *>(S_acc + T::NP));
    else if (GM == GENERAL)
        cols = stage_cols(pc, T::W, S_acc + T::NP);
    else
        pk = stage_packed(pc, T::W, S_acc + T::NP);
    const uint32_t p = threadIdx.x % T::NP, tp = threadIdx.x / T::NP;
    const uint64_t gp = blockIdx.x * (uint64_t)T::NP + p;
    const bool valid = gp < cnt;
    const uint64_t *x = pts + (valid ? gp : 0) * words;
    PointRegs xr{0, 0, 0, 0};
    if (GM == PACKED_REG && valid) {
        xr.x0 = __ldg(x);
        if (words > 1) xr.x1 = __ldg(x + 1);
        if (words > 2) xr.x2 = __ldg(x + 2);
        if (words > 3) xr.x3 = __ldg(x + 3);
    }
    if (threadIdx.x < T::NP) S_acc[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t *S_sm = reinterpret_cast<const uint64_t *>(S_acc);
    phase<LOGW, NP, 0, C::B0, 0, GM>(sm, S_sm, S_acc, p, tp, cols, pk, xr, x, valid, keys, ld, gp);
    __syncthreads();
    if constexpr (C::NPH == 2) {
        phase<LOGW, NP, C::B0, C::B1, 2, GM>(sm, S_sm, S_acc, p, tp, cols, pk, xr, x, valid, keys, ld, gp);
    } else {
        phase<LOGW, NP, C::B0, C::B1, 1, GM>(sm, S_sm, S_acc, p, tp, cols, pk, xr, x, valid, keys, ld, gp);
        __syncthreads();
        phase<LOGW, NP, C::B0 + C::B1, C::B2, 2, GM>(sm, S_sm, S_acc, p, tp, cols, pk, xr, x, valid, keys, ld, gp);
    }
}

template <int LOGW, int NP, int GM>
cudaError_t launch_tile(size_t cbytes, const uint64_t *pts, uint64_t cnt, uint32_t words, PartCols pc, CoordLists cl,
                        uint64_t *keys, uint64_t ld, cudaStream_t s)
{
    using T = Tile<LOGW, NP>;
    const size_t smem = T::VALUES_BYTES + T::NP * 8 + cbytes;
    auto kern = hash_tile_kernel<LOGW, NP, GM>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const uint64_t blocks = (cnt + T::NP - 1) / T::NP;
    kern<<<(unsigned)blocks, T::NT, smem, s>>>(pts, cnt, words, pc, cl, keys, ld);
    note_launch();
    return cudaGetLastError();
}

template <int LOGW, int NP>
cudaError_t launch_gather(uint32_t dk, const uint64_t *pts, uint64_t cnt, uint32_t words, PartCols pc, CoordLists cl,
                          uint64_t *keys, uint64_t ld, cudaStream_t s)
{
    constexpr int W = 1 << LOGW;
    if (dk > (uint32_t)W || words * 64u > kPackedMaxD)   // column lists (general construction, or coordinates past 14 bits)
        return launch_tile<LOGW, NP, GENERAL>(cols_smem_bytes(W, dk), pts, cnt, words, pc, cl, keys, ld, s);
    if (words <= 4) return launch_tile<LOGW, NP, PACKED_REG>((size_t)W * 8, pts, cnt, words, pc, cl, keys, ld, s);
    return launch_tile<LOGW, NP, PACKED_LDG>((size_t)W * 8, pts, cnt, words, pc, cl, keys, ld, s);
}

template <int LOGW>
cudaError_t launch_logw(uint32_t dk, uint32_t tile, const uint64_t *pts, uint64_t cnt, uint32_t words, PartCols pc,
                        CoordLists cl, uint64_t *keys, uint64_t ld, cudaStream_t s)
{
    constexpr int W = 1 << LOGW;
    if (tile == 3) {   // scatter sketch
        if constexpr (LOGW <= 5) {
            const size_t smem = (size_t)W * 128 * 8;
            hash_small_scatter_kernel<LOGW><<<(unsigned)((cnt + 127) / 128), 128, smem, s>>>(pts, cnt, words, cl,
                                                                                                keys, ld);
            note_launch();
            return cudaGetLastError();
        } else {
            return launch_tile<LOGW, tile_points<LOGW>(0), SCATTER>(cl.stage ? scatter_stage_bytes(cl.d, cl.npos) : 0,
                                                                    pts, cnt, words, pc, cl, keys, ld, s);
        }
    }
    if constexpr (LOGW <= 5) {
        const size_t smem = cols_smem_bytes(W, dk);
        const int threads = 128;
        auto kern = hash_small_kernel<LOGW>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        const uint64_t blocks = (cnt + threads - 1) / threads;
        kern<<<(unsigned)blocks, threads, smem, s>>>(pts, cnt, words, pc, keys, ld);
        note_launch();
        return cudaGetLastError();
    } else {
        (void)W;
        constexpr int np0 = tile_points<LOGW>(0), np1 = tile_points<LOGW>(1);
        if (tile == 1 && np1 != np0) return launch_gather<LOGW, np1>(dk, pts, cnt, words, pc, cl, keys, ld, s);
        return launch_gather<LOGW, np0>(dk, pts, cnt, words, pc, cl, keys, ld, s);
    }
}

}  // namespace

template <int LOGW>
size_t tile_smem(uint32_t tile)
{
    const size_t np = (size_t)(tile == 1 ? tile_points<LOGW>(1) : tile_points<LOGW>(0));
    return ((size_t)1 << LOGW) * np * 8 + np * 8;
}

// Shared memory one hash block needs for code length W, a part of dk coordinates
// and the tile choice (3: the scatter sketch, which stages no column lists; 4: the
// direct route's lists of set positions).
size_t hash_smem_bytes(uint32_t W, uint32_t dk, uint32_t tile)
{
    if (tile == 4) return (size_t)kDirectPoints * dk * 10;
    if (tile == 3) return W <= 32 ? (size_t)W * 128 * 8 : hash_smem_bytes(W, 0, 0) - cols_smem_bytes(W, 0);
    size_t t = 0;
    switch (W) {
    case 64: t = tile_smem<6>(tile); break;
    case 128: t = tile_smem<7>(tile); break;
    case 256: t = tile_smem<8>(tile); break;
    case 512: t = tile_smem<9>(tile); break;
    case 1024: t = tile_smem<10>(tile); break;
    case 2048: t = tile_smem<11>(tile); break;
    default: break;
    }
    return t + cols_smem_bytes(W, dk);
}

cudaError_t launch_hash_part(const fclsh_index *idx, uint32_t k, const uint64_t *pts, uint64_t cnt, uint64_t *keys,
                             uint64_t ld, cudaStream_t s, const uint32_t *pidx, const uint64_t *pstart,
                             const uint32_t *plen)
{
    if (cnt == 0) return cudaSuccess;
    if (idx->classic_k) {   // classic bit-sampling LSH: part k = tables k (W-1) .. (k+1)(W-1)-1
        const uint32_t L = idx->W - 1;
        const size_t smem = idx->words <= kClassicSmemWords ? (size_t)kClassicPoints * (idx->words + 1) * 8 : 0;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(classic_hash_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        classic_hash_kernel<<<(unsigned)((cnt + kClassicPoints - 1) / kClassicPoints), kClassicPoints, smem, s>>>(
            pts, cnt, idx->words, idx->cl_off, idx->cl_coord, idx->cl_b, k * L, L, keys, ld);
        note_launch();
        return cudaGetLastError();
    }
    const uint32_t dk = idx->part_off[k + 1] - idx->part_off[k];
    const PartCols pc = idx->part(k);
    if (idx->tune.hash_tile == 2) {   // tensor-core contraction (operands built by the caller)
        if (!idx->mma_g) return cudaErrorInvalidValue;
        return launch_hash_mma(idx->mma_coord + (size_t)k * idx->mma_k,
                               idx->mma_g + (size_t)k * hash_mma_operand_entries(idx->mma_k, idx->W), idx->mma_k,
                               idx->W, pts, cnt, idx->words, keys, ld, idx->status, s);
    }
    const uint32_t logw = idx->rp + 1;
    const uint32_t tl = idx->tune.hash_tile;
    if (tl == 4) {   // direct route: lists of at most dk set positions per point
        if (!idx->sc_b || dk > kDirectMaxPositions) return cudaErrorInvalidValue;
        const size_t smem = hash_smem_bytes(idx->W, dk, 4);
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(hash_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        hash_direct_kernel<<<(unsigned)((cnt + kDirectPoints - 1) / kDirectPoints), kDirectThreads, smem, s>>>(
            pts, cnt, idx->words, idx->coords(k), idx->W, dk, keys, ld);
        note_launch();
        return cudaGetLastError();
    }
    if (tl == 3 && !idx->scatter_ok()) return cudaErrorInvalidValue;
    CoordLists cl = tl == 3 ? idx->coords(k) : CoordLists{nullptr, nullptr, nullptr, 0};
    if (tl == 3 && pidx) {
        cl.pidx = pidx;
        cl.pstart = pstart;
        cl.plen = plen;
    }
    switch (logw) {
    case 1: return launch_logw<1>(dk, tl, pts, cnt, idx->words, pc, cl, keys, ld, s);
    case 2: return launch_logw<2>(dk, tl, pts, cnt, idx->words, pc, cl, keys, ld, s);
    case 3: return launch_logw<3>(dk, tl, pts, cnt, idx->words, pc, cl, keys, ld, s);
    case 4: return launch_logw<4>(dk, tl, pts, cnt, idx->words, pc, cl, keys, ld, s);
    case 5: return launch_logw<5>(dk, tl, pts, cnt, idx->words, pc, cl, keys, ld, s);
    case 6: return launch_logw<6>(dk, tl, pts, cnt, idx->words, pc, cl, keys, ld, s);
    case 7: return launch_logw<7>(dk, tl, pts, cnt, idx->words, pc, cl, keys, ld, s);
    case 8: return launch_logw<8>(dk, tl, pts, cnt, idx->words, pc, cl, keys, ld, s);
    case 9: return launch_logw<9>(dk, tl, pts, cnt, idx->words, pc, cl, keys, ld, s);
    case 10: return launch_logw<10>(dk, tl, pts, cnt, idx->words, pc, cl, keys, ld, s);
    case 11: return launch_logw<11>(dk, tl, pts, cnt, idx->words, pc, cl, keys, ld, s);
    default: return cudaErrorInvalidValue;
    }
}

namespace {

// One warp per point: popcounts of its words (bits past d masked), one atomic reserving
// the point's run, then the set coordinates written in ascending order, 32 words a step
// with a warp scan of the lanes' counts.
__global__ void __launch_bounds__(256) extract_set_bits_kernel(const uint64_t *__restrict__ pts, uint64_t n,
                                                               uint32_t words, uint32_t d, uint64_t cap,
                                                               uint32_t *__restrict__ idx, uint64_t *__restrict__ start,
                                                               uint32_t *__restrict__ len, unsigned long long *cursor)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t lastmask = (d & 63) ? (1ULL << (d & 63)) - 1 : ~0ULL;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t i = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const uint64_t *x = pts + i * words;
        uint32_t mine = 0;
        for (uint32_t w = lane; w < words; w += 32) {
            uint64_t v = __ldg(x + w);
            if (w == words - 1) v &= lastmask;
            mine += __popcll(v);
        }
        const uint32_t total = __reduce_add_sync(0xffffffffu, mine);
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(cursor, (unsigned long long)total);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (lane == 0) {
            start[i] = base;
            len[i] = total;
        }
        if (base + total > cap) continue;   // no room: the caller keeps to the packed words
        uint64_t at = base;
        for (uint32_t w0 = 0; w0 < words; w0 += 32) {
            const uint32_t w = w0 + lane;
            uint64_t v = w < words ? __ldg(x + w) : 0ULL;
            if (w == words - 1) v &= lastmask;
            const uint32_t c = __popcll(v);
            uint32_t incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (uint32_t)o) incl += u;
            }
            uint64_t pos = at + incl - c;
            while (v) {
                idx[pos++] = w * 64 + (uint32_t)(__ffsll((long long)v) - 1);
                v &= v - 1;
            }
            at += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

}  // namespace

cudaError_t launch_extract_set_bits(const uint64_t *pts, uint64_t n, uint32_t words, uint32_t d, uint64_t cap,
                                   uint32_t *idx, uint64_t *start, uint32_t *len, unsigned long long *cursor,
                                   int sm_count, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n == 0) return e;
    const uint64_t blocks = std::min<uint64_t>((n + 7) / 8, (uint64_t)sm_count * 16);
    extract_set_bits_kernel<<<(unsigned)blocks, 256, 0, s>>>(pts, n, words, d, cap, idx, start, len, cursor);
    note_launch();
    return cudaGetLastError();
}

FCLSH_CHECK_READER(check_first_hash)

}  // namespace fclsh
