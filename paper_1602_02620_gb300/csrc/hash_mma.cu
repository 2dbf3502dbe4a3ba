// hash_mma.cu -- the keys of one part as an exact tensor-core contraction.
//
// For a point x and code row v, the key is (Lemma 3 / Eq. 1 on g_v AND x)
//     h_v(x) = ( sum_i x_i * b_i * C(v, m(i)) ) mod P,   C(v, j) = parity(v AND j),
// i.e. row x of the product X * G with X the points' bits (0/1) and
// G[i][v] = b_i C(v, m(i)) -- the O(dL) route, written as a dense contraction over
// the part's d' <= 128 coordinates.  It is made exact on the tensor cores by
// splitting every b_i into five 11-bit limbs: G_l[i][v] = limb_l(b_i) C(v, m(i)).
// X and G_l are exact in fp16 (0/1 and integers below 2^11), every product is exact,
// and every sum of at most 128 of them stays below 2^18, so fp32 accumulation is
// exact.  The epilogue recombines key = sum_l acc_l 2^(11 l) (below 2^63) and reduces
// it mod P.  It gives the same keys as the Walsh-Hadamard route; the autotuner keeps
// whichever runs faster (Sec. 3.2 argues for the transform on a CPU; here the
// contraction runs on the tensor cores).
//
// Kernel: a CTA takes 128 points.  It builds X's tile (128 x K, fp16, K-major,
// 128-byte swizzle) in shared memory, and walks G in chunks of 128 columns (24
// tables x 5 limbs, padded to 16-column groups of 3 tables): each chunk arrives in
// shared memory by one bulk copy (G is stored in global memory already in the
// swizzled shared-memory image), one thread issues K/16 tcgen05.mma (M = N = 128,
// K = 16) into one of two TMEM accumulators, and while the tensor cores work on the
// next chunk, sixteen consumer warps read the finished accumulator with tcgen05.ld (warp w:
// lanes 32 (w mod 4) .. +31 = its points, column groups 2 (w/4) and 2 (w/4) + 1),
// recombine the limbs and store the keys table-major, coalesced over 32 consecutive
// points.
#include "common.cuh"

namespace fclsh {

namespace {

constexpr int kMmaM = 128;              // points per CTA (accumulator lanes)
constexpr int kMmaN = 128;              // accumulator columns per chunk
constexpr int kLimbBits = 11;
constexpr int kLimbs = 5;               // 5 x 11 >= 50 bits of b
constexpr int kTabPerGroup = 3;         // 16-column group: 3 tables x 5 limbs + 1 unused column
constexpr int kGroups = kMmaN / 16;
constexpr int kTabPerChunk = kGroups * kTabPerGroup;   // 24
constexpr int kConsumerWarps = 16;   // warp w: lane quarter w mod 4, column groups {2 (w/4), 2 (w/4) + 1}
constexpr int kMmaThreads = (kConsumerWarps + 1) * 32;   // + one producer warp
constexpr uint32_t kTmemCols = 2 * kMmaN;              // two accumulators

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of 16-bit element (row, k) in a K-major tile of `rows` rows with the
// 128-byte swizzle: blocks of 64 elements along K, each block rows x 128 bytes, the
// 16-byte chunk index XORed with the row index mod 8.
__host__ __device__ __forceinline__ uint32_t sw128_offset(uint32_t row, uint32_t k, uint32_t rows)
{
    const uint32_t blk = k >> 6, c = k & 63;
    return blk * rows * 128u + row * 128u + ((((c >> 3) ^ (row & 7u)) & 7u) << 4) + (c & 7u) * 2u;
}

// Shared-memory matrix descriptor (tcgen05): start address, stride between 8-row
// groups 1,024 bytes, descriptor version 1, 128-byte swizzle.  The leading offset is
// not used by swizzled K-major tiles.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
    return d;
}

// Instruction descriptor, kind::f16: fp32 accumulator, fp16 A and B, both K-major,
// N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kMmaN >> 3) << 17) | ((uint32_t)(kMmaM >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of `parity`; false after about two seconds without it.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = now_ns();
    while (!mbar_try(bar, parity))
        if (now_ns() - t0 > 2000000000ull) return false;
    return true;
}

// One thread: announce `bytes` on the barrier and copy them (pieces of 4 KB).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
    for (uint32_t off = 0; off < bytes; off += 4096) {
        const uint32_t b = bytes - off < 4096u ? bytes - off : 4096u;
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         saddr((char *)dst + off)),
                     "l"((const char *)src + off), "r"(b), "r"(saddr(bar))
                     : "memory");
    }
}

// One thread: K/16 MMAs of a chunk into the accumulator at TMEM column `dcol`, then a
// commit that arrives on `bar` when they are done.
__device__ __forceinline__ void issue_chunk(uint32_t tmem, uint32_t dcol, uint32_t a_base, uint32_t b_base, uint32_t K,
                                            uint64_t *bar)
{
    for (uint32_t s = 0; s < K / 16; ++s) {
        const uint32_t off = (s >> 2) * (128u * 128u) + (s & 3u) * 32u;   // 64-element block, then 16 elements
        const uint64_t da = smem_desc(a_base + off), db = smem_desc(b_base + off);
        const uint32_t acc = s > 0 ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem + dcol),
            "l"(da), "l"(db), "r"(kIdesc), "r"(acc)
            : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ uint32_t limb_value(uint32_t bits)
{
    // an accumulator holds an exact integer below 2^23: adding 2^23 puts it in the mantissa
    return __float_as_uint(__uint_as_float(bits) + 8388608.0f) & 0x7FFFFFu;
}

__device__ __forceinline__ uint64_t mad_wide(uint32_t a, uint32_t b, uint64_t c)
{
    uint64_t r;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"(a), "r"(b), "l"(c));
    return r;
}

// Key of one table from its five limb accumulators (each below 2^18):
// sum_l u_l 2^(11 l) < 2^63 by two wide multiply-adds and one add to the high word,
// then mod P: (x mod 2^50) + 27 (x >> 50), one conditional subtraction.
__device__ __forceinline__ uint64_t key_of(const uint32_t *v)
{
    const uint32_t u0 = limb_value(v[0]), u1 = limb_value(v[1]), u2 = limb_value(v[2]), u3 = limb_value(v[3]),
                   u4 = limb_value(v[4]);
    uint64_t x = mad_wide(u1, 1u << 11, (uint64_t)u0);
    x = mad_wide(u2, 1u << 22, x);
    x += (uint64_t)(u3 * 2u + u4 * 4096u) << 32;   // u3 2^33 + u4 2^44
    const uint32_t hi = (uint32_t)(x >> 32);
    const uint64_t r = mad_wide(hi >> 18, 27u, x & kMask50);
    return r >= kP ? r - kP : r;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}

// Warp-specialised: warps 0..15 read accumulators and write keys, warp 16 allocates
// TMEM and (lane 0) moves G's chunks and issues the MMAs.  Barriers per buffer b:
// gfull[b] (chunk landed), afull[b] (MMAs done: accumulator ready, G buffer free),
// aempty[b] (16 warps have read the accumulator).  Every wait is bounded; a wait that
// runs out sets s_abort and every loop stops at its next check.  Before the tensor memory
// is released after a stop, the producer waits (bounded again) for the MMAs it committed
// and the bulk copies it requested, so that none of them writes TMEM or shared memory
// after the block has let them go.
__global__ void __launch_bounds__(kMmaThreads, 2) hash_mma_kernel(const uint64_t *__restrict__ pts, uint64_t cnt,
                                                                  uint32_t words, const uint32_t *__restrict__ coord,
                                                                  uint32_t K, const uint16_t *__restrict__ gmat,
                                                                  uint32_t chunks, uint32_t L,
                                                                  uint64_t *__restrict__ keys, uint64_t ld,
                                                                  uint32_t *status, uint32_t withhold)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t gfull[2], afull[2], aempty[2];
    __shared__ uint32_t s_tmem;
    __shared__ volatile uint32_t s_abort;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // 1,024-byte aligned tiles: X (128 x K) and two G chunks (128 x K), fp16
    const uint32_t raw = saddr(smem_raw);
    unsigned char *base = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    const uint32_t tile_bytes = K * 256u;
    unsigned char *xa = base;
    auto gb = [&](uint32_t i) { return base + (1 + i) * tile_bytes; };   // the two G chunk buffers
    const uint64_t p0 = (uint64_t)blockIdx.x * kMmaM;
    // producer's record for a clean stop: the last chunk whose MMAs were committed, and per
    // G buffer the chunk whose copy was requested and not yet waited for (-1: none)
    int32_t last_commit = -1, pending0 = -1, pending1 = -1;

    if (warp == kConsumerWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        if (lane == 0) {
            for (int i = 0; i < 2; ++i) {
                mbar_init(&gfull[i], 1);
                mbar_init(&afull[i], 1);
                mbar_init(&aempty[i], kConsumerWarps);
            }
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            s_abort = 0;
            // withhold = c + 1 (tests of the bounded waits): chunk c is never requested, so the
            // wait for it runs out and the kernel reports it in *status
            if (withhold != 1) {
                bulk_load(gb(0), gmat, tile_bytes, &gfull[0]);
                pending0 = 0;
            }
            if (chunks > 1 && withhold != 2) {
                bulk_load(gb(1), gmat + (size_t)K * kMmaN, tile_bytes, &gfull[1]);
                pending1 = 1;
            }
        }
    } else {
        // X's tile: 16-byte chunks of eight fp16 0/1 values (coordinates 8c .. 8c+7 of point p),
        // built in registers and stored whole; lanes take consecutive points, so a warp's
        // stores cover its 32 rows at one chunk (four wavefronts, the 128-byte swizzle's minimum)
        const uint32_t chunks = K / 8;
        for (uint32_t it = tid; it < (uint32_t)kMmaM * chunks; it += kConsumerWarps * 32) {
            const uint32_t p = it & (kMmaM - 1), c8 = it >> 7;
            const uint64_t gp = p0 + p;
            const bool valid = gp < cnt;
            const uint64_t *x = pts + (valid ? gp : 0) * words;
            uint32_t h[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t pair = 0;
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const uint32_t c = __ldg(coord + c8 * 8 + 2 * i + hh);
                    if (valid && c != 0xFFFFFFFFu && ((__ldg(x + (c >> 6)) >> (c & 63)) & 1ull))
                        pair |= 0x3C00u << (16 * hh);
                }
                h[i] = pair;
            }
            *reinterpret_cast<uint4 *>(xa + sw128_offset(p, c8 * 8, kMmaM)) = make_uint4(h[0], h[1], h[2], h[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // X's tile, written by threads, feeds the MMA
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    if (warp == kConsumerWarps) {
        if (lane == 0) {   // producer
            for (uint32_t c = 0; c < chunks && !s_abort; ++c) {
                const uint32_t b = c & 1u;
                bool ok = c < 2 || mbar_wait(&aempty[b], ((c - 2) >> 1) & 1u);   // accumulator b read out
                ok = ok && mbar_wait(&gfull[b], (c >> 1) & 1u);                  // chunk c landed
                if (!ok) {
                    s_abort = 1;
                    break;
                }
                if (b) pending1 = -1; else pending0 = -1;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                issue_chunk(tmem, b * kMmaN, saddr(xa), saddr(gb(b)), K, &afull[b]);
                last_commit = (int32_t)c;
                if (c + 2 < chunks) {   // G buffer b is free once these MMAs are done
                    if (!mbar_wait(&afull[b], (c >> 1) & 1u)) {
                        s_abort = 1;
                        break;
                    }
                    if (withhold != c + 3) {
                        bulk_load(gb(b), gmat + (size_t)(c + 2) * K * kMmaN, tile_bytes, &gfull[b]);
                        if (b) pending1 = (int32_t)(c + 2); else pending0 = (int32_t)(c + 2);
                    }
                }
            }
        }
        __syncwarp();
    } else {   // consumers
        const uint32_t q = warp & 3, g0 = (warp >> 2) * 2;   // TMEM lane quarter (points), first column group
        const uint64_t gp = p0 + 32u * q + lane;
        const bool store = gp < cnt;
        for (uint32_t c = 0; c < chunks; ++c) {
            const uint32_t b = c & 1u;
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&afull[b], (c >> 1) & 1u));   // warp-uniform
            if (!ok || s_abort) {
                s_abort = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t v[32];   // this lane's columns of groups g0 and g0 + 1
            const uint32_t taddr = tmem + ((32u * q) << 16) + b * kMmaN + g0 * 16u;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                  "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
                  "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                  "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&aempty[b]);   // the accumulator may be overwritten now
            const uint32_t tau0 = c * kTabPerChunk + g0 * kTabPerGroup;
            uint64_t *out = keys + (uint64_t)tau0 * ld + gp;
#pragma unroll
            for (int gg = 0; gg < 2; ++gg)
#pragma unroll
                for (int t = 0; t < kTabPerGroup; ++t) {
                    const uint32_t tau = tau0 + gg * kTabPerGroup + t;
                    const uint64_t key = key_of(v + gg * 16 + t * kLimbs);
                    if (store && tau < L) *out = key;
                    out += ld;
                }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && s_abort) atomicOr(status, 1u);
    if (warp == kConsumerWarps) {
        if (lane == 0 && s_abort) {   // drain what was issued before letting TMEM and shared memory go
            // the last commit arrives once every MMA before it is done (they complete in order)
            if (last_commit >= 0) mbar_wait(&afull[last_commit & 1], ((uint32_t)last_commit >> 1) & 1u);
            if (pending0 >= 0) mbar_wait(&gfull[0], ((uint32_t)pending0 >> 1) & 1u);
            if (pending1 >= 0) mbar_wait(&gfull[1], ((uint32_t)pending1 >> 1) & 1u);
        }
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// fp16 bits of an integer 0 <= x < 2^11 (exact).
__device__ __forceinline__ uint16_t half_of(uint32_t x)
{
    if (x == 0) return 0;
    const int e = 31 - __clz(x);                   // 2^e <= x < 2^(e+1), e <= 10
    const uint32_t mant = (x << (10 - e)) & 0x3FFu;
    return (uint16_t)(((uint32_t)(e + 15) << 10) | mant);
}

// G's chunks of part k: one thread per (chunk, row n, coordinate i) writes the fp16
// limb of the chunk's tile, in the swizzled shared-memory image.  Row n of chunk c
// holds limb (n mod 16) mod 5 of table 24 c + 3 (n / 16) + (n mod 16) / 5.
__global__ void __launch_bounds__(256) mma_operand_kernel(const uint32_t *__restrict__ m, const uint64_t *__restrict__ b,
                                                          uint32_t dk, uint32_t K, uint32_t chunks, uint32_t L,
                                                          uint16_t *__restrict__ gmat)
{
    const uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (e >= (uint64_t)chunks * kMmaN * K) return;
    const uint32_t i = (uint32_t)(e % K), n = (uint32_t)((e / K) % kMmaN), c = (uint32_t)(e / ((uint64_t)K * kMmaN));
    const uint32_t j = n & 15u;
    uint16_t val = 0;
    if (i < dk && j < (uint32_t)(kTabPerGroup * kLimbs)) {
        const uint32_t tau = c * kTabPerChunk + (n >> 4) * kTabPerGroup + j / kLimbs, l = j % kLimbs;
        const uint32_t v = tau + 1;   // code row
        if (tau < L && (__popc(v & m[i]) & 1))
            val = half_of((uint32_t)(b[i] >> (kLimbBits * l)) & ((1u << kLimbBits) - 1));
    }
    gmat[(size_t)c * K * kMmaN + sw128_offset(n, i, kMmaN) / 2] = val;
}

}  // namespace

// K (padded coordinates per part) of the contraction, 0 if it does not apply.
uint32_t hash_mma_k(uint32_t W, uint32_t max_dk)
{
    if (W < 64 || max_dk == 0 || max_dk > 128) return 0;
    return max_dk <= 64 ? 64u : 128u;
}

// Chunks of 24 tables per part.
uint32_t hash_mma_chunks(uint32_t W) { return (W - 1 + kTabPerChunk - 1) / kTabPerChunk; }

// G's chunks of one part on the device (m, b: the part's d_k entries, device).
cudaError_t build_mma_operand(const uint32_t *m, const uint64_t *b, uint32_t dk, uint32_t K, uint32_t W,
                              uint16_t *gmat, cudaStream_t s)
{
    const uint32_t chunks = hash_mma_chunks(W);
    const uint64_t total = (uint64_t)chunks * kMmaN * K;
    mma_operand_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(m, b, dk, K, chunks, W - 1, gmat);
    note_launch();
    return cudaGetLastError();
}

// Elements of G's chunks per part.
size_t hash_mma_operand_entries(uint32_t K, uint32_t W) { return (size_t)hash_mma_chunks(W) * K * kMmaN; }

size_t hash_mma_smem(uint32_t K) { return (size_t)3 * K * 256 + 1024; }

cudaError_t launch_hash_mma(const uint32_t *coord, const uint16_t *gmat, uint32_t K, uint32_t W, const uint64_t *pts,
                            uint64_t cnt, uint32_t words, uint64_t *keys, uint64_t ld, uint32_t *status,
                            cudaStream_t s)
{
    if (cnt == 0) return cudaSuccess;
    const size_t smem = hash_mma_smem(K);
    static cudaError_t once =
        cudaFuncSetAttribute(hash_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hash_mma_smem(128));
    if (once != cudaSuccess) return once;
    const uint64_t blocks = (cnt + kMmaM - 1) / kMmaM;
    hash_mma_kernel<<<(unsigned)blocks, kMmaThreads, smem, s>>>(pts, cnt, words, coord, K, gmat, hash_mma_chunks(W),
                                                                 W - 1, keys, ld, status, debug_withhold_loads());
    note_launch();
    return cudaGetLastError();
}

FCLSH_CHECK_READER(check_first_mma)

}  // namespace fclsh
