// query.cu -- Strategy 2 queries (Sec. 2.2) in the cost steps of Sec. 4.1:
//   S1  hash the query into its T keys (Algorithm 2, in the CTA's shared memory),
//   S2  look up the query's bucket in every table and merge the buckets with
//       duplicate elimination (#Collisions, #Candidates),
//   S3  compute the Hamming distance of each distinct candidate by popcount and
//       report it if it is within the query's radius.
//
// Batched form: one persistent kernel; each CTA takes the next query from a
// global work counter, so queries with very different candidate counts balance
// across the GPU.  Inside a CTA, warps take 32 tables at a time: a lane walks its
// own bucket range when it is short, and the whole warp walks a long one, so a
// heavy bucket never serialises on one lane.  Duplicates are removed with a
// shared-memory hash set when the query's bucket ranges hold at most half its
// capacity, and otherwise with an n-bit bitmap owned by the CTA (the bitmap of
// Sec. 4.1), cleared after the query: a returning atomic per collision tells a new
// candidate, or, when the ranges hold more entries than the bitmap has words, the
// collisions only mark it and one sweep of the bitmap then verifies the marked ids.
// Hits collect in shared memory and are sorted there (up to 4,096 per query); a
// query with more hits marks them in the bitmap and reads its ids out of it in
// order.  Each query writes one sorted run; a gather kernel lays the runs out as CSR.
// Very heavy queries (more bucket entries than the bitmap has words) can instead be
// listed for a second kernel, one block of 32 warps per SM, that marks their entries in
// a window of ids held in shared memory, window by window, so that no collision costs
// an atomic on a bitmap in L2.
#include "common.cuh"

namespace fclsh {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr uint32_t kResCap = 4096;   // hits of one query sorted in shared memory

namespace {

__device__ __forceinline__ uint32_t lanemask_lt()
{
    return (1u << (threadIdx.x & 31)) - 1u;
}

// L2 eviction priorities for the loads of the heavy-query kernel: the bucket entries it
// streams are evicted first, the point signatures (read at random, again and again) last.
__device__ __forceinline__ uint64_t l2_policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t ld_nc_hint(const uint64_t *ptr, uint64_t policy)
{
    uint64_t v;
    asm("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(ptr), "l"(policy));
    return v;
}
__device__ __forceinline__ ulonglong2 ld_nc_hint2(const ulonglong2 *ptr, uint64_t policy)
{
    ulonglong2 v;
    asm("ld.global.nc.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;" : "=l"(v.x), "=l"(v.y) : "l"(ptr), "l"(policy));
    return v;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T *red)   // red: >= 32 entries of smem
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T s = 0;
    const uint32_t nw = blockDim.x >> 5;
    for (uint32_t w = 0; w < nw; ++w) s += red[w];
    return s;
}

// Exclusive block-wide prefix of one u32 per thread (red: >= 33 u64 of shared memory).
__device__ __forceinline__ uint64_t block_excl_scan_u32(uint32_t v, unsigned long long *red)
{
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += u;
    }
    __syncthreads();
    if (lane == 31) red[warp] = incl;
    __syncthreads();
    uint64_t before = 0;
    for (uint32_t w = 0; w < warp; ++w) before += red[w];
    (void)nw;
    __syncthreads();
    return before + incl - v;
}

// Hamming distance between the query in shared memory and point `id`.
__device__ __forceinline__ uint32_t distance_to(const QueryArgs &a, const uint64_t *q_s, uint32_t id)
{
    if (!FCLSH_CHECK(id < a.n, 0x0101)) return 0xFFFFFFFFu;
    const uint64_t *x = a.points + (uint64_t)id * a.words;
    uint32_t dist = 0;
    if ((a.words & 1) == 0) {
        const ulonglong2 *x2 = reinterpret_cast<const ulonglong2 *>(x);
        for (uint32_t w = 0; w < a.words / 2; ++w) {
            const ulonglong2 v = __ldg(x2 + w);
            dist += __popcll(v.x ^ q_s[2 * w]) + __popcll(v.y ^ q_s[2 * w + 1]);
        }
    } else {
        for (uint32_t w = 0; w < a.words; ++w) dist += __popcll(__ldg(x + w) ^ q_s[w]);
    }
    return dist;
}

__device__ __forceinline__ bool hset_insert(uint32_t *hset, uint32_t hlog, uint32_t id)
{
    const uint32_t mask = (1u << hlog) - 1u;
    uint32_t s = (id * 0x9E3779B1u) >> (32 - hlog);
    for (;;) {
        const uint32_t old = atomicCAS(hset + s, kEmpty, id);
        if (old == kEmpty) return true;
        if (old == id) return false;
        s = (s + 1) & mask;
    }
}

struct Counters {
    unsigned long long coll = 0, cand = 0;
    uint32_t res = 0;
};

// Append the lanes' hits to the query's hit list in shared memory; warp-collective.  Hits past
// the list's kResCap places are marked in ovf_bm when it is given (the heavy kernel's CTA bitmap).
__device__ __forceinline__ void append_hits(bool hit, uint32_t id, Counters &c, uint32_t *res_s, uint32_t *s_nres,
                                            uint32_t *ovf_bm = nullptr)
{
    const uint32_t m = __ballot_sync(0xffffffffu, hit);
    if (m) {
        const uint32_t lane = threadIdx.x & 31;
        const uint32_t leader = __ffs(m) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(s_nres, (uint32_t)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (hit) {
            c.res++;
            const uint32_t pos = base + __popc(m & lanemask_lt());
            if (pos < kResCap) res_s[pos] = id;
            else if (ovf_bm) atomicOr(ovf_bm + (id >> 5), 1u << (id & 31));
        }
    }
}

// Dedup modes of a query: a shared-memory hash set; the CTA's n-bit bitmap with a
// returning atomic per collision (a new bit = a new candidate, verified at once);
// or, for very heavy queries, the bitmap marked without returns and swept afterwards.
enum DedupMode { DEDUP_HSET = 0, DEDUP_BITMAP = 1, DEDUP_MARK = 2 };

// The query's occupancy levels from warps 0-3 (thread j: signature block j): sigm32 is a
// 32-bit view of sigm[kSigLevels + 1]; warp w gives the bits of blocks 32w .. 32w + 31 of
// every level.
__device__ __forceinline__ void sig_levels(const uint64_t *q_s, uint32_t d, uint32_t sig_block, uint32_t lane,
                                           uint32_t warp, uint32_t *sigm32)
{
    const uint32_t j = warp * 32 + lane, lo = j * sig_block;
    const uint32_t pc = lo < d ? popc_range(q_s, lo, min(lo + sig_block, d)) : 0u;
#pragma unroll
    for (int t = 1; t <= kSigLevels; ++t) {
        const uint32_t bal = __ballot_sync(0xffffffffu, pc >= (uint32_t)t);
        if (lane == 0) sigm32[4 * t + warp] = bal;
    }
}

// S3's pre-filter: false when the signature bound already puts point id beyond the radius.
__device__ __forceinline__ bool sig_pass(const QueryArgs &a, uint32_t id, ulonglong2 sq, const ulonglong2 *sigm,
                                         uint32_t radius)
{
    return !a.sig || sig_bound(sig_of(a.sig, id), sq, sigm) <= radius;
}

// One bucket entry per lane (is_coll = key matched); warp-collective.
__device__ __forceinline__ void process_entry(const QueryArgs &a, const uint64_t *q_s, uint32_t *hset, uint32_t *bm,
                                              int mode, uint32_t radius, bool is_coll, uint32_t id, Counters &c,
                                              uint32_t *res_s, uint32_t *s_nres, ulonglong2 sq, const ulonglong2 *sigm)
{
    bool isnew = false;
    is_coll = is_coll && FCLSH_CHECK(id < a.n, 0x0109);
    if (is_coll) {
        c.coll++;
        const uint32_t bit = 1u << (id & 31);
        if (mode == DEDUP_MARK)
            atomicOr(bm + (id >> 5), bit);   // result unused: a fire-and-forget reduction
        else if (mode == DEDUP_BITMAP)
            isnew = (atomicOr(bm + (id >> 5), bit) & bit) == 0;
        else
            isnew = hset_insert(hset, a.hset_log2, id);
    }
    if (mode == DEDUP_MARK) return;   // warp-uniform
    bool hit = false;
    if (a.words >= kWarpVerifyWords) {   // long points: the warp reads each new candidate together
        const uint32_t lane = threadIdx.x & 31;
        uint32_t need = __ballot_sync(0xffffffffu, isnew && sig_pass(a, id, sq, sigm, radius));
        while (need) {
            const uint32_t src = __ffs(need) - 1;
            need &= need - 1;
            const uint64_t *x = a.points + (uint64_t)__shfl_sync(0xffffffffu, id, src) * a.words;
            // 256 words per step, eight independent loads per lane; stop once the
            // distance so far exceeds the radius (warp-uniform)
            uint32_t dist = 0, wb = 0;   // wb: warp-uniform base of the step
            for (; wb + 256 <= a.words; wb += 256) {
                uint64_t v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = __ldg(x + wb + lane + 32 * u);
                uint32_t part = 0;
#pragma unroll
                for (int u = 0; u < 8; ++u) part += __popcll(v[u] ^ q_s[wb + lane + 32 * u]);
                dist += __reduce_add_sync(0xffffffffu, part);
                if (dist > radius) break;
            }
            if (dist <= radius) {
                uint32_t part = 0;
                for (uint32_t w = wb + lane; w < a.words; w += 32) part += __popcll(__ldg(x + w) ^ q_s[w]);
                dist += __reduce_add_sync(0xffffffffu, part);
            }
            if (lane == src) hit = dist <= radius;
        }
        if (isnew) c.cand++;
    } else if (isnew) {
        c.cand++;
        hit = sig_pass(a, id, sq, sigm, radius) && distance_to(a, q_s, id) <= radius;
    }
    append_hits(hit, id, c, res_s, s_nres);
}

// ---- S2b/S3 over the query's bucket entries as one list: run j (the j-th probed table's
// bucket range) holds list positions [off_s[j], off_s[j+1]), off_s being the exclusive
// prefix of the run lengths.  A chunk gives every thread kU positions at once, so that the
// block has kU independent entry loads per thread in flight, then kU independent dedup
// atomics, and then verifies the chunk's new candidates together (S3).
constexpr int kU = 4;
constexpr uint32_t kCandCap = 512u * kU;   // new candidates of one chunk (blocks of up to 512 threads)
constexpr uint32_t kHeavyThreads = 1024;    // query_heavy_kernel: one block of 32 warps per SM
constexpr uint32_t kHeavyCand = 4096;       // its candidate lists (S3): one of kWarpCand per warp
constexpr uint32_t kWarpCand = kHeavyCand / (kHeavyThreads / 32);
constexpr int kHeavyU = 4;                  // its list positions per thread per chunk (one search)
// bucket entries of a query that query_heavy_kernel walks as one list (32-bit positions)
constexpr unsigned long long kHeavyMaxEntries = 0xFFFFFFFFull - (unsigned long long)kHeavyThreads * kHeavyU;

// The run holding list position pos: the last j < nruns with off[j] <= pos (off[0] = 0).
__device__ __forceinline__ uint32_t run_of(const uint32_t *off, uint32_t nruns, uint32_t pos)
{
    uint32_t lo = 0, hi = nruns;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (off[mid] <= pos) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Stored key bits that no entry has (entry_fp is below 2^50): a chunk position past the list's end.
constexpr uint64_t kNoFp = ~0ULL;

template <int U = kU>
struct Chunk {
    uint64_t en[U];
    uint64_t fp[U];   // the probed key's stored bits (entry_fp of its bucket's entries), kNoFp past the end
};

// The entries at list positions base + U * threadIdx.x + k, k < U: one search for the run of
// the first, then a walk over the runs, the current run's entry row and key bits kept in
// registers (loads issued back to back; a warp's positions are consecutive, so a long run is
// read in whole lines).  An entry is a collision when entry_fp(en) == fp.
template <int U = kU, bool HINT = false>
__device__ __forceinline__ void load_chunk(const QueryArgs &a, const uint64_t *keys_s, const uint32_t *lo_s,
                                           const uint32_t *off_s, uint32_t Tq, uint32_t nt, uint32_t L, uint32_t E,
                                           uint32_t base, Chunk<U> &ch, uint64_t policy = 0)
{
    const uint32_t pos0 = base + U * threadIdx.x;
#pragma unroll
    for (int k = 0; k < U; ++k) {
        ch.en[k] = 0;
        ch.fp[k] = kNoFp;
    }
    if (pos0 >= E) return;
    uint32_t j = run_of(off_s, Tq, pos0);
    uint32_t next = j + 1 < Tq ? off_s[j + 1] : E;   // the list position where run j ends
    uint32_t tau = probed_table(j, nt, L);
    uint64_t fp = keys_s[tau] >> a.slot_bits;
    uint64_t row = (uint64_t)tau * a.n + lo_s[j] - off_s[j];   // list position p of run j: ent[row + p] (mod 2^64)
#pragma unroll
    for (int k = 0; k < U; ++k) {
        const uint32_t pos = pos0 + k;
        if (pos < E) {
            while (pos >= next) {   // the next non-empty run
                ++j;
                next = j + 1 < Tq ? off_s[j + 1] : E;
                tau = probed_table(j, nt, L);
                fp = keys_s[tau] >> a.slot_bits;
                row = (uint64_t)tau * a.n + lo_s[j] - off_s[j];
            }
            const uint64_t e = row + pos;
            if (FCLSH_CHECK(pos - off_s[j] < next - off_s[j] && tau < a.T, 0x0103)) {
                ch.fp[k] = fp;
                ch.en[k] = HINT ? ld_nc_hint(a.ent + e, policy) : __ldg(a.ent + e);
            }
        }
    }
}

// Append the lanes' new candidates to the chunk's list; warp-collective.
__device__ __forceinline__ void push_cand(bool isnew, uint32_t id, uint32_t *cand_s, uint32_t *s_ncand)
{
    const uint32_t m = __ballot_sync(0xffffffffu, isnew);
    if (!m) return;
    const uint32_t lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(s_ncand, (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    const uint32_t at = base + __popc(m & lanemask_lt());
    if (isnew && FCLSH_CHECK(at < kCandCap, 0x0105)) cand_s[at] = id;
}

// Distance of point id read by the whole warp (long points): 256 words per step, eight
// independent loads per lane, stopping once the partial distance exceeds the radius.
// Every lane returns the same value; warp-collective.
__device__ __forceinline__ uint32_t warp_distance(const QueryArgs &a, const uint64_t *q_s, uint32_t id, uint32_t radius)
{
    const uint32_t lane = threadIdx.x & 31;
    if (!FCLSH_CHECK(id < a.n, 0x0102)) return 0xFFFFFFFFu;
    const uint64_t *x = a.points + (uint64_t)id * a.words;
    uint32_t dist = 0, wb = 0;
    for (; wb + 256 <= a.words; wb += 256) {
        uint64_t v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldg(x + wb + lane + 32 * u);
        uint32_t part = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) part += __popcll(v[u] ^ q_s[wb + lane + 32 * u]);
        dist += __reduce_add_sync(0xffffffffu, part);
        if (dist > radius) return dist;
    }
    uint32_t part = 0;
    for (uint32_t w = wb + lane; w < a.words; w += 32) part += __popcll(__ldg(x + w) ^ q_s[w]);
    return dist + __reduce_add_sync(0xffffffffu, part);
}

// Candidates whose points a group of lanes loads before reducing any of them.
constexpr int kV = 4;

// The grouped reads of verify_list for points of H 16-byte pieces per lane (H = 1: up to 16
// words; 2: up to 31).
// The list is shared by the block's warps (block = true) or is the calling warp's own.
template <int H>
__device__ __forceinline__ void verify_groups(const QueryArgs &a, const uint64_t *q_s, const uint32_t *cand_s,
                                              uint32_t m, uint32_t radius, bool count, Counters &c, uint32_t *res_s,
                                              uint32_t *s_nres, uint32_t *ovf_bm, bool block = true)
{
    const uint32_t lane = threadIdx.x & 31, warp = block ? threadIdx.x >> 5 : 0u, nwarps = block ? blockDim.x >> 5 : 1u;
    const uint32_t words = a.words, pieces = (words + 1) >> 1;   // 16-byte pieces of a point
    const uint32_t G = pieces <= 1 ? 1u : pieces <= 2 ? 2u : pieces <= 4 ? 4u : 8u;
    const uint32_t per = 32u / G, sub = lane / G, gl = lane % G;  // candidates per warp step; group, lane in it
    const bool even = (words & 1u) == 0;
    for (uint32_t i0 = warp * per * kV; i0 < m; i0 += nwarps * per * kV) {   // warp-uniform bounds
        uint32_t id[kV];
        bool ok[kV];
        ulonglong2 x[kV][H];
#pragma unroll
        for (int v = 0; v < kV; ++v) {   // the loads of kV candidates, back to back
            const uint32_t i = i0 + v * per + sub;
            ok[v] = i < m;
            id[v] = ok[v] ? cand_s[i] : 0u;
            ok[v] = ok[v] && FCLSH_CHECK(id[v] < a.n, 0x0101);
            const uint64_t *pt = a.points + (uint64_t)id[v] * words;
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const uint32_t pc = gl + h * G;
                x[v][h] = make_ulonglong2(0, 0);
                if (ok[v] && pc < pieces) {
                    if (even) {
                        x[v][h] = __ldg(reinterpret_cast<const ulonglong2 *>(pt) + pc);
                    } else {
                        x[v][h].x = __ldg(pt + 2 * pc);
                        if (2 * pc + 1 < words) x[v][h].y = __ldg(pt + 2 * pc + 1);
                    }
                }
            }
        }
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            uint32_t part = 0;
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const uint32_t pc = gl + h * G;
                if (pc < pieces) {
                    part += __popcll(x[v][h].x ^ q_s[2 * pc]);
                    if (2 * pc + 1 < words) part += __popcll(x[v][h].y ^ q_s[2 * pc + 1]);
                }
            }
            for (uint32_t o = G >> 1; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            const uint32_t i = i0 + v * per + sub;
            const bool lead = gl == 0 && i < m;
            if (lead && count) c.cand++;
            const bool hit = lead && ok[v] && part <= radius;
            append_hits(hit, id[v], c, res_s, s_nres, ovf_bm);
        }
    }
}

// Candidates whose signatures a thread loads before bounding any of them.
constexpr int kF = 4;

// S3 for the candidates cand_s[0..m) (block-wide; the list may be rewritten): each is counted
// once in #Candidates and reported if within the radius.  With the pre-filter, a thread per
// candidate first bounds its distance from the signatures (kF loads in flight per thread) and
// the candidates that pass are compacted to the list's front (s_nsurv: a shared counter).
// Points of up to 31 words are then read by groups of G lanes, one 16-byte piece per lane
// (G = 8 for 16 words: a point is one 128-byte line), kV candidates per group loaded before
// their popcounts are reduced in the group; longer points by the whole warp.
__device__ __forceinline__ void verify_list(const QueryArgs &a, const uint64_t *q_s, uint32_t *cand_s, uint32_t m,
                                            uint32_t radius, ulonglong2 sq, const ulonglong2 *sigm, Counters &c,
                                            uint32_t *res_s, uint32_t *s_nres, uint32_t *s_nsurv,
                                            uint32_t *ovf_bm = nullptr)
{
    const uint32_t B = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = B >> 5;
    const bool count = !a.sig;   // with the pre-filter every candidate is counted as it is bounded
    if (a.sig) {
        if (tid == 0) *s_nsurv = 0;
        __syncthreads();
        for (uint32_t base = 0; base < m; base += B * kF) {
            uint32_t id[kF];
            ulonglong2 sx[kF];
#pragma unroll
            for (int f = 0; f < kF; ++f) {
                const uint32_t i = base + f * B + tid;
                id[f] = i < m ? cand_s[i] : 0u;
                sx[f] = i < m && FCLSH_CHECK(id[f] < a.n, 0x0107) ? sig_of(a.sig, id[f]) : make_ulonglong2(0, 0);
            }
            __syncthreads();   // the round's reads before the survivors overwrite the list's front
#pragma unroll
            for (int f = 0; f < kF; ++f) {
                const bool in = base + f * B + tid < m;
                if (in) c.cand++;
                const bool pass = in && id[f] < a.n && sig_bound(sx[f], sq, sigm) <= radius;
                const uint32_t bal = __ballot_sync(0xffffffffu, pass);
                if (bal) {
                    const uint32_t leader = __ffs(bal) - 1;
                    uint32_t at = 0;
                    if (lane == leader) at = atomicAdd(s_nsurv, (uint32_t)__popc(bal));
                    at = __shfl_sync(0xffffffffu, at, leader) + __popc(bal & lanemask_lt());
                    if (pass) cand_s[at] = id[f];
                }
            }
        }
        __syncthreads();
        m = *s_nsurv;
    }
    if (a.words >= kWarpVerifyWords) {   // a warp per candidate: coalesced reads of long points
        for (uint32_t i0 = 0; i0 < m; i0 += nwarps) {
            const uint32_t i = i0 + warp;
            const bool ok = i < m;
            const uint32_t id = ok ? cand_s[i] : 0;
            bool hit = false;
            if (ok) {
                if (lane == 0 && count) c.cand++;
                hit = warp_distance(a, q_s, id, radius) <= radius;
            }
            append_hits(hit && lane == 0, id, c, res_s, s_nres, ovf_bm);
        }
        return;
    }
    if (a.words <= 16)
        verify_groups<1>(a, q_s, cand_s, m, radius, count, c, res_s, s_nres, ovf_bm);
    else
        verify_groups<2>(a, q_s, cand_s, m, radius, count, c, res_s, s_nres, ovf_bm);
}

// S3 for the candidates buf[0..m) of one warp (warp-collective; counted where they were
// listed): points of up to 31 words read by groups of lanes as in verify_groups, longer ones by
// the whole warp.  No block barrier, so the block's warps go through their lists independently.
__device__ __forceinline__ void verify_warp(const QueryArgs &a, const uint64_t *q_s, const uint32_t *buf, uint32_t m,
                                            uint32_t radius, Counters &c, uint32_t *res_s, uint32_t *s_nres,
                                            uint32_t *ovf_bm)
{
    const uint32_t lane = threadIdx.x & 31;
    if (a.words >= kWarpVerifyWords) {
        for (uint32_t i = 0; i < m; ++i) {
            const uint32_t id = buf[i];
            const bool hit = warp_distance(a, q_s, id, radius) <= radius;
            append_hits(hit && lane == 0, id, c, res_s, s_nres, ovf_bm);
        }
        return;
    }
    if (a.words <= 16)
        verify_groups<1>(a, q_s, buf, m, radius, false, c, res_s, s_nres, ovf_bm, false);
    else
        verify_groups<2>(a, q_s, buf, m, radius, false, c, res_s, s_nres, ovf_bm, false);
}

// Sort of the distinct values v[0..cnt) in shared memory (cnt <= kResCap), ascending; block-wide:
// shuffles up to 32, ranks up to 512, a bitonic network beyond.
__device__ __forceinline__ void block_sort_u32(uint32_t *v, uint32_t cnt)
{
    if (cnt <= 1) return;
    const uint32_t tid = threadIdx.x, B = blockDim.x;
    if (cnt <= 32) {   // one warp, shuffles only
        if (tid < 32) {
            uint32_t x = tid < cnt ? v[tid] : 0xFFFFFFFFu;
            for (uint32_t k = 2; k <= 32; k <<= 1)
                for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
                    const bool lower = (tid & j) == 0, up = (tid & k) == 0;
                    x = (lower == up) ? min(x, y) : max(x, y);
                }
            if (tid < cnt) v[tid] = x;
        }
        __syncthreads();
        return;
    }
    if (cnt <= 512 && cnt <= B) {   // the ids are distinct: each goes to its rank (one read pass, no
        uint32_t x = 0, r = 0;       // merge rounds; the threads read v[j] together, a broadcast)
        if (tid < cnt) {
            x = v[tid];
            for (uint32_t j = 0; j < cnt; ++j) r += v[j] < x ? 1u : 0u;
        }
        __syncthreads();
        if (tid < cnt) v[r] = x;
        __syncthreads();
        return;
    }
    uint32_t size = 64;
    while (size < cnt) size <<= 1;
    for (uint32_t i = cnt + tid; i < size; i += B) v[i] = 0xFFFFFFFFu;
    __syncthreads();
    for (uint32_t k = 2; k <= size; k <<= 1)
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = tid; i < size / 2; i += B) {
                const uint32_t a = 2 * i - (i & (j - 1)), b = a + j;
                const bool up = (a & k) == 0;
                const uint32_t x = v[a], y = v[b];
                if ((x > y) == up) {
                    v[a] = y;
                    v[b] = x;
                }
            }
            __syncthreads();
        }
}


// The query into shared memory and, with the S3 pre-filter, its occupancy levels sigm[t]
// (t = 1..kSigLevels; sigm[1] is its block-occupancy signature): bit j set when the query has
// at least t set coordinates in signature block j.  Read after the barriers of S1.  Block-wide.
__device__ __forceinline__ void load_query(const QueryArgs &a, uint64_t qi, uint64_t *q_s, ulonglong2 *sigm)
{
    const uint32_t tid = threadIdx.x, B = blockDim.x, lane = tid & 31, warp = tid >> 5;
    for (uint32_t w = tid; w < a.words; w += B) q_s[w] = a.queries[qi * a.words + w];
    __syncthreads();
    if (a.sig && tid < kSigBlocks) sig_levels(q_s, a.d, a.sig_block, lane, warp, reinterpret_cast<uint32_t *>(sigm));
}

// S1: Algorithm 2 for every part in shared memory (tbuf: W words), or the keys a hash launch
// computed before the kernel; keys_s[tau] for every table.  Block-wide, ends on a barrier.
__device__ __forceinline__ void query_s1(const QueryArgs &a, uint64_t qi, const uint64_t *q_s, uint64_t *keys_s,
                                         uint64_t *tbuf)
{
    const uint32_t tid = threadIdx.x, B = blockDim.x, L = a.W - 1;
    if (a.qkeys) {
        for (uint32_t tau = tid; tau < a.T; tau += B) keys_s[tau] = a.qkeys[(uint64_t)tau * a.nq + qi];
        __syncthreads();
    }
    for (uint32_t k = 0; k < (a.qkeys ? 0u : a.t); ++k) {
        if (a.s1_scatter) {
            // sketch from the query's set bits: each adds its positions' seed values to
            // their columns (64-bit sums, exact while a column holds <= 16,383 positions)
            for (uint32_t j = tid; j < a.W; j += B) tbuf[j] = 0;
            __syncthreads();
            const uint32_t *off = a.sc_off + (size_t)k * (a.d + 1);
            for (uint32_t w = tid; w < a.words; w += B) {
                uint64_t bits = q_s[w];
                if (w == a.words - 1 && (a.d & 63)) bits &= (1ULL << (a.d & 63)) - 1;
                while (bits) {
                    const uint32_t c = w * 64 + (uint32_t)(__ffsll((long long)bits) - 1);
                    bits &= bits - 1;
                    for (uint32_t e = off[c]; e < off[c + 1]; ++e)
                        atomicAdd(reinterpret_cast<unsigned long long *>(tbuf + a.sc_col[e]),
                                  (unsigned long long)a.sc_b[e]);
                }
            }
            __syncthreads();
            for (uint32_t j = tid; j < a.W; j += B) tbuf[j] = mod_p(tbuf[j]);
        } else {
            const uint32_t *co = a.col_off + (size_t)k * (a.W + 1);
            for (uint32_t j = tid; j < a.W; j += B) {
                uint64_t s = 0;
                const uint32_t e1 = co[j + 1];
                for (uint32_t e = co[j]; e < e1; ++e) {
                    const uint32_t bit = a.col_coord[e];
                    const uint64_t take = 0ULL - ((q_s[bit >> 6] >> (bit & 63)) & 1ULL);
                    s = add_mod_p(s, a.col_b[e] & take);
                }
                tbuf[j] = s;
            }
        }
        __syncthreads();
        for (uint32_t h = 1; h < a.W; h <<= 1) {
            for (uint32_t i = tid; i < a.W / 2; i += B) {
                const uint32_t j = ((i & ~(h - 1)) << 1) | (i & (h - 1));
                const uint64_t x = tbuf[j], y = tbuf[j + h];
                tbuf[j] = x + y;
                tbuf[j + h] = x - y;
            }
            __syncthreads();
        }
        const uint64_t S = tbuf[0];   // y_0 = sum_j t_j
        for (uint32_t v = tid + 1; v < a.W; v += B) keys_s[k * L + v - 1] = finish_key(S, tbuf[v]);
        __syncthreads();
    }
}

// S2a: the bucket range of every probed table (lo_s, len_s), the probed tables' count Tq
// (nt code rows per part) and the query's bucket entries E summed over them.  Block-wide.
__device__ __forceinline__ unsigned long long probe_ranges(const QueryArgs &a, uint32_t radius, const uint64_t *keys_s,
                                                           uint32_t *lo_s, uint32_t *len_s, unsigned long long *red64,
                                                           uint32_t &nt, uint32_t &Tq)
{
    const uint32_t tid = threadIdx.x, B = blockDim.x, L = a.W - 1;
    const uint64_t smask = (1ULL << a.slot_bits) - 1;
    nt = rows_per_part(a, radius);
    Tq = a.t * nt;
    unsigned long long local = 0;
    constexpr int kP = 4;   // tables whose directory words a thread loads before using any
    for (uint32_t j0 = tid; j0 < Tq; j0 += kP * B) {
        uint32_t lo[kP], hi[kP];
#pragma unroll
        for (int u = 0; u < kP; ++u) {
            const uint32_t j = j0 + u * B;
            lo[u] = hi[u] = 0;
            if (j < Tq) {
                const uint32_t tau = probed_table(j, nt, L);
                if (FCLSH_CHECK(tau < a.T, 0x0106)) {
                    const uint32_t *O = a.offs + (uint64_t)tau * a.offs_stride + (keys_s[tau] & smask);
                    lo[u] = O[0];
                    hi[u] = O[1];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kP; ++u) {
            const uint32_t j = j0 + u * B;
            if (j < Tq) {
                lo_s[j] = lo[u];
                len_s[j] = hi[u] - lo[u];
                local += hi[u] - lo[u];
            }
        }
    }
    return block_sum(local, red64);
}

// len_s[0..Tq) -> its exclusive prefix, in place (the runs as one list).  Block-wide.
__device__ __forceinline__ void runs_prefix(uint32_t *len_s, uint32_t Tq, unsigned long long *red64)
{
    const uint32_t tid = threadIdx.x, B = blockDim.x;
    const uint32_t per = (Tq + B - 1) / B, j0 = tid * per, j1 = min(j0 + per, Tq);
    uint32_t mine = 0;
    for (uint32_t j = j0; j < j1; ++j) mine += len_s[j];
    uint32_t run = (uint32_t)block_excl_scan_u32(mine, red64);
    for (uint32_t j = j0; j < j1; ++j) {
        const uint32_t len = len_s[j];
        len_s[j] = run;
        run += len;
    }
}

// The ids marked in the CTA's n-bit bitmap, in ascending order, to runs[base ..] (within the
// buffer's cap); the bitmap is left all-zero.  Block-wide.
__device__ __forceinline__ void bitmap_readout(const QueryArgs &a, uint32_t *bm, unsigned long long base,
                                               unsigned long long *red64)
{
    const uint32_t tid = threadIdx.x, B = blockDim.x;
    const uint64_t per = (a.bm_words + B - 1) / B;
    const uint64_t w0 = (uint64_t)tid * per, w1 = min(w0 + per, a.bm_words);
    uint32_t mine = 0;
    for (uint64_t w = w0; w < w1; ++w) mine += __popc(__ldcg(bm + w));   // marks are made in L2
    const uint32_t before = (uint32_t)block_excl_scan_u32(mine, red64);
    unsigned long long pos = base + before;
    for (uint64_t w = w0; w < w1; ++w) {
        uint32_t bits = __ldcg(bm + w);
        while (bits) {
            const uint32_t b = __ffs(bits) - 1;
            bits &= bits - 1;
            if (pos < a.cap) a.runs[pos] = (uint32_t)(w * 32 + b);
            ++pos;
        }
        bm[w] = 0;
    }
}

}  // namespace

// Dynamic shared memory of the batched kernel.
size_t query_smem_bytes(uint32_t T, uint32_t W, uint32_t words, uint32_t hset_log2)
{
    const size_t tb = (size_t)W * 8 > ((size_t)4 << hset_log2) ? (size_t)W * 8 : ((size_t)4 << hset_log2);
    return (size_t)T * 8 + (size_t)T * 8 + tb + (size_t)words * 8 + (size_t)kResCap * 4 + (size_t)kCandCap * 4 + 64;
}

__global__ void __launch_bounds__(512, 2) query_batch_kernel(QueryArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *keys_s = reinterpret_cast<uint64_t *>(smem_raw);
    uint32_t *lo_s = reinterpret_cast<uint32_t *>(keys_s + a.T);
    uint32_t *len_s = lo_s + a.T;
    uint64_t *tbuf = reinterpret_cast<uint64_t *>(len_s + a.T);   // 8T bytes after keys_s: 8-aligned
    uint32_t *hset = reinterpret_cast<uint32_t *>(tbuf);
    const size_t tb_words = ((size_t)a.W > ((size_t)1 << a.hset_log2) / 2) ? a.W : ((size_t)1 << a.hset_log2) / 2;
    uint64_t *q_s = tbuf + tb_words;
    uint32_t *res_s = reinterpret_cast<uint32_t *>(q_s + a.words);
    uint32_t *cand_s = res_s + kResCap;        // a chunk's new candidates
    __shared__ unsigned long long s_qi;
    __shared__ uint32_t s_nres, s_ncand;
    __shared__ unsigned long long red64[32];
    __shared__ ulonglong2 s_sigm[kSigLevels + 1];   // the query's occupancy levels (sig_bound)
    __shared__ uint32_t s_nsurv;

    const uint32_t tid = threadIdx.x, B = blockDim.x;
    const uint32_t lane = tid & 31, warp = tid >> 5, nwarps = B >> 5;
    const uint32_t L = a.W - 1;
    uint32_t *bm = a.bitmaps + (uint64_t)blockIdx.x * a.bm_words;
    const uint32_t hcap = 1u << a.hset_log2;

    for (;;) {
        if (tid == 0) s_qi = atomicAdd(a.work, 1ULL);
        __syncthreads();
        const uint64_t qi = s_qi;
        if (qi >= a.nq) break;
        if (a.redo_cap && a.run_base[qi] + a.res_cnt[qi] <= a.redo_cap) {   // its run fitted (block-uniform)
            __syncthreads();
            continue;
        }
        const uint32_t radius = a.radii ? a.radii[qi] : a.radius;
        load_query(a, qi, q_s, s_sigm);
        query_s1(a, qi, q_s, keys_s, tbuf);
        uint32_t nt, Tq;
        const unsigned long long E = probe_ranges(a, radius, keys_s, lo_s, len_s, red64, nt, Tq);
        const bool bitmap_mode = E > (hcap >> 1);
        // more bucket entries than bitmap words: mark the bitmap and sweep it once
        const bool sweep_mode = bitmap_mode && E > a.bm_words;
        const int mode = sweep_mode ? DEDUP_MARK : (bitmap_mode ? DEDUP_BITMAP : DEDUP_HSET);
        if ((a.heavy_from_bitmap ? bitmap_mode : sweep_mode) && a.heavy_q &&
            E <= kHeavyMaxEntries) {   // block-uniform: query_heavy_kernel answers it, with these keys
            __shared__ unsigned long long s_hpos;
            if (tid == 0) {
                s_hpos = atomicAdd(a.heavy_n, 1ULL);
                a.heavy_q[s_hpos] = qi;
            }
            __syncthreads();
            if (a.hkeys)
                for (uint32_t tau = tid; tau < a.T; tau += B) a.hkeys[s_hpos * a.T + tau] = keys_s[tau];
            __syncthreads();
            continue;
        }
        // the bucket entries as one list (positions in 32 bits) for the hash-set and bitmap
        // modes; the marking of a very heavy query, and a query of 2^32 entries or more, walk
        // their runs lane by lane instead (measured faster for the marking, whose work is the
        // fire-and-forget reductions, and no limit on the positions)
        const bool listed = !sweep_mode && E <= 0xFFFFFFFFull - (unsigned long long)B * kU;
        const uint32_t E32 = listed ? (uint32_t)E : 0u;
        uint32_t *off_s = len_s;   // len_s becomes the runs' exclusive prefix
        if (listed) runs_prefix(len_s, Tq, red64);
        if (!bitmap_mode)
            for (uint32_t i = tid; i < hcap; i += B) hset[i] = kEmpty;
        if (tid == 0) {
            s_nres = 0;
            s_ncand = 0;
        }
        __syncthreads();

        // ---- S2b + S3 (chunks of the list): collisions -> dedup -> verify of the new candidates
        const ulonglong2 sq = a.sig ? s_sigm[1] : make_ulonglong2(0, 0);
        Counters c;
        for (uint32_t base = 0; base < E32; base += B * kU) {
            Chunk<> ch;
            load_chunk(a, keys_s, lo_s, off_s, Tq, nt, L, E32, base, ch);
            uint32_t ids[kU], old[kU];
            bool coll[kU];
#pragma unroll
            for (int k = 0; k < kU; ++k) {
                coll[k] = entry_fp(ch.en[k], a.ent_ib) == ch.fp[k];
                ids[k] = entry_id(ch.en[k], a.ent_ib);
                old[k] = 0;
            }
#pragma unroll
            for (int k = 0; k < kU; ++k) coll[k] = coll[k] && FCLSH_CHECK(ids[k] < a.n, 0x0104);
            if (mode == DEDUP_MARK) {   // mark only (fire-and-forget reductions); the sweep verifies
#pragma unroll
                for (int k = 0; k < kU; ++k)
                    if (coll[k]) {
                        c.coll++;
                        atomicOr(bm + (ids[k] >> 5), 1u << (ids[k] & 31));
                    }
                continue;   // block-uniform
            }
#pragma unroll
            for (int k = 0; k < kU; ++k)   // the chunk's dedup operations, issued back to back
                if (coll[k]) {
                    c.coll++;
                    const uint32_t bit = 1u << (ids[k] & 31);
                    if (mode == DEDUP_BITMAP)
                        old[k] = atomicOr(bm + (ids[k] >> 5), bit) & bit;
                    else
                        old[k] = hset_insert(hset, a.hset_log2, ids[k]) ? 0u : 1u;
                }
#pragma unroll
            for (int k = 0; k < kU; ++k) push_cand(coll[k] && !old[k], ids[k], cand_s, &s_ncand);
            __syncthreads();
            verify_list(a, q_s, cand_s, s_ncand, radius, sq, s_sigm, c, res_s, &s_nres, &s_nsurv);
            __syncthreads();
            if (tid == 0) s_ncand = 0;
            __syncthreads();
        }
        if (!listed) {
            // marking (sweep mode) or a query with 2^32 bucket entries or more: warps take 32
            // tables, a lane walks its own short run, the warp a long one (the runs' lengths are
            // still in len_s)
            for (uint32_t base = warp * 32; base < Tq; base += nwarps * 32) {
                const uint32_t j = base + lane;
                const bool has = j < Tq;
                const uint32_t tau = has ? probed_table(j, nt, L) : 0;
                const uint32_t lo = has ? lo_s[j] : 0, len = has ? len_s[j] : 0;
                const uint64_t fp = has ? keys_s[tau] >> a.slot_bits : 0;
                const uint64_t *row = a.ent + (uint64_t)tau * a.n;
                const uint32_t short_len = len <= a.inline_len ? len : 0;
                const uint32_t maxs = __reduce_max_sync(0xffffffffu, short_len);
                for (uint32_t e = 0; e < maxs; ++e) {
                    const bool act = e < short_len;
                    const uint64_t en = act ? __ldg(row + lo + e) : 0;
                    process_entry(a, q_s, hset, bm, mode, radius, act && entry_fp(en, a.ent_ib) == fp,
                                  entry_id(en, a.ent_ib), c, res_s, &s_nres, sq, s_sigm);
                }
                uint32_t lmask = __ballot_sync(0xffffffffu, len > a.inline_len);
                while (lmask) {
                    const uint32_t src = __ffs(lmask) - 1;
                    lmask &= lmask - 1;
                    const uint32_t l_lo = __shfl_sync(0xffffffffu, lo, src);
                    const uint32_t l_len = __shfl_sync(0xffffffffu, len, src);
                    const uint64_t l_fp = __shfl_sync(0xffffffffu, fp, src);
                    const uint32_t l_tau = __shfl_sync(0xffffffffu, tau, src);
                    const uint64_t *lrow = a.ent + (uint64_t)l_tau * a.n + l_lo;
                    for (uint32_t cbase = 0; cbase < l_len; cbase += 32) {
                        const uint32_t e = cbase + lane;
                        const bool act = e < l_len;
                        const uint64_t en = act ? __ldg(lrow + e) : 0;
                        process_entry(a, q_s, hset, bm, mode, radius, act && entry_fp(en, a.ent_ib) == l_fp,
                                      entry_id(en, a.ent_ib), c, res_s, &s_nres, sq, s_sigm);
                    }
                }
            }
        }
        if (sweep_mode) {
            // S2/S3 for a very heavy query: every candidate is marked; sweep the bitmap (warps
            // take 32 consecutive words, a lane a word, no block barrier), verify each marked id
            // (a lane reads its point whole: 32 points in flight per warp), and leave only the
            // hits marked (cleared below)
            __threadfence();
            __syncthreads();
            for (uint64_t w0 = (uint64_t)warp * 32; w0 < a.bm_words; w0 += (uint64_t)nwarps * 32) {
                const uint64_t wi = w0 + lane;
                const uint32_t bits = wi < a.bm_words ? __ldcg(bm + wi) : 0u;
                c.cand += __popc(bits);
                uint32_t rem = bits, hits = 0;
                while (__any_sync(0xffffffffu, rem != 0)) {
                    bool hit = false;
                    uint32_t id = 0;
                    if (rem) {
                        const uint32_t b = __ffs(rem) - 1;
                        rem &= rem - 1;
                        id = (uint32_t)(wi * 32 + b);
                        hit = sig_pass(a, id, sq, s_sigm, radius) && distance_to(a, q_s, id) <= radius;
                        if (hit) hits |= 1u << b;
                    }
                    append_hits(hit, id, c, res_s, &s_nres);
                }
                if (bits) bm[wi] = hits;
            }
        }
        const unsigned long long tc = block_sum(c.coll, red64);
        const unsigned long long td = block_sum(c.cand, red64);
        const uint32_t nres = s_nres;   // read after block_sum's barriers
        __shared__ unsigned long long s_base;
        if (sweep_mode && nres <= kResCap) {   // the hits are listed: clear their words
            for (uint32_t i = tid; i < nres; i += B) bm[res_s[i] >> 5] = 0;
            __syncthreads();
        }
        if (bitmap_mode && !sweep_mode) {   // leave the CTA's bitmap all-zero: the list again
            for (uint32_t base = 0; base < E32; base += B * kU) {
                Chunk<> ch;
                load_chunk(a, keys_s, lo_s, off_s, Tq, nt, L, E32, base, ch);
#pragma unroll
                for (int k = 0; k < kU; ++k)
                    if (ch.fp[k] != kNoFp) bm[entry_id(ch.en[k], a.ent_ib) >> 5] = 0;
            }
            if (!listed)
                for (uint32_t j = tid; j < Tq; j += B) {
                    const uint64_t *row = a.ent + (uint64_t)probed_table(j, nt, L) * a.n + lo_s[j];
                    const uint32_t len = len_s[j];
                    for (uint32_t e = 0; e < len; ++e) bm[entry_id(__ldg(row + e), a.ent_ib) >> 5] = 0;
                }
            __syncthreads();
        }
        if (nres <= kResCap) {
            block_sort_u32(res_s, nres);
            if (tid == 0) s_base = a.redo_cap ? a.run_base[qi] : atomicAdd(a.cursor, (unsigned long long)nres);
            __syncthreads();
            const unsigned long long base = s_base;
            for (uint32_t i = tid; i < nres; i += B)
                if (base + i < a.cap) a.runs[base + i] = res_s[i];
        } else {
            // More hits than shared memory holds (only in bitmap mode): mark every hit in
            // the bitmap (the sweep left exactly the hits marked), then read the ids out in
            // ascending order and clear it again.
            for (uint32_t base = 0; !sweep_mode && base < E32; base += B * kU) {   // the list again
                Chunk<> ch;
                load_chunk(a, keys_s, lo_s, off_s, Tq, nt, L, E32, base, ch);
#pragma unroll
                for (int k = 0; k < kU; ++k) {
                    if (entry_fp(ch.en[k], a.ent_ib) != ch.fp[k]) continue;
                    const uint32_t id = entry_id(ch.en[k], a.ent_ib);
                    if (sig_pass(a, id, sq, s_sigm, radius) && distance_to(a, q_s, id) <= radius)
                        atomicOr(bm + (id >> 5), 1u << (id & 31));
                }
            }
            for (uint32_t j = (sweep_mode || listed) ? Tq : tid; j < Tq; j += B) {
                const uint32_t tau = probed_table(j, nt, L);
                const uint64_t *row = a.ent + (uint64_t)tau * a.n + lo_s[j];
                const uint32_t len = len_s[j];
                const uint64_t fp = keys_s[tau] >> a.slot_bits;
                for (uint32_t e = 0; e < len; ++e) {
                    const uint64_t en = __ldg(row + e);
                    if (entry_fp(en, a.ent_ib) != fp) continue;
                    const uint32_t id = entry_id(en, a.ent_ib);
                    if (sig_pass(a, id, sq, s_sigm, radius) && distance_to(a, q_s, id) <= radius)
                        atomicOr(bm + (id >> 5), 1u << (id & 31));
                }
            }
            if (tid == 0) s_base = a.redo_cap ? a.run_base[qi] : atomicAdd(a.cursor, (unsigned long long)nres);
            __syncthreads();
            bitmap_readout(a, bm, s_base, red64);
        }
        if (tid == 0) {
            a.coll[qi] = tc;
            a.cand[qi] = td;
            a.res_cnt[qi] = nres;
            a.run_base[qi] = s_base;
        }
        __syncthreads();
    }
}

// Dynamic shared memory of query_heavy_kernel with windows of win_bits ids: the keys, the
// bucket ranges and their prefix, the query, the hit list, the candidate list and the window
// (which also serves S1 as its W-word transform buffer).
size_t heavy_smem_bytes(uint32_t T, uint32_t words, uint32_t win_bits)
{
    return (size_t)T * 16 + (size_t)words * 8 + (size_t)(kResCap + kHeavyCand) * 4 + (size_t)win_bits / 8;
}

// Very heavy queries -- more bucket entries than the CTA's n-bit bitmap has words, which
// query_batch_kernel lists in heavy_q -- answered by one block of 32 warps per SM, taking the
// listed queries in turn.  S1 and the probes as in the batch kernel.  The duplicate
// elimination of S2 marks the query's bucket entries in a bitmap window held in shared memory,
// one window of win_bits ids after another (each window walks the bucket entries again: a
// shared-memory atomic per collision in place of one on a bitmap in L2); #Collisions is counted
// on the first window.  S3 then takes the window's marked ids -- its distinct candidates -- in
// ascending order, in lists of kHeavyCand verified block-wide.  Hits collect in shared memory
// and are sorted there; a query with more than kResCap hits also marks the rest in the CTA's
// bitmap in global memory and reads its ids out of it in order, leaving it all-zero.
__global__ void __launch_bounds__(kHeavyThreads, 1) query_heavy_kernel(QueryArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *keys_s = reinterpret_cast<uint64_t *>(smem_raw);
    uint32_t *lo_s = reinterpret_cast<uint32_t *>(keys_s + a.T);
    uint32_t *off_s = lo_s + a.T;                                   // run lengths, then their prefix
    uint64_t *q_s = reinterpret_cast<uint64_t *>(off_s + a.T);      // 16T bytes in: 8-aligned
    uint32_t *res_s = reinterpret_cast<uint32_t *>(q_s + a.words);
    uint32_t *cand_s = res_s + kResCap;
    uint64_t *win = reinterpret_cast<uint64_t *>(cand_s + kHeavyCand);   // 8-aligned (kResCap + kHeavyCand even)
    uint32_t *win32 = reinterpret_cast<uint32_t *>(win);
    __shared__ unsigned long long s_h, s_base;
    __shared__ uint32_t s_nres, s_nspill;
    __shared__ unsigned long long red64[32];
    __shared__ ulonglong2 s_sigm[kSigLevels + 1];

    const uint32_t tid = threadIdx.x, B = blockDim.x, L = a.W - 1;
    const uint32_t lane = tid & 31, warp = tid >> 5, nwarps = B >> 5;
    uint32_t *bm = a.bitmaps + (uint64_t)blockIdx.x * a.bm_words;
    uint32_t *spill = a.spill + (uint64_t)blockIdx.x * a.spill_cap;   // ids of the windows after the first
    const uint64_t pol_stream = l2_policy_evict_first(), pol_keep = l2_policy_evict_last();
    const unsigned long long nheavy = *a.heavy_n;   // final: written by the batch kernel before this launch

    for (;;) {
        if (tid == 0) s_h = atomicAdd(a.heavy_work, 1ULL);
        __syncthreads();
        const unsigned long long h = s_h;
        if (h >= nheavy) break;
        const uint64_t qi = a.heavy_q[h];
        if (!FCLSH_CHECK(qi < a.nq, 0x0110)) break;   // block-uniform
        const uint32_t radius = a.radii ? a.radii[qi] : a.radius;
        load_query(a, qi, q_s, s_sigm);
        if (a.hkeys) {   // S1 was done by the batch kernel, which listed the query
            for (uint32_t tau = tid; tau < a.T; tau += B) keys_s[tau] = a.hkeys[h * a.T + tau];
            __syncthreads();
        } else {
            query_s1(a, qi, q_s, keys_s, win);
        }
        uint32_t nt, Tq;
        const unsigned long long E = probe_ranges(a, radius, keys_s, lo_s, off_s, red64, nt, Tq);
        const uint32_t E32 = (uint32_t)min(E, kHeavyMaxEntries);   // the batch kernel lists only E <= the limit
        runs_prefix(off_s, Tq, red64);
        if (tid == 0) {
            s_nres = 0;
            s_nspill = 0;
        }
        __syncthreads();
        const ulonglong2 sq = a.sig ? s_sigm[1] : make_ulonglong2(0, 0);
        Counters c;

        for (uint64_t w_lo = 0; w_lo < a.n; w_lo += a.win_bits) {
            const uint64_t nbits = min((uint64_t)a.win_bits, a.n - w_lo);
            const uint32_t nw = (uint32_t)((nbits + 63) >> 6);
            for (uint32_t i = tid; i < nw; i += B) win[i] = 0;
            __syncthreads();
            // S2: mark the window's ids among the collisions (shared-memory reductions).  The
            // first window walks the bucket entries and lists the collisions of later windows in
            // the CTA's spill list (4 bytes an id, appended a warp at a time); later windows read
            // that list, or walk the entries again when it overflowed.
            const uint32_t nspill = s_nspill;   // final: written before the previous window's barriers
            if (w_lo != 0 && nspill <= a.spill_cap) {
                for (uint32_t i0 = 0; i0 < nspill; i0 += 8 * B) {   // eight loads in flight per thread
                    uint32_t id[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const uint32_t i = i0 + u * B + tid;
                        id[u] = i < nspill ? spill[i] : 0xFFFFFFFFu;
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const uint64_t rel = (uint64_t)id[u] - w_lo;
                        if (id[u] != 0xFFFFFFFFu && rel < nbits) atomicOr(win32 + (rel >> 5), 1u << (rel & 31));
                    }
                }
            } else {
                for (uint32_t base = 0; base < E32; base += B * kHeavyU) {
                    Chunk<kHeavyU> ch;
                    load_chunk<kHeavyU, true>(a, keys_s, lo_s, off_s, Tq, nt, L, E32, base, ch, pol_stream);
#pragma unroll
                    for (int k = 0; k < kHeavyU; ++k) {
                        const uint32_t id = entry_id(ch.en[k], a.ent_ib);
                        const bool coll = entry_fp(ch.en[k], a.ent_ib) == ch.fp[k] && FCLSH_CHECK(id < a.n, 0x0111);
                        const uint64_t rel = (uint64_t)id - w_lo;   // wraps past the window for id < w_lo
                        if (coll && rel < nbits) atomicOr(win32 + (rel >> 5), 1u << (rel & 31));
                        if (w_lo != 0) continue;   // block-uniform
                        if (coll) c.coll++;
                        const bool later = coll && rel >= nbits;
                        const uint32_t m = __ballot_sync(0xffffffffu, later);
                        if (m) {
                            const uint32_t leader = __ffs(m) - 1;
                            uint32_t at = 0;
                            if (lane == leader) at = atomicAdd(&s_nspill, (uint32_t)__popc(m));
                            at = __shfl_sync(0xffffffffu, at, leader) + __popc(m & lanemask_lt());
                            if (later && at < a.spill_cap) spill[at] = id;
                        }
                    }
                }
            }
            __syncthreads();
            // S3: warps sweep the window 32 words at a time, a lane taking the marked ids of its
            // word (the window's distinct candidates) four at a time.  With the pre-filter their
            // signatures are loaded together and bounded; the candidates that pass (all of them
            // without it) join the warp's own list of kWarpCand, which the warp verifies when the
            // next ones would not fit and at the window's end (no block barrier until then).
            uint32_t *wbuf = cand_s + warp * kWarpCand;
            uint32_t nl = 0;   // the warp's listed candidates
            for (uint32_t w0 = warp * 32; w0 < nw; w0 += nwarps * 32) {
                const uint32_t w = w0 + lane;
                uint64_t bits = w < nw ? win[w] : 0ULL;
                while (__any_sync(0xffffffffu, bits != 0)) {
                    uint32_t id[4];
                    ulonglong2 sx[4];
                    bool in[4];
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        in[f] = bits != 0;
                        const uint32_t b = in[f] ? (uint32_t)(__ffsll((long long)bits) - 1) : 0u;
                        bits &= bits - 1;
                        id[f] = (uint32_t)(w_lo + (uint64_t)w * 64 + b);
                        sx[f] = in[f] && a.sig ? ld_nc_hint2(reinterpret_cast<const ulonglong2 *>(a.sig) + id[f], pol_keep)
                                               : make_ulonglong2(0, 0);
                    }
                    uint32_t bal[4], total = 0;
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        if (in[f]) c.cand++;
                        const bool pass = in[f] && (!a.sig || sig_bound(sx[f], sq, s_sigm) <= radius);
                        bal[f] = __ballot_sync(0xffffffffu, pass);
                        total += __popc(bal[f]);
                    }
                    if (nl + total > kWarpCand) {   // warp-uniform
                        __syncwarp();
                        verify_warp(a, q_s, wbuf, nl, radius, c, res_s, &s_nres, bm);
                        __syncwarp();
                        nl = 0;
                    }
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        if ((bal[f] >> lane) & 1) wbuf[nl + __popc(bal[f] & lanemask_lt())] = id[f];
                        nl += __popc(bal[f]);
                    }
                }
            }
            __syncwarp();
            if (nl) verify_warp(a, q_s, wbuf, nl, radius, c, res_s, &s_nres, bm);   // warp-uniform
            __syncthreads();   // every warp's sweep before the next window is cleared
        }
        const unsigned long long tc = block_sum(c.coll, red64);
        const unsigned long long td = block_sum(c.cand, red64);
        const uint32_t nres = s_nres;   // read after block_sum's barriers
        if (nres <= kResCap) {
            block_sort_u32(res_s, nres);
            if (tid == 0) s_base = a.redo_cap ? a.run_base[qi] : atomicAdd(a.cursor, (unsigned long long)nres);
            __syncthreads();
            const unsigned long long base = s_base;
            for (uint32_t i = tid; i < nres; i += B)
                if (base + i < a.cap) a.runs[base + i] = res_s[i];
        } else {
            // the first kResCap hits are listed, the rest marked: mark the listed ones too and
            // read every hit out of the bitmap in order
            for (uint32_t i = tid; i < kResCap; i += B) atomicOr(bm + (res_s[i] >> 5), 1u << (res_s[i] & 31));
            __threadfence_block();
            if (tid == 0) s_base = a.redo_cap ? a.run_base[qi] : atomicAdd(a.cursor, (unsigned long long)nres);
            __syncthreads();
            bitmap_readout(a, bm, s_base, red64);
        }
        if (tid == 0) {
            a.coll[qi] = tc;
            a.cand[qi] = td;
            a.res_cnt[qi] = nres;
            a.run_base[qi] = s_base;
        }
        __syncthreads();
    }
}

// CSR layout of the runs: ids[offs[q] + i] = runs[run_base[q] + i].
// Blocks take equal ranges of the output positions (a query with many hits is copied by many
// blocks): one binary search for the range's first query, then each thread walks forward.
__global__ void __launch_bounds__(256) gather_runs_kernel(const uint32_t *runs, const uint64_t *run_base,
                                                          const uint32_t *res_cnt, const uint64_t *offs, uint64_t nq,
                                                          uint64_t cap, uint32_t *ids)
{
    (void)res_cnt;   // the counts are the differences of offs
    __shared__ uint64_t s_q;
    const uint64_t total = offs[nq];
    const uint64_t per = ((total + gridDim.x - 1) / gridDim.x + blockDim.x - 1) / blockDim.x * blockDim.x;
    const uint64_t lo = blockIdx.x * per, hi = min(total, lo + per);
    if (lo >= hi) return;   // block-uniform
    if (threadIdx.x == 0) {   // the last query q with offs[q] <= lo
        uint64_t a = 0, b = nq;
        while (b - a > 1) {
            const uint64_t m = (a + b) >> 1;
            if (offs[m] <= lo) a = m;
            else b = m;
        }
        s_q = a;
    }
    __syncthreads();
    uint64_t q = s_q;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        while (q + 1 < nq && offs[q + 1] <= i) ++q;
        const uint64_t src = run_base[q] + (i - offs[q]);
        if (src < cap && i < cap) ids[i] = runs[src];
    }
}

// ---------------------------------------------------------------- plain path

// One query: every probed table in its own thread, duplicates removed by a global n-bit bitmap.
// The query's words sit in dynamic shared memory (words * 8 bytes).
__global__ void __launch_bounds__(256) query_plain_kernel(QueryArgs a, const uint64_t *keys, uint32_t *bitmap)
{
    extern __shared__ uint64_t q_s[];
    __shared__ ulonglong2 s_sigm[kSigLevels + 1];
    for (uint32_t w = threadIdx.x; w < a.words; w += blockDim.x) q_s[w] = a.queries[w];
    __syncthreads();
    if (a.sig && threadIdx.x < kSigBlocks)   // the query's occupancy levels (warps 0-3 of 256 threads)
        sig_levels(q_s, a.d, a.sig_block, threadIdx.x & 31, threadIdx.x >> 5, reinterpret_cast<uint32_t *>(s_sigm));
    __syncthreads();
    const ulonglong2 sq = a.sig ? s_sigm[1] : make_ulonglong2(0, 0);
    const uint32_t nt = rows_per_part(a, a.radius), j = blockIdx.x * blockDim.x + threadIdx.x;
    const bool has = j < a.t * nt;   // every lane stays: the long runs are walked by whole warps
    const uint32_t tau = has ? probed_table(j, nt, a.W - 1) : 0u;
    const uint64_t smask = (1ULL << a.slot_bits) - 1;
    const uint64_t key = has ? keys[tau] : 0;
    const uint64_t fp = key >> a.slot_bits;
    uint32_t lo = 0, hi = 0;
    if (has) {
        const uint32_t *O = a.offs + (uint64_t)tau * a.offs_stride + (key & smask);
        lo = O[0];
        hi = O[1];
    }
    unsigned long long coll = 0, cand = 0;
    // one bucket entry: a collision when its key bits match; a new candidate when its bit was clear
    auto entry = [&](uint64_t en, uint64_t f) {
        if (entry_fp(en, a.ent_ib) != f) return;
        const uint32_t id = entry_id(en, a.ent_ib);
        if (!FCLSH_CHECK(id < a.n, 0x0108)) return;
        coll++;
        const uint32_t bit = 1u << (id & 31);
        if (atomicOr(bitmap + (id >> 5), bit) & bit) return;
        cand++;
        if (sig_pass(a, id, sq, s_sigm, a.radius) && distance_to(a, q_s, id) <= a.radius) {
            const unsigned long long pos = atomicAdd(a.cursor, 1ULL);
            if (pos < a.cap) a.staged[pos] = id;
        }
    };
    constexpr uint32_t kLaneRun = 32;   // runs up to this long are walked by their own lane
    if (hi - lo <= kLaneRun) {
        const uint64_t *row = a.ent + (uint64_t)tau * a.n;
        for (uint32_t e = lo; e < hi; ++e) entry(row[e], fp);
    }
    uint32_t lmask = __ballot_sync(0xffffffffu, hi - lo > kLaneRun);
    const uint32_t lane = threadIdx.x & 31;
    while (lmask) {   // a long run: the warp's lanes take its entries together
        const uint32_t src = __ffs(lmask) - 1;
        lmask &= lmask - 1;
        const uint32_t l_lo = __shfl_sync(0xffffffffu, lo, src), l_hi = __shfl_sync(0xffffffffu, hi, src);
        const uint64_t l_fp = __shfl_sync(0xffffffffu, fp, src);
        const uint64_t *row = a.ent + (uint64_t)__shfl_sync(0xffffffffu, tau, src) * a.n;
        for (uint32_t e = l_lo + lane; e < l_hi; e += 32) entry(row[e], l_fp);
    }
    if (coll) atomicAdd(a.coll, coll);
    if (cand) atomicAdd(a.cand, cand);
}

// Sort up to 2048 ids of one query in one CTA (bitonic), in place.
__global__ void __launch_bounds__(1024) sort_small_kernel(unsigned long long *v, const unsigned long long *d_count)
{
    __shared__ unsigned long long s[2048];
    const uint32_t cnt = (uint32_t)*d_count;
    for (uint32_t i = threadIdx.x; i < 2048; i += blockDim.x) s[i] = i < cnt ? v[i] : ~0ULL;
    __syncthreads();
    for (uint32_t size = 2; size <= 2048; size <<= 1)
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t i = threadIdx.x; i < 1024; i += blockDim.x) {
                const uint32_t lo = 2 * i - (i & (stride - 1));
                const uint32_t hi = lo + stride;
                const bool up = ((lo & size) == 0);
                const unsigned long long x = s[lo], y = s[hi];
                if ((x > y) == up) {
                    s[lo] = y;
                    s[hi] = x;
                }
            }
            __syncthreads();
        }
    for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) v[i] = s[i];
}

// ---------------------------------------------------------------- brute force

constexpr int kBfQ = 128;   // queries per CTA tile

// Linear scan: every (query, point) pair within radius, XOR + popcount.
__global__ void __launch_bounds__(256) bruteforce_kernel(const uint64_t *__restrict__ points, uint64_t n,
                                                         uint32_t words, const uint64_t *__restrict__ queries,
                                                         uint64_t nq, uint32_t radius, unsigned long long *cursor,
                                                         unsigned long long *staged, uint64_t cap, uint32_t idbits,
                                                         uint32_t *res_cnt, uint64_t points_per_cta)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *qs = reinterpret_cast<uint64_t *>(smem_raw);   // [kBfQ][words]
    const uint64_t q0 = (uint64_t)blockIdx.y * kBfQ;
    const uint32_t qn = (uint32_t)((nq - q0) < kBfQ ? (nq - q0) : kBfQ);
    for (uint32_t i = threadIdx.x; i < qn * words; i += blockDim.x) qs[i] = queries[q0 * words + i];
    __syncthreads();
    const uint64_t p0 = (uint64_t)blockIdx.x * points_per_cta;
    const uint64_t p1 = (p0 + points_per_cta < n) ? p0 + points_per_cta : n;
    for (uint64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const uint64_t *x = points + p * words;
        if (words <= 4) {
            uint64_t xv[4] = {0, 0, 0, 0};
            for (uint32_t w = 0; w < words; ++w) xv[w] = __ldg(x + w);
            for (uint32_t q = 0; q < qn; ++q) {
                const uint64_t *qq = qs + q * words;
                uint32_t dist = 0;
#pragma unroll
                for (uint32_t w = 0; w < 4; ++w)
                    if (w < words) dist += __popcll(xv[w] ^ qq[w]);
                if (dist <= radius) {
                    const unsigned long long pos = atomicAdd(cursor, 1ULL);
                    if (pos < cap) staged[pos] = ((q0 + q) << idbits) | p;
                    atomicAdd(res_cnt + q0 + q, 1u);
                }
            }
        } else {
            for (uint32_t q = 0; q < qn; ++q) {
                const uint64_t *qq = qs + q * words;
                uint32_t dist = 0;
                for (uint32_t w = 0; w < words && dist <= radius; ++w) dist += __popcll(__ldg(x + w) ^ qq[w]);
                if (dist <= radius) {
                    const unsigned long long pos = atomicAdd(cursor, 1ULL);
                    if (pos < cap) staged[pos] = ((q0 + q) << idbits) | p;
                    atomicAdd(res_cnt + q0 + q, 1u);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- CSR

__global__ void extract_ids_kernel(const unsigned long long *sorted, const unsigned long long *d_count, uint64_t cap,
                                   uint64_t idmask, uint32_t *ids)
{
    unsigned long long cnt = *d_count;
    if (cnt > cap) cnt = cap;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cnt; i += (uint64_t)gridDim.x * blockDim.x)
        ids[i] = (uint32_t)(sorted[i] & idmask);
}

// ---------------------------------------------------------------- launchers

// The shared-memory limit is raised by query_batch_occupancy() before any launch
// (outside stream capture).
cudaError_t launch_query_batch(const QueryArgs &a, uint32_t grid, uint32_t block, size_t smem, cudaStream_t s)
{
    query_batch_kernel<<<grid, block, smem, s>>>(a);
    note_launch();
    return cudaGetLastError();
}

cudaError_t query_batch_occupancy(uint32_t block, size_t smem, int *ctas_per_sm)
{
    if (smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(query_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, query_batch_kernel, (int)block, smem);
}

// Raises query_heavy_kernel's shared-memory limit to smem; outside any stream capture.
cudaError_t query_heavy_prepare(size_t smem)
{
    return cudaFuncSetAttribute(query_heavy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_query_heavy(const QueryArgs &a, uint32_t grid, size_t smem, cudaStream_t s)
{
    query_heavy_kernel<<<grid, kHeavyThreads, smem, s>>>(a);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_query_plain(const QueryArgs &a, const uint64_t *keys, uint32_t *bitmap, cudaStream_t s)
{
    const uint32_t blocks = (a.T + 255) / 256;
    query_plain_kernel<<<blocks, 256, (size_t)a.words * 8, s>>>(a, keys, bitmap);   // <= 32 KB (d <= 262,144)
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_sort_small(unsigned long long *v, const unsigned long long *d_count, cudaStream_t s)
{
    sort_small_kernel<<<1, 1024, 0, s>>>(v, d_count);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_bruteforce(const uint64_t *points, uint64_t n, uint32_t words, const uint64_t *queries, uint64_t nq,
                              uint32_t radius, unsigned long long *cursor, unsigned long long *staged, uint64_t cap,
                              uint32_t idbits, uint32_t *res_cnt, int sm_count, cudaStream_t s)
{
    if (nq == 0 || n == 0) return cudaSuccess;
    const uint64_t qtiles = (nq + kBfQ - 1) / kBfQ;
    // enough point tiles that the grid covers the GPU several times
    uint64_t ptiles = ((uint64_t)sm_count * 8 + qtiles - 1) / qtiles;
    if (ptiles < 1) ptiles = 1;
    uint64_t ppc = (n + ptiles - 1) / ptiles;
    ppc = ((ppc + 255) / 256) * 256;
    ptiles = (n + ppc - 1) / ppc;
    const size_t smem = (size_t)kBfQ * words * 8;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(bruteforce_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)ptiles, (unsigned)qtiles);
    bruteforce_kernel<<<grid, 256, smem, s>>>(points, n, words, queries, nq, radius, cursor, staged, cap, idbits,
                                               res_cnt, ppc);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gather_runs(const uint32_t *runs, const uint64_t *run_base, const uint32_t *res_cnt,
                               const uint64_t *offs, uint64_t nq, uint64_t cap, uint32_t *ids, int sm_count, cudaStream_t s)
{
    if (nq == 0) return cudaSuccess;
    gather_runs_kernel<<<(unsigned)(sm_count * 8), 256, 0, s>>>(runs, run_base, res_cnt, offs, nq, cap, ids);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_extract_ids(const unsigned long long *sorted, const unsigned long long *d_count, uint64_t cap,
                               uint64_t idmask, uint32_t *ids, int sm_count, cudaStream_t s)
{
    extract_ids_kernel<<<(unsigned)(sm_count * 4), 256, 0, s>>>(sorted, d_count, cap, idmask, ids);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- point signatures

// One warp per point: lane l counts blocks l, l + 32, l + 64 and l + 96 (B coordinates each),
// the ballots give the point's 128-bit block-occupancy signature; the popcounts are summed
// per warp and added to *pop_total once per warp.
__global__ void __launch_bounds__(256) point_sig_kernel(const uint64_t *__restrict__ pts, uint64_t n, uint32_t words,
                                                        uint32_t d, uint32_t B, uint64_t *__restrict__ sig,
                                                        unsigned long long *pop_total)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long pop = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const uint64_t *x = pts + i * words;
        uint32_t q[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const uint32_t lo = (lane + 32u * h) * B;
            const uint32_t c = lo < d ? popc_range(x, lo, min(lo + B, d)) : 0u;
            pop += c;
            q[h] = __ballot_sync(0xffffffffu, c > 0);
        }
        if (lane == 0)
            reinterpret_cast<ulonglong2 *>(sig)[i] = make_ulonglong2((uint64_t)q[1] << 32 | q[0], (uint64_t)q[3] << 32 | q[2]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pop += __shfl_xor_sync(0xffffffffu, pop, o);
    if (lane == 0 && pop) atomicAdd(pop_total, pop);
}

cudaError_t launch_point_sig(const uint64_t *pts, uint64_t n, uint32_t words, uint32_t d, uint32_t sig_block,
                             uint64_t *sig, unsigned long long *pop_total, int sm_count, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = std::min<uint64_t>((n + 7) / 8, (uint64_t)sm_count * 16);
    point_sig_kernel<<<(unsigned)blocks, 256, 0, s>>>(pts, n, words, d, sig_block, sig, pop_total);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- sparse input

// Rows given as lists of set coordinates (CSR: row i = indices[indptr[i] .. indptr[i+1]))
// packed into bit vectors: one warp per row, each lane setting the bits of its entries
// with atomic ORs into the zeroed row.  Entries past nnz, coordinates >= d and rows whose
// bounds run backwards are skipped and flagged in *bad.
__global__ void __launch_bounds__(256) pack_sparse_kernel(const uint64_t *__restrict__ indptr,
                                                          const uint32_t *__restrict__ indices, uint64_t n,
                                                          uint64_t nnz, uint32_t d, uint32_t words,
                                                          unsigned long long *__restrict__ out, uint32_t *bad)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t i = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const uint64_t lo = indptr[i], hi = indptr[i + 1];
        if (hi < lo || hi > nnz) {
            if (lane == 0) atomicOr(bad, 1u);
            continue;
        }
        unsigned long long *row = out + i * words;
        for (uint64_t e = lo + lane; e < hi; e += 32) {
            const uint32_t c = indices[e];
            if (c >= d) {
                atomicOr(bad, 2u);
                continue;
            }
            atomicOr(row + (c >> 6), 1ULL << (c & 63));
        }
    }
}

cudaError_t launch_pack_sparse(const uint64_t *indptr, const uint32_t *indices, uint64_t n, uint64_t nnz, uint32_t d,
                               uint64_t *out, uint32_t *bad, int sm_count, cudaStream_t s)
{
    const uint32_t words = (d + 63) / 64;
    cudaError_t e = cudaMemsetAsync(out, 0, n * words * 8, s);
    if (e != cudaSuccess || n == 0) return e;
    const uint64_t blocks = std::min<uint64_t>((n + 7) / 8, (uint64_t)sm_count * 16);
    pack_sparse_kernel<<<(unsigned)blocks, 256, 0, s>>>(indptr, indices, n, nnz, d, words,
                                                        reinterpret_cast<unsigned long long *>(out), bad);
    note_launch();
    return cudaGetLastError();
}

FCLSH_CHECK_READER(check_first_query)

}  // namespace fclsh
