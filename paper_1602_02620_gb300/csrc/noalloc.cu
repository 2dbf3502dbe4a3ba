// noalloc.cu -- a one-query probe that allocates no memory.
//
// Some callers cannot call cudaMalloc while they query: code running under a
// memory pool or allocator it does not own, callers inside a framework whose
// allocator is busy or capped, and real-time loops where an allocation (and the
// device synchronisation cudaMalloc/cudaFree may cause) is not allowed.  For them
// fclsh_query_plain_noalloc answers one query with all of its scratch in the
// file-scope device array below, sized once for the largest supported index.
//
// The array is ordinary device memory of this library: every GPU that loads the
// library holds it (about 1.1 MB) until the process exits.  Its host-side symbol
// is only a stand-in, so host code never passes `g_noalloc_scratch` to a kernel;
// it passes the device address that cudaGetSymbolAddress returns, looked up once
// per device with that device current.
#include <mutex>

#include "common.cuh"

namespace fclsh {

constexpr uint64_t kNoallocMaxN = 1ULL << 22;   // points
constexpr uint32_t kNoallocMaxT = 4094;          // tables
constexpr uint64_t kNoallocBmWords = kNoallocMaxN / 32;
// layout (uint64 units): keys [kNoallocMaxT] | counters [4] | candidate bitmap | hit bitmap (uint32 words)
constexpr uint64_t kNoallocU64 = kNoallocMaxT + 4 + kNoallocBmWords;   // two bitmaps of kNoallocBmWords uint32

static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoallocU64];

namespace {

struct NoallocScratch {
    uint64_t *keys;            // [T]
    unsigned long long *cnt;   // [0] hits, [1] #Collisions, [2] #Candidates
    uint32_t *cand_bm;         // [bm_words]
    uint32_t *hit_bm;          // [bm_words]
};

NoallocScratch carve(uint64_t *base, uint64_t bm_words)
{
    NoallocScratch s;
    s.keys = base;
    s.cnt = reinterpret_cast<unsigned long long *>(base + kNoallocMaxT);
    s.cand_bm = reinterpret_cast<uint32_t *>(base + kNoallocMaxT + 4);
    s.hit_bm = s.cand_bm + bm_words;
    return s;
}

// Device address of the scratch array on the current device (set up once per device).
fclsh_status scratch_address(int device, uint64_t **out)
{
    static std::mutex mu;
    static uint64_t *addr[64] = {nullptr};
    if (device < 0 || device >= 64) {
        set_error("device ordinal %d out of range", device);
        return FCLSH_EINVAL;
    }
    std::lock_guard<std::mutex> g(mu);
    if (!addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        addr[device] = static_cast<uint64_t *>(p);
    }
    *out = addr[device];
    return FCLSH_OK;
}

// Probe every table of the probe rule for one query: mark each distinct candidate in cand_bm and
// each candidate within the radius in hit_bm (one thread per table).
__global__ void __launch_bounds__(256) noalloc_probe_kernel(QueryArgs a, NoallocScratch sc)
{
    __shared__ uint64_t q_s[256];
    for (uint32_t w = threadIdx.x; w < a.words; w += blockDim.x) q_s[w] = a.queries[w];
    __syncthreads();
    const uint32_t nt = rows_per_part(a, a.radius), j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.t * nt) return;
    const uint32_t tau = probed_table(j, nt, a.W - 1);
    const uint64_t key = sc.keys[tau];
    const uint64_t fp = key >> a.slot_bits;
    const uint32_t *O = a.offs + (uint64_t)tau * a.offs_stride + (key & ((1ULL << a.slot_bits) - 1));
    const uint32_t lo = O[0], hi = O[1];
    const uint64_t *row = a.ent + (uint64_t)tau * a.n;
    unsigned long long coll = 0, cand = 0;
    for (uint32_t e = lo; e < hi; ++e) {
        const uint64_t en = row[e];
        if (entry_fp(en, a.ent_ib) != fp) continue;
        const uint32_t id = entry_id(en, a.ent_ib);
        if (!FCLSH_CHECK(id < a.n, 0x0501)) continue;
        coll++;
        const uint32_t bit = 1u << (id & 31);
        if (atomicOr(sc.cand_bm + (id >> 5), bit) & bit) continue;
        cand++;
        const uint64_t *x = a.points + (uint64_t)id * a.words;
        uint32_t dist = 0;
        for (uint32_t w = 0; w < a.words; ++w) dist += __popcll(__ldg(x + w) ^ q_s[w]);
        if (dist <= a.radius) atomicOr(sc.hit_bm + (id >> 5), bit);
    }
    if (coll) atomicAdd(sc.cnt + 1, coll);
    if (cand) atomicAdd(sc.cnt + 2, cand);
}

// One block: read the hit bitmap in order, write ids ascending (up to cap) and the counts.
__global__ void __launch_bounds__(1024) noalloc_extract_kernel(NoallocScratch sc, uint64_t bm_words, uint32_t *ids_out,
                                                               uint64_t cap, uint64_t *counts_out)
{
    __shared__ unsigned long long warp_tot[32];
    __shared__ unsigned long long carry;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (uint64_t base = 0; base < bm_words; base += blockDim.x) {
        const uint64_t w = base + tid;
        const uint32_t bits = w < bm_words ? sc.hit_bm[w] : 0u;
        uint32_t c = __popc(bits), incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += u;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        unsigned long long before = carry;
        for (uint32_t v = 0; v < warp; ++v) before += warp_tot[v];
        unsigned long long pos = before + incl - c;
        uint32_t rest = bits;
        while (rest) {
            const uint32_t b = __ffs(rest) - 1;
            rest &= rest - 1;
            if (pos < cap) ids_out[pos] = (uint32_t)(w * 32 + b);
            ++pos;
        }
        __syncthreads();
        if (tid == 0) {
            unsigned long long t = 0;
            for (uint32_t v = 0; v < nw; ++v) t += warp_tot[v];
            carry += t;
        }
        __syncthreads();
    }
    if (tid == 0) {
        counts_out[0] = carry;
        counts_out[1] = sc.cnt[1];
        counts_out[2] = sc.cnt[2];
    }
}

}  // namespace

FCLSH_CHECK_READER(check_first_noalloc)

}  // namespace fclsh

using namespace fclsh;

extern "C" fclsh_status fclsh_query_plain_noalloc(const fclsh_index *cidx, const uint64_t *query, uint32_t radius,
                                                  uint32_t *ids_out, uint64_t cap, uint64_t *counts_out, void *stream)
{
    fclsh_index *idx = const_cast<fclsh_index *>(cidx);
    if (!idx || !query || !counts_out || (cap && !ids_out)) {
        set_error("NULL argument");
        return FCLSH_EINVAL;
    }
    if (radius > idx->r) {
        set_error("radius %u exceeds the build radius %u", radius, idx->r);
        return FCLSH_ERADIUS;
    }
    if (idx->n > kNoallocMaxN || idx->T > kNoallocMaxT || idx->words > 256) {
        set_error("fclsh_query_plain_noalloc supports n <= %llu points, T <= %u tables and d <= 16384 "
                  "(index has n = %llu, T = %u)",
                  (unsigned long long)kNoallocMaxN, kNoallocMaxT, (unsigned long long)idx->n, idx->T);
        return FCLSH_EINVAL;
    }
    FCLSH_CUDA(cudaSetDevice(idx->device));
    // the kernels read the query and write the outputs on the device: host memory is refused
    // here rather than faulting there
    if (!is_device_ptr(query) || !is_device_ptr(counts_out) || (cap && !is_device_ptr(ids_out))) {
        set_error("fclsh_query_plain_noalloc needs device memory for query, ids_out and counts_out");
        return FCLSH_EINVAL;
    }
    uint64_t *base = nullptr;
    fclsh_status st = scratch_address(idx->device, &base);
    if (st != FCLSH_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t bm_words = (idx->n + 31) / 32;
    NoallocScratch sc = carve(base, bm_words);
    // counters and both bitmaps start at zero on every call
    FCLSH_CUDA(cudaMemsetAsync(sc.cnt, 0, 4 * sizeof(unsigned long long) + 2 * bm_words * 4, s));
    const uint32_t L = idx->W - 1;
    for (uint32_t k = 0; k < idx->t; ++k)
        FCLSH_CUDA(launch_hash_part(idx, k, query, 1, sc.keys + (uint64_t)k * L, 1, s));
    QueryArgs a{};
    a.points = idx->points;
    a.n = idx->n;
    a.words = idx->words;
    a.t = idx->t;
    a.W = idx->W;
    a.T = idx->T;
    a.probe_rows = idx->tune.probe_rows;
    a.rep = idx->rep;
    a.ent_ib = idx->ent_ib;
    a.slot_bits = idx->slot_bits;
    a.offs = idx->offs;
    a.offs_stride = idx->offs_stride();
    a.ent = idx->ent;
    a.queries = query;
    a.radius = radius;
    noalloc_probe_kernel<<<(idx->T + 255) / 256, 256, 0, s>>>(a, sc);
    note_launch();
    noalloc_extract_kernel<<<1, 1024, 0, s>>>(sc, bm_words, ids_out, cap, counts_out);
    note_launch();
    FCLSH_CUDA(cudaGetLastError());
    return FCLSH_OK;
}
