// api.cu -- the C ABI of libfclsh (declared in include/fclsh.h): index build,
// batched / plain / brute-force queries, per-stream query contexts, timing and
// kernel-shape tuning.  Host code only orchestrates; every step of the hot path
// runs in the kernels of hash.cu, sort.cu and query.cu.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cstring>
#include <atomic>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

#include <nvtx3/nvToolsExt.h>

namespace fclsh {

// ---- declarations from query.cu / hash.cu

size_t query_smem_bytes(uint32_t T, uint32_t W, uint32_t words, uint32_t hset_log2);
cudaError_t launch_query_batch(const QueryArgs &a, uint32_t grid, uint32_t block, size_t smem, cudaStream_t s);
cudaError_t query_batch_occupancy(uint32_t block, size_t smem, int *ctas_per_sm);
size_t heavy_smem_bytes(uint32_t T, uint32_t words, uint32_t win_bits);
constexpr uint32_t kHeavySpillCap = 1u << 20;   // ids per heavy block's spill list (4 MB)
cudaError_t query_heavy_prepare(size_t smem);
cudaError_t launch_query_heavy(const QueryArgs &a, uint32_t grid, size_t smem, cudaStream_t s);
cudaError_t launch_query_plain(const QueryArgs &a, const uint64_t *keys, uint32_t *bitmap, cudaStream_t s);
cudaError_t launch_sort_small(unsigned long long *v, const unsigned long long *d_count, cudaStream_t s);
cudaError_t launch_bruteforce(const uint64_t *points, uint64_t n, uint32_t words, const uint64_t *queries, uint64_t nq,
                              uint32_t radius, unsigned long long *cursor, unsigned long long *staged, uint64_t cap,
                              uint32_t idbits, uint32_t *res_cnt, int sm_count, cudaStream_t s);
cudaError_t launch_extract_ids(const unsigned long long *sorted, const unsigned long long *d_count, uint64_t cap,
                               uint64_t idmask, uint32_t *ids, int sm_count, cudaStream_t s);
cudaError_t launch_gather_runs(const uint32_t *runs, const uint64_t *run_base, const uint32_t *res_cnt,
                               const uint64_t *offs, uint64_t nq, uint64_t cap, uint32_t *ids, int sm_count, cudaStream_t s);
size_t hash_smem_bytes(uint32_t W, uint32_t dk, uint32_t tile);
cudaError_t launch_pack_sparse(const uint64_t *indptr, const uint32_t *indices, uint64_t n, uint64_t nnz, uint32_t d,
                               uint64_t *out, uint32_t *bad, int sm_count, cudaStream_t s);

// ---------------------------------------------------------------- errors

static thread_local std::string g_err;

void set_error(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

fclsh_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return FCLSH_ENOMEM;
    }
    return FCLSH_ECUDA;
}

static fclsh_status fail(fclsh_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

// ---------------------------------------------------------------- launch accounting

static std::atomic<int64_t> g_launches{0};

void note_launch(uint64_t kernels) { g_launches.fetch_add((int64_t)kernels); }
uint64_t launch_count() { return (uint64_t)g_launches.load(); }
int64_t launch_count_adjust(int64_t delta) { return g_launches.fetch_add(delta) + delta; }

// ---------------------------------------------------------------- helpers

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static uint32_t bits_for(uint64_t v)   // bits needed for values 0..v-1 (at least 1)
{
    uint32_t b = 1;
    while (b < 64 && (1ULL << b) < v) ++b;
    return b;
}

// Device memory of the library comes from one stream-ordered pool per device that
// keeps freed memory (release threshold = all of it), so building indexes and
// query contexts again and again reuses memory instead of mapping it anew.
static cudaMemPool_t device_pool(int dev)
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {nullptr};
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> g(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = ~0ULL;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = p;
    }
    return pools[dev];
}

// Allocation-failure injection for tests of the out-of-memory paths: while >= 0, the
// device allocation that finds it at 0 fails with cudaErrorMemoryAllocation (and the
// countdown stops); each earlier one decrements it.
static std::atomic<int64_t> g_fail_alloc{-1};

static bool injected_alloc_failure()
{
    int64_t v = g_fail_alloc.load();
    while (v >= 0) {
        if (g_fail_alloc.compare_exchange_weak(v, v - 1)) return v == 0;
    }
    return false;
}

cudaError_t dev_alloc(void **p, size_t bytes)
{
    if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool = device_pool(dev);
    if (!pool) return cudaMalloc(p, bytes);
    e = cudaMallocFromPoolAsync(p, bytes, pool, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);   // usable on any stream from here on
    return e;
}

void dev_free(void *p)
{
    if (!p) return;
    cudaFreeAsync(p, 0);
}

// Allocation ordered on the legacy stream only: for memory that this stream alone uses
// until the caller synchronises it (the build), so no synchronisation here.
static cudaError_t dev_alloc_ordered(void **p, size_t bytes)
{
    if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool = device_pool(dev);
    if (!pool) return cudaMalloc(p, bytes);
    return cudaMallocFromPoolAsync(p, bytes, pool, 0);
}

// Device allocation list freed together on error.  `ordered`: every use is on the
// legacy stream, so allocation and release are stream-ordered and never synchronise.
struct DevAllocs {
    std::vector<void *> ptrs;
    bool ordered = false;
    DevAllocs() = default;
    explicit DevAllocs(bool on_legacy_stream) : ordered(on_legacy_stream) {}
    ~DevAllocs()
    {
        if (!ordered && !ptrs.empty()) cudaDeviceSynchronize();
        for (void *p : ptrs) dev_free(p);
    }
    template <typename T>
    cudaError_t alloc(T **p, size_t count)
    {
        *p = nullptr;
        if (count == 0) count = 1;
        cudaError_t e = ordered ? dev_alloc_ordered((void **)p, count * sizeof(T)) : dev_alloc((void **)p, count * sizeof(T));
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    void release()   // keep the allocations
    {
        ptrs.clear();
    }
};

// ---------------------------------------------------------------- tracing

// NVTX range for profilers and tracers (free when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// ---------------------------------------------------------------- timing

struct PendingTimer {
    int phase;
    cudaEvent_t a, b;
};
static std::mutex g_timer_mu;
static std::vector<std::pair<fclsh_index *, PendingTimer>> g_pending;

struct PhaseTimer {
    fclsh_index *idx;
    int phase;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    PhaseTimer(fclsh_index *i, int ph, cudaStream_t st) : idx(i), phase(ph), s(st)
    {
        if (idx && idx->timing) {
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            cudaEventRecord(a, s);
        }
    }
    ~PhaseTimer()
    {
        if (a) {
            cudaEventRecord(b, s);
            std::lock_guard<std::mutex> g(g_timer_mu);
            g_pending.push_back({idx, PendingTimer{phase, a, b}});
        }
    }
};

static void resolve_timers(fclsh_index *idx)
{
    std::lock_guard<std::mutex> g(g_timer_mu);
    std::vector<std::pair<fclsh_index *, PendingTimer>> keep;
    for (auto &pt : g_pending) {
        if (pt.first != idx) {
            keep.push_back(pt);
            continue;
        }
        if (cudaEventQuery(pt.second.b) != cudaSuccess) {
            cudaGetLastError();
            keep.push_back(pt);
            continue;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, pt.second.a, pt.second.b);
        idx->ms[pt.second.phase] += ms;
        idx->cnt[pt.second.phase] += 1;
        cudaEventDestroy(pt.second.a);
        cudaEventDestroy(pt.second.b);
    }
    g_pending.swap(keep);
}

static void drop_timers(fclsh_index *idx)
{
    std::lock_guard<std::mutex> g(g_timer_mu);
    std::vector<std::pair<fclsh_index *, PendingTimer>> keep;
    for (auto &pt : g_pending) {
        if (pt.first == idx) {
            cudaEventSynchronize(pt.second.b);
            cudaEventDestroy(pt.second.a);
            cudaEventDestroy(pt.second.b);
        } else {
            keep.push_back(pt);
        }
    }
    g_pending.swap(keep);
}

}  // namespace fclsh

using namespace fclsh;

// ---------------------------------------------------------------- query context

struct fclsh_qctx {
    fclsh_index *idx = nullptr;
    unsigned long long *counters = nullptr;   // [0] work, [1] cursor, [2] heavy queries listed, [3] heavy work
    uint32_t *runs = nullptr;                 // [cap] each query's sorted hits
    uint64_t cap = 0;
    uint64_t nq_cap = 0;
    uint64_t *run_base = nullptr;
    uint32_t *res_cnt = nullptr;
    uint64_t *res_offs = nullptr;
    uint32_t *res_ids = nullptr;
    unsigned long long *coll = nullptr, *cand = nullptr;
    uint64_t *scan_part = nullptr;
    uint32_t *bitmaps = nullptr;
    uint32_t grid = 0, block = 0;
    size_t smem = 0;
    uint64_t *heavy_q = nullptr;   // [nq_cap] the batch's very heavy queries, for query_heavy_kernel
    uint32_t win_bits = 0;         // its window of ids (0: the batch kernel sweeps heavy queries itself)
    size_t heavy_smem = 0;
    uint32_t *spill = nullptr;     // [heavy blocks][spill_cap]: ids of the windows after the first
    uint32_t spill_cap = 0;
    uint64_t *hkeys = nullptr;     // [nq_cap][T]: the keys of the queries listed for the heavy kernel
    uint64_t hkeys_cap = 0;
    uint64_t *qbuf = nullptr;   // device copy of host queries
    uint64_t qbuf_cap = 0;
    uint32_t *rbuf = nullptr;   // device copy of host radii
    uint64_t rbuf_cap = 0;
    uint64_t *qkeys = nullptr;  // classic LSH: the batch's query keys [T][nq], hashed before the query kernel
    uint64_t qkeys_cap = 0;
    // last batch
    const uint64_t *last_q = nullptr;
    uint64_t last_nq = 0;
    uint32_t last_radius = 0;
    const uint32_t *last_radii = nullptr;
    cudaStream_t last_stream = nullptr;
    bool pending = false;
    // graph cache
    cudaGraphExec_t gexec = nullptr;
    const uint64_t *g_q = nullptr;
    uint64_t g_nq = 0;
    uint32_t g_radius = 0;
    const uint32_t *g_radii = nullptr;
    cudaStream_t g_stream = nullptr;
    uint64_t g_cap = 0;
    fclsh_tuning g_tune{};
    bool g_seen = false;       // the g_* shape ran once eagerly; its next repeat is captured
    uint64_t g_kernels = 0;
    cudaStream_t own = nullptr;   // used for the NULL stream: blocking, so it orders after legacy-stream work
};

static void ctx_free_buffers(fclsh_qctx *c)
{
    void *ps[] = {c->counters, c->runs, c->run_base, c->res_cnt, c->res_offs, c->res_ids, c->coll,
                  c->cand, c->scan_part, c->bitmaps, c->qbuf, c->rbuf, c->qkeys, c->heavy_q, c->spill, c->hkeys};
    for (void *p : ps)
        if (p) dev_free(p);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->own) cudaStreamDestroy(c->own);
}

static fclsh_status ctx_shape(fclsh_qctx *c)
{
    fclsh_index *idx = c->idx;
    const fclsh_tuning &tu = idx->tune;
    const uint32_t block = tu.query_block;
    const size_t smem = query_smem_bytes(idx->T, idx->W, idx->words, tu.hash_set_log2);
    if (smem > idx->smem_optin)
        return fail(FCLSH_EINVAL, "query kernel needs %zu bytes of shared memory (limit %zu)", smem, idx->smem_optin);
    int occ = 0;
    FCLSH_CUDA(query_batch_occupancy(block, smem, &occ));
    if (occ < 1) return fail(FCLSH_EINVAL, "query kernel does not fit on an SM (block %u, smem %zu)", block, smem);
    const uint32_t per_sm = std::max(1u, std::min<uint32_t>((uint32_t)occ, tu.query_ctas_per_sm));
    const uint32_t grid = per_sm * (uint32_t)idx->sm_count;
    if (grid != c->grid) {
        if (c->bitmaps) dev_free(c->bitmaps);
        c->bitmaps = nullptr;
        c->grid = 0;   // a failed allocation below leaves no shape that looks usable
        if (c->gexec) {   // a captured batch refers to the old bitmaps
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        c->g_seen = false;
        const uint64_t bm_words = (idx->n + 31) / 32;
        FCLSH_CUDA(dev_alloc((void **)&c->bitmaps, (size_t)grid * bm_words * 4));
        FCLSH_CUDA(cudaMemset(c->bitmaps, 0, (size_t)grid * bm_words * 4));
        c->grid = grid;
    }
    c->block = block;
    c->smem = smem;
    // the heavy-query kernel: windows of ids as large as shared memory allows (at most n, at
    // least the 64 W bits that S1's transform buffer takes), or at most tu.heavy_kernel ids
    c->win_bits = 0;
    c->heavy_smem = 0;
    if (tu.heavy_kernel) {
        const size_t fixed = heavy_smem_bytes(idx->T, idx->words, 0) + 4096;   // + the kernel's static arrays
        const uint64_t room = idx->smem_optin > fixed ? ((uint64_t)(idx->smem_optin - fixed) * 8) & ~63ULL : 0;
        const uint64_t need = idx->classic_k ? 64 : 64ULL * idx->W;
        uint64_t wb = std::min<uint64_t>(room, (idx->n + 63) & ~63ULL);
        if (tu.heavy_kernel >= 64) wb = std::min<uint64_t>(wb, (uint64_t)tu.heavy_kernel & ~63ULL);
        wb = std::max(wb, need);
        if (wb <= room) {
            c->heavy_smem = heavy_smem_bytes(idx->T, idx->words, (uint32_t)wb);
            FCLSH_CUDA(query_heavy_prepare(c->heavy_smem));
            c->win_bits = (uint32_t)wb;
        }
    }
    // several windows: the spill lists of the heavy kernel's blocks (a query whose collisions
    // past the first window overflow its list walks the bucket entries again)
    uint32_t want_cap = c->win_bits && c->win_bits < idx->n ? kHeavySpillCap : 0;
    if (want_cap && tu.heavy_kernel >= 64) want_cap = std::min<uint32_t>(want_cap, 4 * (c->win_bits / 64) * 64);
    if (want_cap != c->spill_cap) {
        if (c->spill) dev_free(c->spill);
        c->spill = nullptr;
        c->spill_cap = 0;
        if (c->gexec) {   // a captured batch refers to the old lists
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        c->g_seen = false;
        if (want_cap) {
            const uint64_t blocks = std::min<uint32_t>(c->grid, (uint32_t)idx->sm_count);
            FCLSH_CUDA(dev_alloc((void **)&c->spill, blocks * want_cap * 4));
            c->spill_cap = want_cap;
        }
    }
    return FCLSH_OK;
}

static fclsh_status ctx_reserve(fclsh_qctx *c, uint64_t nq, uint64_t cap)
{
    if (nq > c->nq_cap) {
        void *ps[] = {c->res_cnt, c->res_offs, c->coll, c->cand, c->scan_part, c->run_base, c->heavy_q};
        for (void *p : ps)
            if (p) dev_free(p);
        c->heavy_q = nullptr;
        c->res_cnt = nullptr;
        c->res_offs = nullptr;
        c->coll = c->cand = nullptr;
        c->scan_part = nullptr;
        c->run_base = nullptr;
        c->nq_cap = 0;   // a failed allocation below leaves no capacity that looks usable
        const uint64_t m = std::max<uint64_t>(nq, 1024);
        FCLSH_CUDA(dev_alloc((void **)&c->run_base, m * 8));
        FCLSH_CUDA(dev_alloc((void **)&c->res_cnt, m * 4));
        FCLSH_CUDA(dev_alloc((void **)&c->res_offs, (m + 1) * 8));
        FCLSH_CUDA(dev_alloc((void **)&c->coll, m * 8));
        FCLSH_CUDA(dev_alloc((void **)&c->cand, m * 8));
        FCLSH_CUDA(dev_alloc((void **)&c->scan_part, scan_partials_entries(m) * 8));
        FCLSH_CUDA(dev_alloc((void **)&c->heavy_q, m * 8));
        c->nq_cap = m;
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        c->g_seen = false;
    }
    if (cap > c->cap) {
        void *ps[] = {c->runs, c->res_ids};
        for (void *p : ps)
            if (p) dev_free(p);
        c->runs = nullptr;
        c->res_ids = nullptr;
        c->cap = 0;
        FCLSH_CUDA(dev_alloc((void **)&c->runs, cap * 4));
        FCLSH_CUDA(dev_alloc((void **)&c->res_ids, cap * 4));
        c->cap = cap;
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        c->g_seen = false;
    }
    return FCLSH_OK;
}

// Grow the runs to `cap` ids keeping the first c->cap of them (the CSR ids buffer is
// rebuilt by the gather); a captured batch refers to the old buffers and is dropped.
static fclsh_status ctx_grow_runs(fclsh_qctx *c, uint64_t cap, cudaStream_t s)
{
    if (cap <= c->cap) return FCLSH_OK;
    uint32_t *runs = nullptr, *ids = nullptr;
    cudaError_t e = dev_alloc((void **)&runs, cap * 4);
    if (e == cudaSuccess) e = dev_alloc((void **)&ids, cap * 4);
    if (e == cudaSuccess && c->cap) e = cudaMemcpyAsync(runs, c->runs, c->cap * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        dev_free(runs);
        dev_free(ids);
        return cuda_fail(e, "growing the query results");
    }
    dev_free(c->runs);
    dev_free(c->res_ids);
    c->runs = runs;
    c->res_ids = ids;
    c->cap = cap;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    c->g_seen = false;
    return FCLSH_OK;
}

static QueryArgs make_args(fclsh_index *idx)
{
    QueryArgs a{};
    a.points = idx->points;
    a.n = idx->n;
    a.words = idx->words;
    a.t = idx->t;
    a.W = idx->W;
    a.T = idx->T;
    a.slot_bits = idx->slot_bits;
    a.hset_log2 = idx->tune.hash_set_log2;
    a.inline_len = idx->tune.inline_probe;
    a.probe_rows = idx->tune.probe_rows;
    a.rep = idx->rep;
    a.ent_ib = idx->ent_ib;
    a.d = idx->d;
    a.sig = idx->tune.verify_filter ? idx->sig : nullptr;
    a.sig_block = idx->sig_block;
    // long parts: the query's sketch from its set bits (O(nnz)) rather than from every position
    a.s1_scatter = idx->scatter_ok() && idx->positions() / idx->t >= kS1ScatterPositions;
    a.sc_off = idx->sc_off;
    a.sc_col = idx->sc_col;
    a.sc_b = idx->sc_b;
    a.col_off = idx->col_off;
    a.col_coord = idx->col_coord;
    a.col_b = idx->col_b;
    a.offs = idx->offs;
    a.offs_stride = idx->offs_stride();
    a.ent = idx->ent;
    a.idbits = bits_for(idx->n);
    return a;
}

// Enqueue the launches of one batch (no host synchronisation inside).
// redo_cap != 0: the second pass after the runs overflowed a buffer of redo_cap ids (see
// QueryArgs::redo_cap); the cursor keeps the first pass's total.
static fclsh_status enqueue_batch(fclsh_qctx *c, const uint64_t *q, uint64_t nq, uint32_t radius, const uint32_t *radii,
                                  cudaStream_t s, uint64_t redo_cap = 0)
{
    fclsh_index *idx = c->idx;
    QueryArgs a = make_args(idx);
    a.queries = q;
    a.nq = nq;
    a.radius = radius;
    a.radii = radii;
    a.work = c->counters;
    a.cursor = c->counters + 1;
    a.runs = c->runs;
    a.run_base = c->run_base;
    a.cap = c->cap;
    a.res_cnt = c->res_cnt;
    a.coll = c->coll;
    a.cand = c->cand;
    a.bitmaps = c->bitmaps;
    a.bm_words = (idx->n + 31) / 32;
    a.redo_cap = redo_cap;
    if (c->win_bits) {
        a.heavy_q = c->heavy_q;
        a.heavy_n = c->counters + 2;
        a.heavy_work = c->counters + 3;
        a.win_bits = c->win_bits;
        a.spill = c->spill;
        a.spill_cap = c->spill_cap;
        a.heavy_from_bitmap = idx->tune.heavy_kernel == 2;
        if ((uint64_t)idx->T * nq <= c->hkeys_cap) a.hkeys = c->hkeys;
    }
    if (idx->classic_k) {   // S1 of classic LSH: the queries' keys by the classic hash kernel
        const uint32_t L = idx->W - 1;
        for (uint32_t k = 0; k < idx->t; ++k)
            FCLSH_CUDA(launch_hash_part(idx, k, q, nq, c->qkeys + (uint64_t)k * L * nq, nq, s));
        a.qkeys = c->qkeys;
    }
    if (redo_cap) {   // the cursor keeps the first pass's total
        FCLSH_CUDA(cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long), s));
        FCLSH_CUDA(cudaMemsetAsync(c->counters + 2, 0, 2 * sizeof(unsigned long long), s));
    } else {
        FCLSH_CUDA(cudaMemsetAsync(c->counters, 0, 4 * sizeof(unsigned long long), s));
    }
    {
        PhaseTimer pt(idx, 2, s);
        const uint32_t grid = (uint32_t)std::min<uint64_t>(c->grid, std::max<uint64_t>(nq, 1));
        FCLSH_CUDA(launch_query_batch(a, grid, c->block, c->smem, s));
        if (c->win_bits) {   // one block per SM (and no more blocks than there are CTA bitmaps)
            PhaseTimer ph(idx, 8, s);
            FCLSH_CUDA(launch_query_heavy(a, std::min<uint32_t>(c->grid, (uint32_t)idx->sm_count), c->heavy_smem, s));
        }
    }
    {
        PhaseTimer pt(idx, 3, s);
        FCLSH_CUDA(scan_u32_to_u64(c->res_cnt, c->res_offs, nq, c->scan_part, s));
        FCLSH_CUDA(launch_gather_runs(c->runs, c->run_base, c->res_cnt, c->res_offs, nq, c->cap, c->res_ids,
                                      idx->sm_count, s));
    }
    return FCLSH_OK;
}

// A batch runs eagerly the first time its shape (inputs, sizes, stream, tuning) is
// seen; when the same shape comes again it is captured into a CUDA graph, which
// later repeats replay.  One-off batches never pay for a capture.
static fclsh_status run_batch(fclsh_qctx *c, const uint64_t *q, uint64_t nq, uint32_t radius, const uint32_t *radii,
                              cudaStream_t s)
{
    fclsh_index *idx = c->idx;
    const bool graph = idx->tune.use_graph && !idx->timing;
    if (!graph) return enqueue_batch(c, q, nq, radius, radii, s);
    const bool same = c->g_q == q && c->g_nq == nq && c->g_radius == radius && c->g_radii == radii &&
                      c->g_stream == s && c->g_cap == c->cap &&
                      memcmp(&c->g_tune, &idx->tune, sizeof(fclsh_tuning)) == 0;
    if (!same || !c->g_seen) {
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        c->g_q = q;
        c->g_nq = nq;
        c->g_radius = radius;
        c->g_radii = radii;
        c->g_stream = s;
        c->g_cap = c->cap;
        c->g_tune = idx->tune;
        c->g_seen = true;
        return enqueue_batch(c, q, nq, radius, radii, s);
    }
    if (!c->gexec) {
        cudaGraph_t g = nullptr;
        FCLSH_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const uint64_t before = launch_count();
        fclsh_status st = enqueue_batch(c, q, nq, radius, radii, s);
        cudaError_t e = cudaStreamEndCapture(s, &g);
        c->g_kernels = launch_count() - before;   // captured, not run: counted at each replay
        launch_count_adjust(-(int64_t)c->g_kernels);
        if (st != FCLSH_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    }
    FCLSH_CUDA(cudaGraphLaunch(c->gexec, s));
    note_launch(c->g_kernels);
    return FCLSH_OK;
}

// ---------------------------------------------------------------- build

// The tensor-core hash's operands (coordinate lists and G's fp16 chunks), built once.
// s == nullptr (the build, on the legacy stream): stream-ordered, no synchronisation.
// owner: the build's allocation list, which keeps the operands on success and frees
// them if the build fails later (nullptr: the index owns them from here on).
static fclsh_status ensure_mma_operands(fclsh_index *idx, cudaStream_t s, DevAllocs *owner = nullptr)
{
    if (idx->mma_g) return FCLSH_OK;
    if (!idx->mma_k)
        return fail(FCLSH_EINVAL, "the tensor-core hash needs W >= 64 and parts of at most 128 coordinates");
    const uint32_t K = idx->mma_k, t = idx->t;
    std::vector<uint32_t> coord((size_t)t * K, 0xFFFFFFFFu);
    for (uint32_t k = 0; k < t; ++k)
        for (uint32_t i = idx->part_off[k]; i < idx->part_off[k + 1]; ++i)
            coord[(size_t)k * K + (i - idx->part_off[k])] = idx->perm[i];
    const size_t per = hash_mma_operand_entries(K, idx->W);
    DevAllocs tmp(s == nullptr), own(s == nullptr);
    DevAllocs &keep = owner ? *owner : own;
    const uint32_t D = idx->positions();
    std::vector<uint64_t> mb(D + (D + 1) / 2);   // b values, then m (32-bit)
    std::memcpy(mb.data(), idx->b.data(), (size_t)D * 8);
    std::memcpy(reinterpret_cast<uint32_t *>(mb.data() + D), idx->m.data(), (size_t)D * 4);
    uint64_t *dmb = nullptr;
    uint32_t *mc = nullptr;   // the index takes these only once they are complete
    uint16_t *mg = nullptr;
    cudaError_t e;
    if ((e = keep.alloc(&mc, coord.size())) != cudaSuccess || (e = keep.alloc(&mg, per * t)) != cudaSuccess ||
        (e = tmp.alloc(&dmb, mb.size())) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(tensor-core hash operands)");
    const uint64_t *db = dmb;
    const uint32_t *dm = reinterpret_cast<const uint32_t *>(dmb + D);
    FCLSH_CUDA(cudaMemcpyAsync(mc, coord.data(), coord.size() * 4, cudaMemcpyHostToDevice, s));
    FCLSH_CUDA(cudaMemcpyAsync(dmb, mb.data(), mb.size() * 8, cudaMemcpyHostToDevice, s));
    for (uint32_t k = 0; k < t; ++k) {
        const uint32_t lo = idx->part_off[k];
        FCLSH_CUDA(build_mma_operand(dm + lo, db + lo, idx->part_off[k + 1] - lo, K, idx->W, mg + k * per, s));
    }
    if (s) FCLSH_CUDA(cudaStreamSynchronize(s));
    own.release();
    idx->mma_coord = mc;
    idx->mma_g = mg;
    idx->device_bytes += coord.size() * 4 + per * t * 2;
    return FCLSH_OK;
}

// Bit 0 of the index's status word: a kernel's bounded wait ran out (reset on read).
static fclsh_status check_status(fclsh_index *idx, cudaStream_t s)
{
    uint32_t st = 0;
    FCLSH_CUDA(cudaMemcpyAsync(&st, idx->status, 4, cudaMemcpyDeviceToHost, s));
    FCLSH_CUDA(cudaStreamSynchronize(s));
    if (!st) return FCLSH_OK;
    FCLSH_CUDA(cudaMemsetAsync(idx->status, 0, 4, s));
    return fail(FCLSH_ETIMEOUT, "a kernel's wait for its tensor-core or copy completion ran out");
}

// Algorithm 1's shape of an index: t parts or rep copies (from the options, the rule for
// approx_c, or the default of Sec. 4.4) and the covered radius per part r' = floor(r rep / t).
static fclsh_status index_shape(uint64_t n, uint32_t d, uint32_t r, const fclsh_build_opts &o, uint32_t *t_out,
                                uint32_t *rep_out, uint32_t *rp_out)
{
    if (!(o.approx_c >= 0.0)) return fail(FCLSH_EINVAL, "approx_c must be >= 0");
    uint32_t t = o.t, rep = o.replicate ? o.replicate : 1;
    if (o.approx_c > 0.0 && !o.t && !o.replicate) algorithm1_rule(n, r, o.approx_c, &t, &rep);
    if (!t) t = rep > 1 ? 1 : default_parts(r);
    if (rep > 32) return fail(FCLSH_EINVAL, "replicate must be at most 32 (got %u)", rep);
    if (rep > 1 && t > 1) return fail(FCLSH_EINVAL, "replication and partitioning exclude each other (t = %u, replicate = %u)", t, rep);
    if (t > d) return fail(FCLSH_EINVAL, "t = %u parts exceed d = %u", t, d);
    const uint32_t rp = r * rep / t;
    if (rp + 1 > (uint32_t)kMaxLogW)
        return fail(FCLSH_EINVAL, "per-part radius floor(r*replicate/t) = %u exceeds 10", rp);
    *t_out = t;
    *rep_out = rep;
    *rp_out = rp;
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_derive_params(uint64_t n, uint32_t d, uint32_t r, uint64_t seed,
                                            const fclsh_build_opts *opts, uint32_t shape[3], uint32_t *perm,
                                            uint32_t *part_off, uint32_t *m, uint64_t *b)
{
    if (!shape) return fail(FCLSH_EINVAL, "shape is NULL");
    if (n == 0 || n > 0xFFFFFFFFULL - 1) return fail(FCLSH_EINVAL, "n must be in 1..2^32-2 (got %llu)", (unsigned long long)n);
    if (d == 0 || d > kMaxD) return fail(FCLSH_EINVAL, "d must be in 1..%u (got %u)", kMaxD, d);
    fclsh_build_opts o{};
    if (opts) o = *opts;
    if (o.perm || o.part_off || o.m || o.b) return fail(FCLSH_EINVAL, "explicit parameters are not derived");
    uint32_t t = 0, rep = 0, rp = 0;
    const fclsh_status st = index_shape(n, d, r, o, &t, &rep, &rp);
    if (st != FCLSH_OK) return st;
    const uint32_t W = 2u << rp;
    shape[0] = t;
    shape[1] = rep;
    shape[2] = W;
    if (!perm && !part_off && !m && !b) return FCLSH_OK;
    std::vector<uint32_t> vp, vo, vm;
    std::vector<uint64_t> vb;
    if (derive_params(seed, d, t, rep, W, vp, vo, vm, vb) != 0) return fail(FCLSH_EINVAL, "cannot derive parameters");
    if (perm) memcpy(perm, vp.data(), vp.size() * 4);
    if (part_off) memcpy(part_off, vo.data(), vo.size() * 4);
    if (m) memcpy(m, vm.data(), vm.size() * 4);
    if (b) memcpy(b, vb.data(), vb.size() * 8);
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_build(const uint64_t *points, uint64_t n, uint32_t d, uint32_t r, uint64_t seed,
                                    const fclsh_build_opts *opts, fclsh_index **out)
{
    NvtxRange nv("fclsh_build");
    if (!out) return fail(FCLSH_EINVAL, "out is NULL");
    *out = nullptr;
    if (!points) return fail(FCLSH_EINVAL, "points is NULL");
    if (n == 0 || n > 0xFFFFFFFFULL - 1) return fail(FCLSH_EINVAL, "n must be in 1..2^32-2 (got %llu)", (unsigned long long)n);
    if (d == 0 || d > kMaxD) return fail(FCLSH_EINVAL, "d must be in 1..%u (got %u)", kMaxD, d);
    fclsh_build_opts o{};
    if (opts) o = *opts;
    uint32_t t = 0, rep = 0, rp = 0;
    {
        const fclsh_status st = index_shape(n, d, r, o, &t, &rep, &rp);
        if (st != FCLSH_OK) return st;
    }
    // classic bit-sampling LSH (the baseline of Sec. 4.1): the covering index's table count
    // (2^(r+1) - 1 per part, as Sec. 4.1 sets it) unless classic_tables says otherwise, in t
    // chunks of W - 1 tables; k sampled coordinates per table by the rule of Sec. 4.1
    const bool classic = o.classic_k > 0 || o.classic_delta > 0.0;
    uint32_t Wc = 2u << rp, ck = 0;
    if (classic) {
        if (o.perm || o.part_off || o.m || o.b) return fail(FCLSH_EINVAL, "classic LSH draws its own samples");
        if (rep > 1) return fail(FCLSH_EINVAL, "classic LSH takes no replication");
        if (o.hash_tile) return fail(FCLSH_EINVAL, "classic LSH has its own hash kernel (hash_tile must be 0)");
        const uint32_t Tcov = t * (Wc - 1);
        const uint32_t L = o.classic_tables ? o.classic_tables : Tcov;
        if (L != Tcov) {
            if (L > 2047) return fail(FCLSH_EINVAL, "classic_tables above 2,047 must equal the covering table count %u", Tcov);
            t = 1;
            Wc = L + 1;
        }
        ck = o.classic_k ? o.classic_k : classic_rule_k(L, r, d, o.classic_delta);
        if (ck == 0 || ck > 8192)
            return fail(FCLSH_EINVAL, "classic LSH needs 1 <= k <= 8192 (got %u; the rule needs 0 < r < d and 0 < delta < 1)",
                        ck);
    }
    const uint32_t W = Wc;
    const uint32_t D = d * rep;   // positions of the (replicated) vector

    auto idx = new fclsh_index();
    std::unique_ptr<fclsh_index> guard(idx);
    FCLSH_CUDA(cudaGetDevice(&idx->device));
    cudaDeviceProp prop;
    FCLSH_CUDA(cudaGetDeviceProperties(&prop, idx->device));
    idx->sm_count = prop.multiProcessorCount;
    idx->smem_optin = prop.sharedMemPerBlockOptin;
    idx->n = n;
    idx->d = d;
    idx->words = (d + 63) / 64;
    idx->r = r;
    idx->t = t;
    idx->rep = rep;
    idx->rp = rp;
    idx->W = W;
    idx->T = t * (W - 1);
    if (o.hash_tile > 4) return fail(FCLSH_EINVAL, "hash_tile must be 0..4");
    idx->tune = fclsh_tuning{256, 4, 12, 4, 1, o.hash_tile, 0, 0, 1};
    idx->timing = o.timing != 0;
    idx->classic_k = ck;
    idx->classic_delta = o.classic_delta;

    const bool explicit_params = o.perm || o.part_off || o.m || o.b;
    if (classic) {
        classic_params(seed, d, idx->T, ck, idx->cl_samples, idx->cl_seed);
    } else if (explicit_params) {
        if (!(o.perm && o.part_off && o.m && o.b)) return fail(FCLSH_EINVAL, "explicit parameters need all of perm, part_off, m, b");
        idx->perm.assign(o.perm, o.perm + D);
        idx->part_off.assign(o.part_off, o.part_off + t + 1);
        idx->m.assign(o.m, o.m + D);
        idx->b.assign(o.b, o.b + D);
        std::vector<char> seen(d, 0);
        for (uint32_t i = 0; i < D; ++i) {
            if (rep > 1) {
                if (idx->perm[i] != i % d) return fail(FCLSH_EINVAL, "with replication perm[i] must be i mod d");
            } else {
                if (idx->perm[i] >= d || seen[idx->perm[i]]) return fail(FCLSH_EINVAL, "perm is not a permutation of [d]");
                seen[idx->perm[i]] = 1;
            }
            if (idx->m[i] >= W) return fail(FCLSH_EINVAL, "m[%u] = %u is not below W = %u", i, idx->m[i], W);
            if (idx->b[i] >= kP) return fail(FCLSH_EINVAL, "b[%u] is not below P", i);
        }
        if (idx->part_off[0] != 0 || idx->part_off[t] != D) return fail(FCLSH_EINVAL, "part_off must run from 0 to D");
        for (uint32_t k = 0; k < t; ++k)
            if (idx->part_off[k + 1] <= idx->part_off[k]) return fail(FCLSH_EINVAL, "parts must be non-empty and ordered");
    } else if (derive_params(seed, d, t, rep, W, idx->perm, idx->part_off, idx->m, idx->b) != 0) {
        return fail(FCLSH_EINVAL, "cannot derive parameters");
    }
    uint32_t max_dk = 0;
    for (uint32_t k = 0; k < (classic ? 0u : t); ++k) max_dk = std::max(max_dk, idx->part_off[k + 1] - idx->part_off[k]);
    idx->mma_k = classic ? 0 : hash_mma_k(W, max_dk);
    if (o.hash_tile == 2 && !idx->mma_k)
        return fail(FCLSH_EINVAL, "hash_tile 2 (tensor cores) needs W >= 64 and parts of at most 128 coordinates");
    // coordinate lists of the scatter sketch (hash_tile 3)
    std::vector<uint32_t> sc_off, sc_col;
    std::vector<uint64_t> sc_bv;
    if (!classic) coord_lists(d, t, W, idx->perm, idx->part_off, idx->m, idx->b, sc_off, sc_col, sc_bv, &idx->sc_pop);
    const bool scatter_fits = idx->sc_pop <= kScatterMaxPop;
    idx->sc_stage = !classic && scatter_stage_bytes(d, max_dk) <= kScatterStageMaxBytes;
    if (!classic && o.hash_tile < 2 && hash_smem_bytes(W, max_dk, o.hash_tile) > idx->smem_optin) {
        // the part's column lists do not fit in shared memory: sketch by scattering set bits
        if (!scatter_fits)
            return fail(FCLSH_EINVAL,
                        "a part of %u positions with W = %u fits neither the hash kernel's shared memory nor the "
                        "scatter sketch (a column holds %u > %u positions)",
                        max_dk, W, idx->sc_pop, kScatterMaxPop);
        idx->tune.hash_tile = 3;
    }
    if (o.hash_tile == 3 && !scatter_fits)
        return fail(FCLSH_EINVAL, "hash_tile 3 (scatter sketch) needs at most %u positions per column (have %u)",
                    kScatterMaxPop, idx->sc_pop);
    if (o.hash_tile == 4 && max_dk > kDirectMaxPositions)
        return fail(FCLSH_EINVAL, "hash_tile 4 (direct route) needs parts of at most %u positions", kDirectMaxPositions);

    uint32_t sb = o.slot_bits;
    if (!sb) {   // about one slot per point
        sb = 13;
        while (sb < 32 && (1ULL << sb) < n) ++sb;
    }
    if (sb < 13 || sb > 32) return fail(FCLSH_EINVAL, "slot_bits must be in 13..32");
    // an entry holds the key's top 50 - s bits above the id: below s = 18 the id gets 14 + s bits
    if (bits_for(n) > entry_id_bits(sb))
        return fail(FCLSH_EINVAL, "slot_bits %u leaves %u id bits, too few for %llu points", sb, entry_id_bits(sb),
                    (unsigned long long)n);
    idx->slot_bits = sb;
    idx->ent_ib = entry_id_bits(sb);

    // the sketch's column lists (covering LSH), or classic LSH's per-table lists of sampled
    // coordinates and summed seed values, uploaded as one block either way
    std::vector<uint32_t> col_off, coord;
    std::vector<uint64_t> bval;
    if (classic)
        classic_lists(idx->T, ck, idx->cl_samples, idx->cl_seed, col_off, coord, bval);
    else
        column_lists(D, t, W, idx->perm, idx->part_off, idx->m, idx->b, col_off, coord, bval);

    DevAllocs keep(true);   // index memory (released into idx on success); the build runs on the legacy stream
    cudaError_t e;
    if ((e = keep.alloc(&idx->points, n * idx->words)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(points)");
    // the part's column lists in one block (one copy): b values, offsets, coordinates
    std::vector<uint64_t> block(bval.size() + (col_off.size() + coord.size() + 1) / 2, 0);
    std::memcpy(block.data(), bval.data(), bval.size() * 8);
    std::memcpy(reinterpret_cast<uint32_t *>(block.data() + bval.size()), col_off.data(), col_off.size() * 4);
    std::memcpy(reinterpret_cast<uint32_t *>(block.data() + bval.size()) + col_off.size(), coord.data(), coord.size() * 4);
    uint64_t *dblock = nullptr;
    if ((e = keep.alloc(&dblock, block.size())) != cudaSuccess) return cuda_fail(e, "cudaMalloc(column lists)");
    idx->col_b = dblock;
    idx->col_off = reinterpret_cast<uint32_t *>(dblock + bval.size());
    idx->col_coord = idx->col_off + col_off.size();
    if (classic) {   // the same block holds the classic lists
        idx->cl_b = idx->col_b;
        idx->cl_off = idx->col_off;
        idx->cl_coord = idx->col_coord;
    }
    std::vector<uint64_t> sblock;
    if (!classic) {   // b values, then offsets, then columns
        sblock.assign(sc_bv.size() + (sc_off.size() + sc_col.size() + 1) / 2, 0);
        std::memcpy(sblock.data(), sc_bv.data(), sc_bv.size() * 8);
        std::memcpy(reinterpret_cast<uint32_t *>(sblock.data() + sc_bv.size()), sc_off.data(), sc_off.size() * 4);
        std::memcpy(reinterpret_cast<uint32_t *>(sblock.data() + sc_bv.size()) + sc_off.size(), sc_col.data(),
                    sc_col.size() * 4);
        uint64_t *sdev = nullptr;
        if ((e = keep.alloc(&sdev, sblock.size())) != cudaSuccess) return cuda_fail(e, "cudaMalloc(coordinate lists)");
        idx->sc_b = sdev;
        idx->sc_off = reinterpret_cast<uint32_t *>(sdev + sc_bv.size());
        idx->sc_col = idx->sc_off + sc_off.size();
    }
    if ((e = keep.alloc(&idx->offs, (size_t)idx->T * idx->offs_stride())) != cudaSuccess) return cuda_fail(e, "cudaMalloc(directory)");
    if ((e = keep.alloc(&idx->ent, (size_t)idx->T * n)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(entries)");
    idx->device_bytes = n * idx->words * 8 + col_off.size() * 4 + coord.size() * 12 + sblock.size() * 8 +
                        (uint64_t)idx->T * idx->offs_stride() * 4 + (uint64_t)idx->T * n * 8;

    cudaStream_t s = nullptr;
    FCLSH_CUDA(cudaMemcpyAsync(idx->points, points, n * idx->words * 8, cudaMemcpyDefault, s));
    FCLSH_CUDA(cudaMemcpyAsync(dblock, block.data(), block.size() * 8, cudaMemcpyHostToDevice, s));
    if (idx->sc_b) FCLSH_CUDA(cudaMemcpyAsync(idx->sc_b, sblock.data(), sblock.size() * 8, cudaMemcpyHostToDevice, s));
    if ((e = keep.alloc(&idx->status, 1)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(status)");
    FCLSH_CUDA(cudaMemsetAsync(idx->status, 0, 4, s));
    // block-occupancy signatures of the points (S3's pre-filter; off by default, timed by
    // fclsh_autotune on points that average at most d/8 set bits) and their popcount total
    idx->sig_block = (d + kSigBlocks - 1) / kSigBlocks;
    if ((e = keep.alloc(&idx->sig, 2 * n)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(signatures)");
    idx->device_bytes += n * 16;
    // (the total is read after the build's final synchronisation: no wait here)
    unsigned long long *d_pop = nullptr, pop_total = 0;
    DevAllocs pop_buf(true);
    if ((e = pop_buf.alloc(&d_pop, 1)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(popcount total)");
    FCLSH_CUDA(cudaMemsetAsync(d_pop, 0, 8, s));
    FCLSH_CUDA(launch_point_sig(idx->points, n, idx->words, d, idx->sig_block, idx->sig, d_pop, idx->sm_count, s));
    FCLSH_CUDA(cudaMemcpyAsync(&pop_total, d_pop, 8, cudaMemcpyDeviceToHost, s));
    if (o.hash_tile == 2) {
        fclsh_status st = ensure_mma_operands(idx, s, &keep);
        if (st != FCLSH_OK) return st;
    }

    // Transient buffers: the keys of one part, and radix-sort buffers for a chunk of its tables.
    const uint32_t L = W - 1;
    DevAllocs tmp(true);
    uint64_t *keys = nullptr;
    if ((e = tmp.alloc(&keys, (size_t)L * n)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(build keys)");
    size_t free_b = 0, total_b = 0;
    FCLSH_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const uint64_t budget = o.mem_budget ? o.mem_budget : free_b / 4;
    // radix-sort buffers for a chunk of tables: (key, id) twice, plus histograms
    const bool msd = msd_path_applies(sb, n);
    // per table: the partition pass's packed entries (MSD: compact, or in bins of `cap` per segment)
    // or two (key, id) buffers (LSD), plus histograms
    const uint32_t dbits = msd ? msd_dbits(sb) : 8;
    const uint64_t nd = (uint64_t)1 << dbits;   // segments per table
    const uint32_t cap = msd ? msd_bin_capacity(n, dbits) : 0;
    const uint64_t width = msd ? std::max<uint64_t>(n, nd * cap + msd_bin0_extra(n)) : n;   // packed entries per table
    const uint64_t per_row = (msd ? width * 8 : n * 24) + sort_hist_entries(1, n, dbits) * 4 + (2 * nd + 1) * 4 + 64;
    uint64_t rows = std::max<uint64_t>(1, budget / per_row);
    rows = std::min<uint64_t>(rows, L);
    rows = std::min<uint64_t>(rows, std::max<uint64_t>(1, 0xFFFFFFF0ULL / width));   // 32-bit entry indexes
    SortBuffers sbuf{};
    if ((e = tmp.alloc(&sbuf.keys_a, rows * width)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(sort keys)");
    if (!msd) {   // (key, id) radix buffers of the LSD path
        if ((e = tmp.alloc(&sbuf.keys_b, rows * n)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(sort keys)");
        if ((e = tmp.alloc(&sbuf.ids_a, rows * n)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(sort ids)");
        if ((e = tmp.alloc(&sbuf.ids_b, rows * n)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(sort ids)");
    }
    sbuf.hist_cap = sort_hist_entries((uint32_t)rows, n, dbits);
    sbuf.partials_cap = scan_partials_entries(sbuf.hist_cap);
    if ((e = tmp.alloc(&sbuf.hist, sbuf.hist_cap)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(sort hist)");
    if ((e = tmp.alloc(&sbuf.partials, sbuf.partials_cap)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(sort scan)");
    unsigned long long *big_cnt = nullptr;
    uint32_t *big = nullptr;
    if (msd) {
        if ((e = tmp.alloc(&big_cnt, 1)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(segment list)");
        if ((e = tmp.alloc(&big, rows * nd)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(segment list)");
        if ((e = tmp.alloc(&sbuf.seg_out, rows * (nd + 1))) != cudaSuccess ||
            (e = tmp.alloc(&sbuf.bin_cnt, rows * nd)) != cudaSuccess || (e = tmp.alloc(&sbuf.status, 1)) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc(segment bounds)");
    }
    // Long points with the scatter sketch: their set coordinates are listed once (one pass over
    // the packed words, ~4 B per set bit), and every part's sketch reads the list.
    uint32_t *pidx = nullptr, *plen = nullptr;
    uint64_t *pstart = nullptr;
    if (idx->tune.hash_tile == 3 && idx->words >= kCsrMinWords) {
        const uint64_t cap = n * idx->words * 2;   // room for one set bit in 32
        unsigned long long *cursor = nullptr;
        if ((e = tmp.alloc(&pidx, cap)) != cudaSuccess || (e = tmp.alloc(&pstart, n)) != cudaSuccess ||
            (e = tmp.alloc(&plen, n)) != cudaSuccess || (e = tmp.alloc(&cursor, 1)) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc(set coordinates)");
        FCLSH_CUDA(launch_extract_set_bits(idx->points, n, idx->words, d, cap, pidx, pstart, plen, cursor,
                                           idx->sm_count, s));
        unsigned long long total = 0;
        FCLSH_CUDA(cudaMemcpyAsync(&total, cursor, 8, cudaMemcpyDeviceToHost, s));
        FCLSH_CUDA(cudaStreamSynchronize(s));
        if (total > cap) pidx = nullptr;   // denser than one bit in 32: the sketch reads the packed words
    }
    // The partition path first partitions into fixed-capacity bins (no histogram pass).
    // A row chunk whose bins overflow (skewed keys) is partitioned again the exact way,
    // with a per-tile digit histogram, and the remaining chunks go that way at once.  The
    // first binned chunk is a single table, so that data whose every table overflows (the
    // empty-sum bucket of sparse points) loses one table's partition, not a chunk's.  Its bin
    // fills size the bins of the other tables: where a bin filled past 7/8 of its room, the
    // bins become 5/4 of the fullest (fewer tables per chunk in the same buffer).
    bool use_bins = msd;
    bool bins_tried = false;
    std::vector<uint32_t> fill(msd ? nd : 0);   // the trial table's bin fills
    uint32_t bcap = cap, bx0 = msd ? msd_bin0_extra(n) : 0;   // the bins: bin 0 holds bcap + bx0
    uint64_t brows = rows;                                    // tables per binned chunk

    for (uint32_t k = 0; k < t; ++k) {
        {
            NvtxRange nh("fclsh_build: hash part");
            PhaseTimer pt(idx, 0, s);
            FCLSH_CUDA(launch_hash_part(idx, k, idx->points, n, keys, n, s, pidx, pstart, plen));
        }
        NvtxRange ns("fclsh_build: bucket tables of the part");
        PhaseTimer pt(idx, 1, s);
        for (uint64_t r0 = 0; r0 < L;) {
            const uint32_t nr =
                (uint32_t)std::min<uint64_t>(msd && use_bins ? (bins_tried ? brows : 1) : rows, L - r0);
            const uint64_t grow = (uint64_t)k * L + r0;
            if (msd) {
                bool binned = false;
                const uint32_t ccap = bcap, cx0 = bx0;   // this chunk's bins (the trial may resize later ones)
                if (use_bins) {
                    {
                        PhaseTimer p5(idx, 5, s);
                        FCLSH_CUDA(msd_partition_scatter(keys + r0 * n, nr, n, sb, ccap, cx0, sbuf, s));
                    }
                    uint32_t status = 0;
                    FCLSH_CUDA(cudaMemcpyAsync(&status, sbuf.status, 4, cudaMemcpyDeviceToHost, s));
                    if (!bins_tried) FCLSH_CUDA(cudaMemcpyAsync(fill.data(), sbuf.bin_cnt, nd * 4, cudaMemcpyDeviceToHost, s));
                    FCLSH_CUDA(cudaStreamSynchronize(s));
                    binned = status == 0;
                    use_bins = binned;
                    if (!bins_tried && use_bins) {   // the single-table trial
                        bool tight = false;
                        uint64_t most = 0;
                        for (uint64_t dg = 0; dg < nd; ++dg) {
                            tight = tight || (uint64_t)fill[dg] * 8 > (uint64_t)bin_capacity((uint32_t)dg, bcap, bx0) * 7;
                            if (dg) most = std::max<uint64_t>(most, fill[dg]);
                        }
                        if (tight) {
                            const uint64_t c2 = std::max<uint64_t>(bcap, ((most * 5 / 4 + 64) + 3) & ~3ULL);
                            const uint64_t b0 = ((uint64_t)fill[0] * 5 / 4 + 64 + 3) & ~3ULL;
                            const uint64_t x2 = std::max<uint64_t>(bx0, b0 > c2 ? b0 - c2 : 0);
                            const uint64_t w2 = nd * c2 + x2;
                            const uint64_t r2 = rows * width / w2;   // the same buffer, fewer tables
                            if (r2 >= 1 && c2 < (1ULL << 31) && x2 < (1ULL << 31)) {
                                bcap = (uint32_t)c2;
                                bx0 = (uint32_t)x2;
                                brows = r2;
                            } else {
                                use_bins = false;
                            }
                        }
                    }
                    bins_tried = true;
                }
                if (!binned) {
                    {
                        PhaseTimer p7(idx, 7, s);
                        FCLSH_CUDA(msd_partition_hist(keys + r0 * n, nr, n, sb, sbuf, s));
                    }
                    PhaseTimer p5(idx, 5, s);
                    FCLSH_CUDA(msd_partition_scatter(keys + r0 * n, nr, n, sb, 0, 0, sbuf, s));
                }
                PhaseTimer p6(idx, 6, s);
                FCLSH_CUDA(msd_finish(nr, n, sb, binned ? ccap : 0, binned ? cx0 : 0, sbuf, big_cnt, big, idx->ent + grow * n,
                                      idx->offs + grow * idx->offs_stride(), idx->sm_count, s));
                r0 += nr;
                continue;
            }
            bool in_b = false;
            FCLSH_CUDA(radix_sort_rows(keys + r0 * n, nr, n, sb, sbuf, &in_b, s));
            FCLSH_CUDA(launch_finalize_rows(in_b ? sbuf.keys_b : sbuf.keys_a, in_b ? sbuf.ids_b : sbuf.ids_a, nr, n, sb,
                                            idx->ent + grow * n, idx->offs + grow * idx->offs_stride(), s));
            r0 += nr;
        }
    }
    FCLSH_CUDA(cudaStreamSynchronize(s));
    idx->sparse = (double)pop_total <= (double)n * d / 8.0;
    {
        fclsh_status st = check_status(idx, s);
        if (st != FCLSH_OK) return st;
    }
    resolve_timers(idx);
    keep.release();
    *out = guard.release();
    return FCLSH_OK;
}

extern "C" void fclsh_free(fclsh_index *idx)
{
    if (!idx) return;
    cudaSetDevice(idx->device);
    cudaDeviceSynchronize();
    drop_timers(idx);
    void *ps[] = {idx->points, idx->col_b /* the column-list block */, idx->sc_b /* the coordinate-list block */,
                  idx->offs, idx->ent, idx->mma_coord, idx->mma_g, idx->sig,
                  idx->status};
    for (void *p : ps)
        if (p) dev_free(p);
    delete idx;
}

extern "C" fclsh_status fclsh_get_info(const fclsh_index *idx, fclsh_info *out)
{
    if (!idx || !out) return fail(FCLSH_EINVAL, "NULL argument");
    out->n = idx->n;
    out->d = idx->d;
    out->words = idx->words;
    out->r = idx->r;
    out->t = idx->t;
    out->rp = idx->rp;
    out->W = idx->W;
    out->T = idx->T;
    out->slot_bits = idx->slot_bits;
    out->P = idx->P;
    out->device_bytes = idx->device_bytes;
    out->device = idx->device;
    out->rep = idx->rep;
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_get_classic_params(const fclsh_index *idx, uint32_t *k, uint32_t *samples, uint64_t *b)
{
    if (!idx || !k) return fail(FCLSH_EINVAL, "NULL argument");
    if (!idx->classic_k) return fail(FCLSH_EINVAL, "not a classic LSH index");
    *k = idx->classic_k;
    if (samples) memcpy(samples, idx->cl_samples.data(), idx->cl_samples.size() * 4);
    if (b) memcpy(b, idx->cl_seed.data(), idx->cl_seed.size() * 8);
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_get_params(const fclsh_index *idx, uint32_t *perm, uint32_t *part_off, uint32_t *m,
                                         uint64_t *b)
{
    if (!idx) return fail(FCLSH_EINVAL, "index is NULL");
    if (idx->classic_k) return fail(FCLSH_EINVAL, "a classic LSH index has no covering parameters (fclsh_get_classic_params)");
    const size_t D = idx->positions();
    if (perm) memcpy(perm, idx->perm.data(), D * 4);
    if (part_off) memcpy(part_off, idx->part_off.data(), (idx->t + 1) * 4);
    if (m) memcpy(m, idx->m.data(), D * 4);
    if (b) memcpy(b, idx->b.data(), D * 8);
    return FCLSH_OK;
}

// ---------------------------------------------------------------- hash / bucket / export

extern "C" fclsh_status fclsh_hash(const fclsh_index *cidx, const uint64_t *pts, uint64_t cnt, uint64_t *keys_out,
                                   void *stream)
{
    fclsh_index *idx = const_cast<fclsh_index *>(cidx);
    if (!idx || !keys_out || (!pts && cnt)) return fail(FCLSH_EINVAL, "NULL argument");
    if (cnt == 0) return FCLSH_OK;
    FCLSH_CUDA(cudaSetDevice(idx->device));
    cudaStream_t s = (cudaStream_t)stream;
    DevAllocs tmp;
    const uint64_t *dp = pts;
    uint64_t *dk = keys_out;
    cudaError_t e;
    const bool keys_host = !is_device_ptr(keys_out);
    if (!is_device_ptr(pts)) {
        uint64_t *p = nullptr;
        if ((e = tmp.alloc(&p, cnt * idx->words)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(points)");
        FCLSH_CUDA(cudaMemcpyAsync(p, pts, cnt * idx->words * 8, cudaMemcpyHostToDevice, s));
        dp = p;
    }
    if (keys_host) {
        if ((e = tmp.alloc(&dk, (size_t)idx->T * cnt)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(keys)");
    }
    {
        PhaseTimer pt(idx, 4, s);
        const uint32_t L = idx->W - 1;
        for (uint32_t k = 0; k < idx->t; ++k) FCLSH_CUDA(launch_hash_part(idx, k, dp, cnt, dk + (uint64_t)k * L * cnt, cnt, s));
    }
    if (keys_host) {
        FCLSH_CUDA(cudaMemcpyAsync(keys_out, dk, (size_t)idx->T * cnt * 8, cudaMemcpyDeviceToHost, s));
        FCLSH_CUDA(cudaStreamSynchronize(s));
        resolve_timers(idx);
        return check_status(idx, s);
    } else if (!tmp.ptrs.empty()) {
        FCLSH_CUDA(cudaStreamSynchronize(s));   // temporaries are freed on return
        resolve_timers(idx);
        return check_status(idx, s);
    }
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_bucket(const fclsh_index *idx, uint32_t table, uint64_t key, uint32_t *ids_out,
                                     uint64_t cap, uint64_t *count)
{
    if (!idx || !count || (cap && !ids_out)) return fail(FCLSH_EINVAL, "NULL argument");
    if (table >= idx->T) return fail(FCLSH_EINVAL, "table %u out of range (T = %u)", table, idx->T);
    FCLSH_CUDA(cudaSetDevice(idx->device));
    const uint64_t sl = key & (idx->slots() - 1);
    uint32_t lohi[2];
    FCLSH_CUDA(cudaMemcpy(lohi, idx->offs + (uint64_t)table * idx->offs_stride() + sl, 8, cudaMemcpyDeviceToHost));
    std::vector<uint64_t> ent(lohi[1] - lohi[0]);
    if (!ent.empty())
        FCLSH_CUDA(cudaMemcpy(ent.data(), idx->ent + (uint64_t)table * idx->n + lohi[0], ent.size() * 8,
                              cudaMemcpyDeviceToHost));
    // the bucket: the slot's entries with equal high key bits (their order in the run is unspecified)
    std::vector<uint32_t> ids;
    const uint64_t fp = key >> idx->slot_bits;
    const uint32_t ib = idx->ent_ib;
    const uint64_t idmask = (1ULL << ib) - 1;
    for (uint64_t e : ent)
        if ((e >> ib) == fp && key < kP) ids.push_back((uint32_t)(e & idmask));
    std::sort(ids.begin(), ids.end());
    for (uint64_t i = 0; i < ids.size() && i < cap; ++i) ids_out[i] = ids[i];
    *count = ids.size();
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_export_table(const fclsh_index *idx, uint32_t table, uint64_t *keys_out, uint32_t *ids_out)
{
    if (!idx || !keys_out || !ids_out) return fail(FCLSH_EINVAL, "NULL argument");
    if (table >= idx->T) return fail(FCLSH_EINVAL, "table %u out of range (T = %u)", table, idx->T);
    FCLSH_CUDA(cudaSetDevice(idx->device));
    std::vector<uint32_t> offs(idx->offs_stride());
    std::vector<uint64_t> ent(idx->n);
    FCLSH_CUDA(cudaMemcpy(offs.data(), idx->offs + (uint64_t)table * idx->offs_stride(), offs.size() * 4,
                          cudaMemcpyDeviceToHost));
    FCLSH_CUDA(cudaMemcpy(ent.data(), idx->ent + (uint64_t)table * idx->n, idx->n * 8, cudaMemcpyDeviceToHost));
    const uint32_t ib = idx->ent_ib;
    const uint64_t idmask = (1ULL << ib) - 1;
    for (uint64_t sl = 0; sl < idx->slots(); ++sl)
        for (uint32_t e = offs[sl]; e < offs[sl + 1]; ++e) {
            keys_out[e] = ((ent[e] >> ib) << idx->slot_bits) | sl;
            ids_out[e] = (uint32_t)(ent[e] & idmask);
        }
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_export_keys(const fclsh_index *idx, const uint32_t *ids, uint64_t cnt, uint64_t *keys_out)
{
    if (!idx || (cnt && (!ids || !keys_out))) return fail(FCLSH_EINVAL, "NULL argument");
    if (cnt == 0) return FCLSH_OK;
    if (cnt > 0xFFFFFFFEULL) return fail(FCLSH_EINVAL, "too many ids");
    std::vector<uint32_t> slot(idx->n, 0xFFFFFFFFu);
    for (uint64_t j = 0; j < cnt; ++j) {
        if (ids[j] >= idx->n) return fail(FCLSH_EINVAL, "id %u out of range (n = %llu)", ids[j], (unsigned long long)idx->n);
        if (slot[ids[j]] != 0xFFFFFFFFu) return fail(FCLSH_EINVAL, "id %u given twice", ids[j]);
        slot[ids[j]] = (uint32_t)j;
    }
    FCLSH_CUDA(cudaSetDevice(idx->device));
    DevAllocs tmp;
    uint32_t *dslot = nullptr;
    uint64_t *dkeys = nullptr;
    cudaError_t e;
    if ((e = tmp.alloc(&dslot, idx->n)) != cudaSuccess || (e = tmp.alloc(&dkeys, (size_t)idx->T * cnt)) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(key read-back)");
    cudaStream_t s = nullptr;
    FCLSH_CUDA(cudaMemcpyAsync(dslot, slot.data(), idx->n * 4, cudaMemcpyHostToDevice, s));
    FCLSH_CUDA(cudaMemsetAsync(dkeys, 0xFF, (size_t)idx->T * cnt * 8, s));   // ids a table misses read 2^64 - 1
    FCLSH_CUDA(launch_export_keys(idx->offs, idx->offs_stride(), idx->ent, idx->n, idx->T, idx->slot_bits, idx->ent_ib,
                                  dslot, cnt, dkeys, idx->sm_count, s));
    FCLSH_CUDA(cudaMemcpyAsync(keys_out, dkeys, (size_t)idx->T * cnt * 8, cudaMemcpyDeviceToHost, s));
    FCLSH_CUDA(cudaStreamSynchronize(s));
    return FCLSH_OK;
}

// ---------------------------------------------------------------- contexts

// Device buffers of a context's last batch (valid from fclsh_query_async until the next one;
// the result ids are complete once the counters read back show at most `cap` hits).
void fclsh::qctx_result_ptrs(const fclsh_qctx *c, const uint64_t **offs, const uint32_t **ids,
                             const uint64_t **coll, const uint64_t **cand, const unsigned long long **hits,
                             uint64_t *cap)
{
    *offs = c->res_offs;
    *ids = c->res_ids;
    *coll = (const uint64_t *)c->coll;
    *cand = (const uint64_t *)c->cand;
    *hits = c->counters + 1;
    *cap = c->cap;
}

// Device bytes fclsh_query_async would add to the context for a batch of nq queries.
uint64_t fclsh::qctx_grow_bytes(const fclsh_qctx *c, uint64_t nq)
{
    const fclsh_index *idx = c->idx;
    uint64_t b = 0;
    if (nq > c->nq_cap) b += std::max<uint64_t>(nq, 1024) * (8 + 4 + 8 + 8 + 8 + 8 + 8) + 64;
    if (c->win_bits && (uint64_t)idx->T * nq > c->hkeys_cap) b += (uint64_t)idx->T * nq * 8;
    const uint64_t want = std::min<uint64_t>(nq * 512, 1ULL << 28);
    if (want > c->cap) b += want * 8;
    if (idx->classic_k && (uint64_t)idx->T * nq > c->qkeys_cap) b += (uint64_t)idx->T * nq * 8;
    return b;
}

extern "C" fclsh_status fclsh_qctx_create(fclsh_index *idx, fclsh_qctx **out)
{
    if (!idx || !out) return fail(FCLSH_EINVAL, "NULL argument");
    *out = nullptr;
    FCLSH_CUDA(cudaSetDevice(idx->device));
    fclsh_qctx *c = new fclsh_qctx();
    c->idx = idx;
    fclsh_status st = FCLSH_OK;
    cudaError_t e = dev_alloc((void **)&c->counters, 4 * sizeof(unsigned long long));
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMalloc(counters)");
    if (st == FCLSH_OK && (e = cudaStreamCreate(&c->own)) != cudaSuccess)
        st = cuda_fail(e, "cudaStreamCreate");
    if (st == FCLSH_OK) st = ctx_shape(c);
    if (st == FCLSH_OK) st = ctx_reserve(c, 1024, 1ULL << 22);
    if (st != FCLSH_OK) {
        ctx_free_buffers(c);
        delete c;
        return st;
    }
    *out = c;
    return FCLSH_OK;
}

extern "C" void fclsh_qctx_free(fclsh_qctx *c)
{
    if (!c) return;
    cudaSetDevice(c->idx->device);
    if (c->pending && c->last_stream) cudaStreamSynchronize(c->last_stream);
    cudaDeviceSynchronize();
    ctx_free_buffers(c);
    delete c;
}

static fclsh_status check_radius(const fclsh_index *idx, uint32_t radius)
{
    if (radius > idx->r) return fail(FCLSH_ERADIUS, "radius %u exceeds the build radius %u", radius, idx->r);
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_query_async(fclsh_qctx *c, const uint64_t *queries, uint64_t nq, uint32_t radius,
                                          const uint32_t *radii, void *stream)
{
    NvtxRange nv("fclsh_query_async");
    if (!c || (!queries && nq)) return fail(FCLSH_EINVAL, "NULL argument");
    fclsh_index *idx = c->idx;
    fclsh_status st = check_radius(idx, radius);
    if (st != FCLSH_OK) return st;
    FCLSH_CUDA(cudaSetDevice(idx->device));
    if (nq && !is_device_ptr(queries)) return fail(FCLSH_EINVAL, "fclsh_query_async needs device queries");
    if (radii && !is_device_ptr(radii)) return fail(FCLSH_EINVAL, "fclsh_query_async needs device radii");
    if (nq >= (1ULL << (64 - bits_for(idx->n) - 1))) return fail(FCLSH_EINVAL, "too many queries in one batch");
    if ((st = ctx_shape(c)) != FCLSH_OK) return st;
    // room for 512 hits per query (up to 2^28 ids, 2 GB with the CSR copy): dense workloads
    // average hundreds of neighbours per query, and a batch that passes it runs its
    // overflowed queries a second time
    const uint64_t want = std::max<uint64_t>(c->cap, std::min<uint64_t>(nq * 512, 1ULL << 28));
    if ((st = ctx_reserve(c, nq, want)) != FCLSH_OK) return st;
    if (idx->classic_k && (uint64_t)idx->T * nq > c->qkeys_cap) {
        dev_free(c->qkeys);
        c->qkeys = nullptr;
        c->qkeys_cap = 0;
        FCLSH_CUDA(dev_alloc((void **)&c->qkeys, (size_t)idx->T * nq * 8));
        c->qkeys_cap = (uint64_t)idx->T * nq;
        if (c->gexec) {   // a captured batch refers to the old buffer
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        c->g_seen = false;
    }
    if (c->win_bits && (uint64_t)idx->T * nq > c->hkeys_cap) {   // the heavy kernel's keys of listed queries
        dev_free(c->hkeys);
        c->hkeys = nullptr;
        c->hkeys_cap = 0;
        FCLSH_CUDA(dev_alloc((void **)&c->hkeys, (size_t)idx->T * nq * 8));
        c->hkeys_cap = (uint64_t)idx->T * nq;
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        c->g_seen = false;
    }
    cudaStream_t s = stream ? (cudaStream_t)stream : c->own;
    c->last_q = queries;
    c->last_nq = nq;
    c->last_radius = radius;
    c->last_radii = radii;
    c->last_stream = s;
    c->pending = true;
    if (nq == 0) return FCLSH_OK;
    return run_batch(c, queries, nq, radius, radii, s);
}

extern "C" fclsh_status fclsh_qctx_wait(fclsh_qctx *c, fclsh_device_result *out)
{
    NvtxRange nv("fclsh_qctx_wait");
    if (!c) return fail(FCLSH_EINVAL, "NULL argument");
    fclsh_index *idx = c->idx;
    FCLSH_CUDA(cudaSetDevice(idx->device));
    if (c->pending && c->last_nq) {
        unsigned long long cur = 0;
        FCLSH_CUDA(cudaMemcpyAsync(&cur, c->counters + 1, 8, cudaMemcpyDeviceToHost, c->last_stream));
        FCLSH_CUDA(cudaStreamSynchronize(c->last_stream));
        if (cur > c->cap) {
            // The runs passed the buffer: every query reserved its run all the same (the cursor
            // is the batch's total), so grow the buffer to the total, keep the runs that fitted,
            // and run only the queries whose run passed the old end again, into their places.
            const uint64_t old_cap = c->cap;
            fclsh_status st = ctx_grow_runs(c, cur + 1024, c->last_stream);
            if (st != FCLSH_OK) return st;
            st = enqueue_batch(c, c->last_q, c->last_nq, c->last_radius, c->last_radii, c->last_stream, old_cap);
            if (st != FCLSH_OK) return st;
            FCLSH_CUDA(cudaStreamSynchronize(c->last_stream));
        }
    }
    c->pending = false;
    resolve_timers(idx);
    if (out) {
        out->nq = c->last_nq;
        out->offs = c->res_offs;
        out->ids = c->res_ids;
        out->collisions = (const uint64_t *)c->coll;
        out->candidates = (const uint64_t *)c->cand;
        uint64_t total = 0;
        if (c->last_nq) FCLSH_CUDA(cudaMemcpy(&total, c->res_offs + c->last_nq, 8, cudaMemcpyDeviceToHost));
        out->total = total;
    }
    return FCLSH_OK;
}

static fclsh_result *alloc_result(uint64_t nq, uint64_t total)
{
    fclsh_result *r = (fclsh_result *)calloc(1, sizeof(fclsh_result));
    if (!r) return nullptr;
    r->nq = nq;
    r->offs = (uint64_t *)malloc((nq + 1) * 8);
    r->ids = (uint32_t *)malloc(std::max<uint64_t>(total, 1) * 4);
    r->collisions = (uint64_t *)malloc(std::max<uint64_t>(nq, 1) * 8);
    r->candidates = (uint64_t *)malloc(std::max<uint64_t>(nq, 1) * 8);
    if (!r->offs || !r->ids || !r->collisions || !r->candidates) {
        fclsh_result_free(r);
        return nullptr;
    }
    return r;
}

extern "C" void fclsh_result_free(fclsh_result *r)
{
    if (!r) return;
    free(r->offs);
    free(r->ids);
    free(r->collisions);
    free(r->candidates);
    free(r);
}

extern "C" fclsh_status fclsh_qctx_fetch(fclsh_qctx *c, fclsh_result **out)
{
    if (!c || !out) return fail(FCLSH_EINVAL, "NULL argument");
    *out = nullptr;
    fclsh_device_result dr;
    fclsh_status st = fclsh_qctx_wait(c, &dr);
    if (st != FCLSH_OK) return st;
    fclsh_result *r = alloc_result(dr.nq, dr.total);
    if (!r) return fail(FCLSH_ENOMEM, "host allocation of results failed");
    if (dr.nq) {
        cudaError_t e;
        if ((e = cudaMemcpy(r->offs, dr.offs, (dr.nq + 1) * 8, cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (dr.total && (e = cudaMemcpy(r->ids, dr.ids, dr.total * 4, cudaMemcpyDeviceToHost)) != cudaSuccess) ||
            (e = cudaMemcpy(r->collisions, dr.collisions, dr.nq * 8, cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (e = cudaMemcpy(r->candidates, dr.candidates, dr.nq * 8, cudaMemcpyDeviceToHost)) != cudaSuccess) {
            fclsh_result_free(r);
            return cuda_fail(e, "cudaMemcpy(results)");
        }
    } else {
        r->offs[0] = 0;
    }
    *out = r;
    return FCLSH_OK;
}

// Device copies of host queries / radii owned by the context.
static fclsh_status stage_inputs(fclsh_qctx *c, const uint64_t *queries, uint64_t nq, const uint32_t *radii,
                                 cudaStream_t s, const uint64_t **dq, const uint32_t **dr)
{
    fclsh_index *idx = c->idx;
    *dq = queries;
    *dr = radii;
    if (nq && !is_device_ptr(queries)) {
        if (nq * idx->words > c->qbuf_cap) {
            if (c->qbuf) dev_free(c->qbuf);
            c->qbuf = nullptr;
            c->qbuf_cap = 0;
            FCLSH_CUDA(dev_alloc((void **)&c->qbuf, nq * idx->words * 8));
            c->qbuf_cap = nq * idx->words;
        }
        FCLSH_CUDA(cudaMemcpyAsync(c->qbuf, queries, nq * idx->words * 8, cudaMemcpyHostToDevice, s));
        *dq = c->qbuf;
    }
    if (radii && nq && !is_device_ptr(radii)) {
        for (uint64_t i = 0; i < nq; ++i)
            if (radii[i] > idx->r) return fail(FCLSH_ERADIUS, "radius %u of query %llu exceeds the build radius %u",
                                              radii[i], (unsigned long long)i, idx->r);
        if (nq > c->rbuf_cap) {
            if (c->rbuf) dev_free(c->rbuf);
            c->rbuf = nullptr;
            c->rbuf_cap = 0;
            FCLSH_CUDA(dev_alloc((void **)&c->rbuf, nq * 4));
            c->rbuf_cap = nq;
        }
        FCLSH_CUDA(cudaMemcpyAsync(c->rbuf, radii, nq * 4, cudaMemcpyHostToDevice, s));
        *dr = c->rbuf;
    }
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_query(fclsh_index *idx, const uint64_t *queries, uint64_t nq, uint32_t radius,
                                    const uint32_t *radii, void *stream, fclsh_result **out)
{
    if (!idx || !out || (!queries && nq)) return fail(FCLSH_EINVAL, "NULL argument");
    *out = nullptr;
    fclsh_status st = check_radius(idx, radius);
    if (st != FCLSH_OK) return st;
    fclsh_qctx *c = nullptr;
    if ((st = fclsh_qctx_create(idx, &c)) != FCLSH_OK) return st;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->own;
    const uint64_t *dq;
    const uint32_t *dr;
    st = stage_inputs(c, queries, nq, radii, s, &dq, &dr);
    if (st == FCLSH_OK) st = fclsh_query_async(c, dq, nq, radius, dr, s);
    if (st == FCLSH_OK) st = fclsh_qctx_fetch(c, out);
    fclsh_qctx_free(c);
    return st;
}

// ---------------------------------------------------------------- plain path

extern "C" fclsh_status fclsh_query_plain(fclsh_index *idx, const uint64_t *queries, uint64_t nq, uint32_t radius,
                                          void *stream, fclsh_result **out)
{
    NvtxRange nv("fclsh_query_plain");
    if (!idx || !out || (!queries && nq)) return fail(FCLSH_EINVAL, "NULL argument");
    *out = nullptr;
    fclsh_status st = check_radius(idx, radius);
    if (st != FCLSH_OK) return st;
    FCLSH_CUDA(cudaSetDevice(idx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const bool qdev = nq && is_device_ptr(queries);
    DevAllocs tmp;
    cudaError_t e;
    uint64_t *dq = nullptr, *dkeys = nullptr;
    uint32_t *bitmap = nullptr;
    unsigned long long *cnt = nullptr, *staged = nullptr, *staged_b = nullptr;
    uint32_t *hist = nullptr, *partials = nullptr;
    const uint64_t bm_words = (idx->n + 31) / 32;
    const uint64_t cap = idx->n;   // one query reports at most n ids
    if ((e = tmp.alloc(&dq, idx->words)) != cudaSuccess || (e = tmp.alloc(&dkeys, idx->T)) != cudaSuccess ||
        (e = tmp.alloc(&bitmap, bm_words)) != cudaSuccess || (e = tmp.alloc(&cnt, 3)) != cudaSuccess ||
        (e = tmp.alloc(&staged, cap)) != cudaSuccess || (e = tmp.alloc(&staged_b, cap)) != cudaSuccess ||
        (e = tmp.alloc(&hist, sort_keys_hist_entries(cap))) != cudaSuccess ||
        (e = tmp.alloc(&partials, scan_partials_entries(sort_keys_hist_entries(cap)))) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(plain query scratch)");
    FCLSH_CUDA(cudaMemsetAsync(bitmap, 0, bm_words * 4, s));
    std::vector<uint64_t> offs(1, 0), coll, cand;
    std::vector<uint32_t> ids;
    const uint32_t L = idx->W - 1;
    const uint32_t idbits = bits_for(idx->n);
    for (uint64_t i = 0; i < nq; ++i) {
        const uint64_t *qsrc = queries + i * idx->words;
        FCLSH_CUDA(cudaMemcpyAsync(dq, qsrc, idx->words * 8, qdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        FCLSH_CUDA(cudaMemsetAsync(cnt, 0, 3 * 8, s));
        for (uint32_t k = 0; k < idx->t; ++k) FCLSH_CUDA(launch_hash_part(idx, k, dq, 1, dkeys + (uint64_t)k * L, 1, s));
        QueryArgs a = make_args(idx);
        a.queries = dq;
        a.nq = 1;
        a.radius = radius;
        a.cursor = cnt;
        a.coll = cnt + 1;
        a.cand = cnt + 2;
        a.staged = staged;
        a.cap = cap;
        FCLSH_CUDA(launch_query_plain(a, dkeys, bitmap, s));
        unsigned long long h[3];
        FCLSH_CUDA(cudaMemcpyAsync(h, cnt, 24, cudaMemcpyDeviceToHost, s));
        FCLSH_CUDA(cudaStreamSynchronize(s));
        const uint64_t m = h[0];
        const unsigned long long *sorted = staged;
        if (m > 2048) {
            bool in_b = false;
            FCLSH_CUDA(radix_sort_keys_dev((uint64_t *)staged, (uint64_t *)staged_b, cnt, cap, idbits, hist, partials,
                                           &in_b, s));
            sorted = in_b ? staged_b : staged;
        } else if (m > 1) {
            FCLSH_CUDA(launch_sort_small(staged, cnt, s));
        }
        const size_t at = ids.size();
        ids.resize(at + m);
        if (m) {
            std::vector<unsigned long long> tmpk(m);
            FCLSH_CUDA(cudaMemcpyAsync(tmpk.data(), sorted, m * 8, cudaMemcpyDeviceToHost, s));
            FCLSH_CUDA(cudaStreamSynchronize(s));
            for (uint64_t j = 0; j < m; ++j) ids[at + j] = (uint32_t)tmpk[j];
        }
        offs.push_back(ids.size());
        coll.push_back(h[1]);
        cand.push_back(h[2]);
        // leave the bitmap clear for the next query
        FCLSH_CUDA(cudaMemsetAsync(bitmap, 0, bm_words * 4, s));
    }
    FCLSH_CUDA(cudaStreamSynchronize(s));
    fclsh_result *r = alloc_result(nq, ids.size());
    if (!r) return fail(FCLSH_ENOMEM, "host allocation of results failed");
    memcpy(r->offs, offs.data(), offs.size() * 8);
    if (!ids.empty()) memcpy(r->ids, ids.data(), ids.size() * 4);
    if (nq) {
        memcpy(r->collisions, coll.data(), nq * 8);
        memcpy(r->candidates, cand.data(), nq * 8);
    }
    *out = r;
    return FCLSH_OK;
}

// ---------------------------------------------------------------- brute force

extern "C" fclsh_status fclsh_bruteforce(fclsh_index *idx, const uint64_t *queries, uint64_t nq, uint32_t radius,
                                         void *stream, fclsh_result **out)
{
    if (!idx || !out || (!queries && nq)) return fail(FCLSH_EINVAL, "NULL argument");
    *out = nullptr;
    FCLSH_CUDA(cudaSetDevice(idx->device));
    if (idx->words > 48) return fail(FCLSH_EINVAL, "brute force supports d <= 3072");
    cudaStream_t s = (cudaStream_t)stream;
    DevAllocs tmp;
    cudaError_t e;
    const uint64_t *dq = queries;
    if (nq && !is_device_ptr(queries)) {
        uint64_t *p;
        if ((e = tmp.alloc(&p, nq * idx->words)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(queries)");
        FCLSH_CUDA(cudaMemcpyAsync(p, queries, nq * idx->words * 8, cudaMemcpyHostToDevice, s));
        dq = p;
    }
    const uint32_t idbits = bits_for(idx->n);
    const uint32_t bits = idbits + bits_for(std::max<uint64_t>(nq, 2));
    if (bits > 64) return fail(FCLSH_EINVAL, "too many queries");
    uint64_t cap = std::max<uint64_t>(1ULL << 20, nq * 16);
    for (int attempt = 0; attempt < 6; ++attempt) {
        DevAllocs b;
        unsigned long long *cnt, *sa, *sb;
        uint32_t *res_cnt, *hist, *partials, *ids;
        uint64_t *offs, *sp;
        const size_t h = sort_keys_hist_entries(cap);
        if ((e = b.alloc(&cnt, 1)) != cudaSuccess || (e = b.alloc(&sa, cap)) != cudaSuccess ||
            (e = b.alloc(&sb, cap)) != cudaSuccess || (e = b.alloc(&res_cnt, nq)) != cudaSuccess ||
            (e = b.alloc(&hist, h)) != cudaSuccess || (e = b.alloc(&partials, scan_partials_entries(h))) != cudaSuccess ||
            (e = b.alloc(&ids, cap)) != cudaSuccess || (e = b.alloc(&offs, nq + 1)) != cudaSuccess ||
            (e = b.alloc(&sp, scan_partials_entries(nq))) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc(brute-force scratch)");
        FCLSH_CUDA(cudaMemsetAsync(cnt, 0, 8, s));
        FCLSH_CUDA(cudaMemsetAsync(res_cnt, 0, std::max<uint64_t>(nq, 1) * 4, s));
        FCLSH_CUDA(launch_bruteforce(idx->points, idx->n, idx->words, dq, nq, radius, cnt, sa, cap, idbits, res_cnt,
                                     idx->sm_count, s));
        unsigned long long total = 0;
        FCLSH_CUDA(cudaMemcpyAsync(&total, cnt, 8, cudaMemcpyDeviceToHost, s));
        FCLSH_CUDA(cudaStreamSynchronize(s));
        if (total > cap) {
            cap = total + total / 4;
            continue;
        }
        bool in_b = false;
        FCLSH_CUDA(radix_sort_keys_dev((uint64_t *)sa, (uint64_t *)sb, cnt, cap, bits, hist, partials, &in_b, s));
        FCLSH_CUDA(scan_u32_to_u64(res_cnt, offs, nq, sp, s));
        FCLSH_CUDA(launch_extract_ids(in_b ? sb : sa, cnt, cap, (1ULL << idbits) - 1, ids, idx->sm_count, s));
        fclsh_result *r = alloc_result(nq, total);
        if (!r) return fail(FCLSH_ENOMEM, "host allocation of results failed");
        cudaError_t e2 = cudaMemcpyAsync(r->offs, offs, (nq + 1) * 8, cudaMemcpyDeviceToHost, s);
        if (e2 == cudaSuccess && total) e2 = cudaMemcpyAsync(r->ids, ids, total * 4, cudaMemcpyDeviceToHost, s);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
        if (e2 != cudaSuccess) {
            fclsh_result_free(r);
            return cuda_fail(e2, "cudaMemcpy(brute-force results)");
        }
        for (uint64_t i = 0; i < nq; ++i) r->collisions[i] = r->candidates[i] = 0;
        *out = r;
        return FCLSH_OK;
    }
    return fail(FCLSH_EOVERFLOW, "brute-force result buffer kept overflowing");
}

// ---------------------------------------------------------------- tuning / timing / misc

extern "C" fclsh_status fclsh_get_tuning(const fclsh_index *idx, fclsh_tuning *out)
{
    if (!idx || !out) return fail(FCLSH_EINVAL, "NULL argument");
    *out = idx->tune;
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_set_tuning(fclsh_index *idx, const fclsh_tuning *t)
{
    if (!idx || !t) return fail(FCLSH_EINVAL, "NULL argument");
    if (t->query_block != 128 && t->query_block != 256 && t->query_block != 512)
        return fail(FCLSH_EINVAL, "query_block must be 128, 256 or 512");
    if (t->hash_set_log2 < 10 || t->hash_set_log2 > 13) return fail(FCLSH_EINVAL, "hash_set_log2 must be in 10..13");
    if (t->inline_probe < 1 || t->inline_probe > 32) return fail(FCLSH_EINVAL, "inline_probe must be in 1..32");
    if (t->query_ctas_per_sm < 1 || t->query_ctas_per_sm > 16) return fail(FCLSH_EINVAL, "query_ctas_per_sm must be in 1..16");
    if (t->hash_tile > 4) return fail(FCLSH_EINVAL, "hash_tile must be 0..4");
    if (t->hash_tile == 3 && !idx->scatter_ok())
        return fail(FCLSH_EINVAL, "hash_tile 3 (scatter sketch) needs at most %u positions per column (have %u)",
                    kScatterMaxPop, idx->sc_pop);
    if (t->hash_tile == 2) {
        fclsh_status st = ensure_mma_operands(idx, nullptr);
        if (st != FCLSH_OK) return st;
    }
    if (t->probe_rows > 1) return fail(FCLSH_EINVAL, "probe_rows must be 0 or 1");
    if (t->verify_filter > 1) return fail(FCLSH_EINVAL, "verify_filter must be 0 or 1");
    if (t->heavy_kernel > 2 && t->heavy_kernel < 64) return fail(FCLSH_EINVAL, "heavy_kernel must be 0, 1, 2 or >= 64");
    if (idx->classic_k && (t->hash_tile || t->probe_rows))
        return fail(FCLSH_EINVAL, "a classic LSH index has one hash kernel and no row rule (hash_tile, probe_rows = 0)");
    if (idx->classic_k) {
        idx->tune = *t;
        return FCLSH_OK;
    }
    uint32_t max_dk = 0;
    for (uint32_t k = 0; k < idx->t; ++k) max_dk = std::max(max_dk, idx->part_off[k + 1] - idx->part_off[k]);
    if (t->hash_tile == 4 && max_dk > kDirectMaxPositions)
        return fail(FCLSH_EINVAL, "hash_tile 4 (direct route) needs parts of at most %u positions", kDirectMaxPositions);
    if (t->hash_tile != 2 && hash_smem_bytes(idx->W, max_dk, t->hash_tile) > idx->smem_optin)
        return fail(FCLSH_EINVAL, "the hash tile does not fit in shared memory");
    idx->tune = *t;
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_timing_enable(fclsh_index *idx, int on)
{
    if (!idx) return fail(FCLSH_EINVAL, "NULL argument");
    idx->timing = on != 0;
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_timing_read(fclsh_index *idx, double ms[9], uint64_t counts[9], int reset)
{
    if (!idx) return fail(FCLSH_EINVAL, "NULL argument");
    cudaSetDevice(idx->device);
    resolve_timers(idx);
    for (int i = 0; i < kTimedPhases; ++i) {
        if (ms) ms[i] = idx->ms[i];
        if (counts) counts[i] = idx->cnt[i];
        if (reset) {
            idx->ms[i] = 0;
            idx->cnt[i] = 0;
        }
    }
    return FCLSH_OK;
}

// ---------------------------------------------------------------- sparse input

extern "C" fclsh_status fclsh_pack_sparse(const uint64_t *indptr, const uint32_t *indices, uint64_t n, uint64_t nnz,
                                          uint32_t d, uint64_t *out, void *stream)
{
    if ((n && (!indptr || !out)) || (nnz && !indices)) return fail(FCLSH_EINVAL, "NULL argument");
    if (d == 0 || d > kMaxD) return fail(FCLSH_EINVAL, "d must be in 1..%u (got %u)", kMaxD, d);
    if (n == 0) return FCLSH_OK;
    int dev = 0;
    FCLSH_CUDA(cudaGetDevice(&dev));
    int sms = 0;
    FCLSH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t words = (d + 63) / 64;
    DevAllocs tmp;
    cudaError_t e;
    const uint64_t *dp = indptr;
    const uint32_t *di = indices;
    uint64_t *dout = out;
    uint32_t *bad = nullptr;
    if (!is_device_ptr(indptr)) {
        uint64_t *p = nullptr;
        if ((e = tmp.alloc(&p, n + 1)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(indptr)");
        FCLSH_CUDA(cudaMemcpyAsync(p, indptr, (n + 1) * 8, cudaMemcpyHostToDevice, s));
        dp = p;
    }
    if (nnz && !is_device_ptr(indices)) {
        uint32_t *p = nullptr;
        if ((e = tmp.alloc(&p, nnz)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(indices)");
        FCLSH_CUDA(cudaMemcpyAsync(p, indices, nnz * 4, cudaMemcpyHostToDevice, s));
        di = p;
    }
    const bool out_host = !is_device_ptr(out);
    if (out_host && (e = tmp.alloc(&dout, n * words)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(points)");
    if ((e = tmp.alloc(&bad, 1)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(status)");
    FCLSH_CUDA(cudaMemsetAsync(bad, 0, 4, s));
    FCLSH_CUDA(launch_pack_sparse(dp, di, n, nnz, d, dout, bad, sms, s));
    uint32_t hb = 0;
    FCLSH_CUDA(cudaMemcpyAsync(&hb, bad, 4, cudaMemcpyDeviceToHost, s));
    if (out_host) FCLSH_CUDA(cudaMemcpyAsync(out, dout, n * words * 8, cudaMemcpyDeviceToHost, s));
    FCLSH_CUDA(cudaStreamSynchronize(s));
    if (hb & 1) return fail(FCLSH_EINVAL, "indptr must be non-decreasing and end at most at nnz");
    if (hb & 2) return fail(FCLSH_EINVAL, "a coordinate in indices is not below d = %u", d);
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_build_sparse(const uint64_t *indptr, const uint32_t *indices, uint64_t n, uint64_t nnz,
                                           uint32_t d, uint32_t r, uint64_t seed, const fclsh_build_opts *opts,
                                           fclsh_index **out)
{
    if (!out) return fail(FCLSH_EINVAL, "out is NULL");
    *out = nullptr;
    if (n == 0 || n > 0xFFFFFFFFULL - 1) return fail(FCLSH_EINVAL, "n must be in 1..2^32-2 (got %llu)", (unsigned long long)n);
    if (d == 0 || d > kMaxD) return fail(FCLSH_EINVAL, "d must be in 1..%u (got %u)", kMaxD, d);
    DevAllocs tmp;
    uint64_t *pts = nullptr;
    cudaError_t e;
    if ((e = tmp.alloc(&pts, n * ((d + 63) / 64))) != cudaSuccess) return cuda_fail(e, "cudaMalloc(points)");
    fclsh_status st = fclsh_pack_sparse(indptr, indices, n, nnz, d, pts, nullptr);
    if (st != FCLSH_OK) return st;
    return fclsh_build(pts, n, d, r, seed, opts, out);
}

// ---------------------------------------------------------------- save / load

// File layout (little-endian): the 8-byte magic, a header of u32 fields {d, r, t, rep,
// slot_bits, hash_tile, W, version} and u64 {n, P}, the tuning (7 x u32), the random
// choices perm[D], part_off[t+1], m[D] (u32) and b[D] (u64), the points [n][words]
// (u64), and an FNV-1a 64 checksum of everything before it.  The tables are not
// stored: loading rebuilds them from the points with the stored choices (the same
// keys and buckets), which on the GPU is faster than reading them back.
static const char kMagic[8] = {'F', 'C', 'L', 'S', 'H', 'I', 'X', '1'};
constexpr uint32_t kFileVersion = 1;

struct Fnv64 {
    uint64_t h = 0xcbf29ce484222325ULL;
    void add(const void *p, size_t len)
    {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < len; ++i) h = (h ^ c[i]) * 0x100000001b3ULL;
    }
};

struct FileWriter {
    FILE *f = nullptr;
    Fnv64 sum;
    bool ok = true;
    void put(const void *p, size_t len)
    {
        if (ok && len && fwrite(p, 1, len, f) != len) ok = false;
        sum.add(p, len);
    }
};

struct FileReader {
    FILE *f = nullptr;
    Fnv64 sum;
    bool ok = true;
    void get(void *p, size_t len)
    {
        if (ok && len && fread(p, 1, len, f) != len) ok = false;
        if (ok) sum.add(p, len);
    }
};

extern "C" fclsh_status fclsh_save(const fclsh_index *idx, const char *path)
{
    if (!idx || !path) return fail(FCLSH_EINVAL, "NULL argument");
    if (idx->classic_k) return fail(FCLSH_EINVAL, "a classic LSH index is not saved (rebuild it from its points)");
    FCLSH_CUDA(cudaSetDevice(idx->device));
    FileWriter w;
    w.f = fopen(path, "wb");
    if (!w.f) return fail(FCLSH_EINVAL, "cannot open %s for writing", path);
    const uint32_t hdr[8] = {idx->d, idx->r, idx->t, idx->rep, idx->slot_bits, idx->tune.hash_tile, idx->W,
                             kFileVersion};
    const uint64_t hdr64[2] = {idx->n, idx->P};
    const uint32_t tune[7] = {idx->tune.query_block, idx->tune.query_ctas_per_sm, idx->tune.hash_set_log2,
                              idx->tune.inline_probe, idx->tune.use_graph, idx->tune.hash_tile,
                              idx->tune.probe_rows};
    w.put(kMagic, 8);
    w.put(hdr, sizeof hdr);
    w.put(hdr64, sizeof hdr64);
    w.put(tune, sizeof tune);
    const size_t D = idx->positions();
    w.put(idx->perm.data(), D * 4);
    w.put(idx->part_off.data(), (idx->t + 1) * 4);
    w.put(idx->m.data(), D * 4);
    w.put(idx->b.data(), D * 8);
    // the points, through a host buffer of at most 64 MB
    const uint64_t total = idx->n * idx->words;
    const uint64_t chunk = std::min<uint64_t>(total, 8ULL << 20);
    std::vector<uint64_t> buf(chunk);
    for (uint64_t at = 0; at < total && w.ok; at += chunk) {
        const uint64_t len = std::min<uint64_t>(chunk, total - at);
        cudaError_t e = cudaMemcpy(buf.data(), idx->points + at, len * 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            fclose(w.f);
            return cuda_fail(e, "cudaMemcpy(points)");
        }
        w.put(buf.data(), len * 8);
    }
    const uint64_t sum = w.sum.h;
    if (w.ok && fwrite(&sum, 1, 8, w.f) != 8) w.ok = false;
    if (fclose(w.f) != 0) w.ok = false;
    if (!w.ok) return fail(FCLSH_EINVAL, "writing %s failed", path);
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_load(const char *path, fclsh_index **out)
{
    if (!path || !out) return fail(FCLSH_EINVAL, "NULL argument");
    *out = nullptr;
    FileReader rd;
    rd.f = fopen(path, "rb");
    if (!rd.f) return fail(FCLSH_EINVAL, "cannot open %s", path);
    std::unique_ptr<FILE, int (*)(FILE *)> closer(rd.f, fclose);
    char magic[8];
    uint32_t hdr[8];
    uint64_t hdr64[2];
    uint32_t tune[7];
    rd.get(magic, 8);
    if (!rd.ok || memcmp(magic, kMagic, 8) != 0) return fail(FCLSH_EINVAL, "%s is not an fclsh index file", path);
    rd.get(hdr, sizeof hdr);
    rd.get(hdr64, sizeof hdr64);
    rd.get(tune, sizeof tune);
    if (!rd.ok) return fail(FCLSH_EINVAL, "%s: truncated header", path);
    const uint32_t d = hdr[0], r = hdr[1], t = hdr[2], rep = hdr[3], sb = hdr[4], tile = hdr[5], W = hdr[6];
    const uint64_t n = hdr64[0];
    if (hdr[7] != kFileVersion) return fail(FCLSH_EINVAL, "%s: file version %u, expected %u", path, hdr[7], kFileVersion);
    if (hdr64[1] != kP) return fail(FCLSH_EINVAL, "%s: the prime differs from this library's", path);
    if (d == 0 || d > kMaxD || t == 0 || t > d || rep == 0 || rep > 32 || n == 0 || n > 0xFFFFFFFFULL - 1 ||
        W < 2 || W > (1u << kMaxLogW) || (W & (W - 1)))
        return fail(FCLSH_EINVAL, "%s: header out of range", path);
    const uint64_t words = (d + 63) / 64, D = (uint64_t)d * rep;
    std::vector<uint32_t> perm(D), part_off(t + 1), m(D);
    std::vector<uint64_t> b(D), pts;
    rd.get(perm.data(), D * 4);
    rd.get(part_off.data(), (t + 1) * 4);
    rd.get(m.data(), D * 4);
    rd.get(b.data(), D * 8);
    if (!rd.ok) return fail(FCLSH_EINVAL, "%s: truncated parameters", path);
    try {
        pts.resize(n * words);
    } catch (const std::bad_alloc &) {
        return fail(FCLSH_ENOMEM, "host memory for %llu points", (unsigned long long)n);
    }
    rd.get(pts.data(), pts.size() * 8);
    uint64_t sum = 0;
    const uint64_t want = rd.sum.h;
    if (!rd.ok || fread(&sum, 1, 8, rd.f) != 8) return fail(FCLSH_EINVAL, "%s: truncated", path);
    if (sum != want) return fail(FCLSH_EINVAL, "%s: checksum mismatch (the file is damaged)", path);
    fclsh_build_opts o{};
    o.t = t;
    o.replicate = rep;
    o.slot_bits = sb;
    o.hash_tile = tile;
    o.perm = perm.data();
    o.part_off = part_off.data();
    o.m = m.data();
    o.b = b.data();
    fclsh_index *idx = nullptr;
    fclsh_status st = fclsh_build(pts.data(), n, d, r, 0, &o, &idx);
    if (st != FCLSH_OK) return st;
    if (idx->W != W) {
        fclsh_free(idx);
        return fail(FCLSH_EINVAL, "%s: code length %u does not follow from its header", path, W);
    }
    const fclsh_tuning tu{tune[0], tune[1], tune[2], tune[3], tune[4],
                          tune[5], tune[6], idx->tune.verify_filter, idx->tune.heavy_kernel};
    if ((st = fclsh_set_tuning(idx, &tu)) != FCLSH_OK) {
        fclsh_free(idx);
        return st;
    }
    *out = idx;
    return FCLSH_OK;
}

extern "C" uint64_t fclsh_kernel_launches(void) { return launch_count(); }

static std::atomic<uint32_t> g_withhold{0};

uint32_t fclsh::debug_withhold_loads() { return g_withhold.load(); }

extern "C" fclsh_status fclsh_debug_withhold_hash_loads(int on)
{
    g_withhold.store(on > 0 ? (uint32_t)on : 0u);
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_debug_fail_alloc(int64_t after)
{
    g_fail_alloc.store(after < 0 ? -1 : after);
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_debug_pool_used(uint64_t *bytes)
{
    if (!bytes) return fail(FCLSH_EINVAL, "NULL argument");
    int dev = 0;
    FCLSH_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool = device_pool(dev);
    if (!pool) return fail(FCLSH_ECUDA, "no memory pool on device %d", dev);
    uint64_t used = 0;   // the attribute is a 64-bit unsigned count
    FCLSH_CUDA(cudaDeviceSynchronize());   // stream-ordered frees have completed
    FCLSH_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
    *bytes = (uint64_t)used;
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_debug_check_status(int *checked, uint32_t *first)
{
    if (!checked || !first) return fail(FCLSH_EINVAL, "NULL argument");
#ifdef FCLSH_CHECKED
    *checked = 1;
#else
    *checked = 0;
#endif
    FCLSH_CUDA(cudaDeviceSynchronize());
    const uint32_t v[] = {check_first_query(), check_first_hash(), check_first_sort(), check_first_mma(),
                          check_first_noalloc()};
    *first = 0;
    for (uint32_t x : v)
        if (x && !*first) *first = x;
    return FCLSH_OK;
}

extern "C" const char *fclsh_last_error(void) { return g_err.c_str(); }

extern "C" const char *fclsh_version(void) { return "fclsh-gb300 0.1 (sm_103a)"; }

// ---------------------------------------------------------------- autotuner

static std::string tune_key(const fclsh_index *idx)
{
    char buf[160];
    snprintf(buf, sizeof buf, "n=%llu,d=%u,r=%u,t=%u,rep=%u,W=%u", (unsigned long long)idx->n, idx->d, idx->r, idx->t,
             idx->rep, idx->W);
    return buf;
}

static bool read_field(const std::string &obj, const char *name, uint32_t *v)
{
    const std::string pat = std::string("\"") + name + "\":";
    size_t at = obj.find(pat);
    if (at == std::string::npos) return false;
    *v = (uint32_t)strtoul(obj.c_str() + at + pat.size(), nullptr, 10);
    return true;
}

// The cache is a JSON object: {"<key>": {"query_block": 256, ...}, ...}, one entry per line.
static bool cache_lookup(const char *path, const std::string &key, fclsh_tuning *t)
{
    FILE *f = fopen(path, "r");
    if (!f) return false;
    std::string all;
    char buf[4096];
    size_t got;
    while ((got = fread(buf, 1, sizeof buf, f)) > 0) all.append(buf, got);
    fclose(f);
    const std::string pat = "\"" + key + "\":";
    size_t at = all.find(pat);
    if (at == std::string::npos) return false;
    size_t end = all.find('}', at);
    if (end == std::string::npos) return false;
    const std::string obj = all.substr(at + pat.size(), end - at - pat.size() + 1);
    fclsh_tuning v{};
    if (!read_field(obj, "query_block", &v.query_block) || !read_field(obj, "query_ctas_per_sm", &v.query_ctas_per_sm) ||
        !read_field(obj, "hash_set_log2", &v.hash_set_log2) || !read_field(obj, "inline_probe", &v.inline_probe) ||
        !read_field(obj, "use_graph", &v.use_graph) || !read_field(obj, "hash_tile", &v.hash_tile) ||
        !read_field(obj, "verify_filter", &v.verify_filter))
        return false;
    if (!read_field(obj, "heavy_kernel", &v.heavy_kernel)) v.heavy_kernel = 1;   // entries written before it
    *t = v;
    return true;
}

static void cache_store(const char *path, const std::string &key, const fclsh_tuning &t)
{
    std::vector<std::string> lines;
    if (FILE *f = fopen(path, "r")) {
        char buf[1024];
        while (fgets(buf, sizeof buf, f)) {
            std::string l(buf);
            while (!l.empty() && (l.back() == '\n' || l.back() == ',')) l.pop_back();
            if (l.size() > 2 && l[0] == ' ' && l.find("\"" + key + "\":") == std::string::npos) lines.push_back(l);
        }
        fclose(f);
    }
    char ent[512];
    snprintf(ent, sizeof ent,
             "  \"%s\": {\"query_block\": %u, \"query_ctas_per_sm\": %u, \"hash_set_log2\": %u, \"inline_probe\": %u, "
             "\"use_graph\": %u, \"hash_tile\": %u, \"verify_filter\": %u, \"heavy_kernel\": %u}",
             key.c_str(), t.query_block, t.query_ctas_per_sm, t.hash_set_log2, t.inline_probe, t.use_graph, t.hash_tile,
             t.verify_filter, t.heavy_kernel);
    lines.push_back(ent);
    std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n");
    for (size_t i = 0; i < lines.size(); ++i) fprintf(f, "%s%s\n", lines[i].c_str(), i + 1 < lines.size() ? "," : "");
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), path);
}

extern "C" fclsh_status fclsh_autotune(fclsh_index *idx, const uint64_t *queries, uint64_t nq, uint32_t radius,
                                       const char *cache_path, fclsh_tuning *chosen)
{
    if (!idx || (!queries && nq)) return fail(FCLSH_EINVAL, "NULL argument");
    fclsh_status st = check_radius(idx, radius);
    if (st != FCLSH_OK) return st;
    FCLSH_CUDA(cudaSetDevice(idx->device));
    const std::string key = tune_key(idx);
    fclsh_tuning best{};
    if (cache_path && cache_lookup(cache_path, key, &best) &&
        (best.probe_rows = idx->tune.probe_rows, fclsh_set_tuning(idx, &best) == FCLSH_OK)) {
        if (chosen) *chosen = best;
        return FCLSH_OK;
    }
    const fclsh_tuning saved = idx->tune;
    const bool saved_timing = idx->timing;
    idx->timing = false;
    fclsh_qctx *c = nullptr;
    if ((st = fclsh_qctx_create(idx, &c)) != FCLSH_OK) return st;
    cudaStream_t s = c->own;
    const uint64_t *dq;
    const uint32_t *dr;
    st = stage_inputs(c, queries, nq, nullptr, s, &dq, &dr);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    best = saved;
    // inline_probe only shapes the lane-by-lane walk of queries with 2^32 bucket entries or
    // more, so it keeps its value; the block, blocks per SM and dedup set are timed
    const uint32_t blocks[] = {128, 256, 512};
    const uint32_t hlogs[] = {11, 12, 13};
    const uint32_t inl[] = {saved.inline_probe};
    const uint32_t ctas[] = {1, 2, 4, 8};
    for (uint32_t bk : blocks)
        for (uint32_t hl : hlogs)
            for (uint32_t il : inl)
                for (uint32_t ct : ctas) {
                    if (st != FCLSH_OK) break;
                    fclsh_tuning t{bk, ct, hl, il, 0, saved.hash_tile, saved.probe_rows, saved.verify_filter,
                                   saved.heavy_kernel};
                    if (query_smem_bytes(idx->T, idx->W, idx->words, hl) > idx->smem_optin) continue;
                    int occ = 0;
                    if (query_batch_occupancy(bk, query_smem_bytes(idx->T, idx->W, idx->words, hl), &occ) != cudaSuccess ||
                        occ < (int)ct) {
                        cudaGetLastError();
                        continue;
                    }
                    idx->tune = t;
                    if (fclsh_query_async(c, dq, nq, radius, nullptr, s) != FCLSH_OK ||
                        fclsh_qctx_wait(c, nullptr) != FCLSH_OK)
                        continue;
                    cudaEventRecord(e0, s);
                    for (int rep = 0; rep < 2; ++rep) fclsh_query_async(c, dq, nq, radius, nullptr, s);
                    cudaEventRecord(e1, s);
                    if (fclsh_qctx_wait(c, nullptr) != FCLSH_OK) continue;
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best_ms) {
                        best_ms = ms;
                        best = t;
                    }
                }
    // S3's signature pre-filter, on and off, with the chosen shape (sparse points only: on dense
    // ones the bound never rejects)
    if (st == FCLSH_OK && idx->sparse) {
        float ms_f[2] = {1e30f, 1e30f};
        for (uint32_t vf = 0; vf <= 1; ++vf) {
            fclsh_tuning t = best;
            t.use_graph = 0;
            t.verify_filter = vf;
            idx->tune = t;
            if (fclsh_query_async(c, dq, nq, radius, nullptr, s) != FCLSH_OK || fclsh_qctx_wait(c, nullptr) != FCLSH_OK)
                continue;
            cudaEventRecord(e0, s);
            for (int rep = 0; rep < 2; ++rep) fclsh_query_async(c, dq, nq, radius, nullptr, s);
            cudaEventRecord(e1, s);
            if (fclsh_qctx_wait(c, nullptr) != FCLSH_OK) continue;
            cudaEventElapsedTime(&ms_f[vf], e0, e1);
        }
        if (ms_f[0] < 1e30f || ms_f[1] < 1e30f) best.verify_filter = ms_f[1] <= ms_f[0] ? 1u : 0u;
        idx->tune = best;
    }
    // very heavy queries by the second kernel or by the batch kernel's own sweep
    if (st == FCLSH_OK) {
        float ms_h[3] = {1e30f, 1e30f, 1e30f};
        for (uint32_t hk = 0; hk <= 2; ++hk) {
            fclsh_tuning t = best;
            t.use_graph = 0;
            t.heavy_kernel = hk;
            idx->tune = t;
            if (fclsh_query_async(c, dq, nq, radius, nullptr, s) != FCLSH_OK || fclsh_qctx_wait(c, nullptr) != FCLSH_OK)
                continue;
            cudaEventRecord(e0, s);
            for (int rep = 0; rep < 2; ++rep) fclsh_query_async(c, dq, nq, radius, nullptr, s);
            cudaEventRecord(e1, s);
            if (fclsh_qctx_wait(c, nullptr) != FCLSH_OK) continue;
            cudaEventElapsedTime(&ms_h[hk], e0, e1);
        }
        uint32_t hbest = 1;   // the default unless a measured setting beats it
        for (uint32_t hk = 0; hk <= 2; ++hk)
            if (ms_h[hk] < ms_h[hbest]) hbest = hk;
        if (ms_h[hbest] < 1e30f) best.heavy_kernel = hbest;
        idx->tune = best;
    }
    // the hash kernel: WHT tiles and the tensor-core contraction on the index's first points
    // (about 2 GB of keys: enough blocks that the timing reflects a full build); classic LSH
    // has one hash kernel
    if (st == FCLSH_OK && !idx->classic_k) {
        const uint32_t L = idx->W - 1;
        const uint64_t cnt = std::min<uint64_t>(idx->n, std::max<uint64_t>(4096, (256ULL << 20) / L));
        uint32_t max_dk = 0;
        for (uint32_t k = 0; k < idx->t; ++k) max_dk = std::max(max_dk, idx->part_off[k + 1] - idx->part_off[k]);
        uint64_t *kbuf = nullptr;
        if (dev_alloc((void **)&kbuf, cnt * L * 8) == cudaSuccess) {
            float best_h = 1e30f;
            for (uint32_t tl = 0; tl <= 3; ++tl) {
                if (tl != 2 && hash_smem_bytes(idx->W, max_dk, tl) > idx->smem_optin) continue;
                if (tl == 2 && (!idx->mma_k || ensure_mma_operands(idx, s) != FCLSH_OK)) continue;
                if (tl == 3 && !idx->scatter_ok()) continue;
                idx->tune.hash_tile = tl;
                if (launch_hash_part(idx, 0, idx->points, cnt, kbuf, cnt, s) != cudaSuccess) continue;
                cudaEventRecord(e0, s);
                for (int rep = 0; rep < 3; ++rep) launch_hash_part(idx, 0, idx->points, cnt, kbuf, cnt, s);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) continue;
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best_h) {
                    best_h = ms;
                    best.hash_tile = tl;
                }
            }
            dev_free(kbuf);
        }
        cudaGetLastError();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    fclsh_qctx_free(c);
    idx->timing = saved_timing;
    best.use_graph = 1;
    best.probe_rows = saved.probe_rows;
    idx->tune = best;
    if (st != FCLSH_OK) return st;
    if (cache_path) cache_store(cache_path, key, best);
    if (chosen) *chosen = best;
    return FCLSH_OK;
}
