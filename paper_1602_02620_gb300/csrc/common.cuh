// common.cuh -- shared definitions of libfclsh (internal; not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fclsh.h"

namespace fclsh {

// Checked build (compiled with -DFCLSH_CHECKED; the stand-in for a memory checker): the
// kernels' computed indexes are bounds-checked before the access; a failed check skips the
// access and records its code in the translation unit's device word (the first one wins),
// and fclsh_debug_check_status reads the words.  No trap, no abort: the call completes with
// whatever the skipped accesses leave, and the test harness fails the run.  In a normal
// build every check is the constant true.
#if defined(FCLSH_CHECKED) && defined(__CUDACC__)
static __device__ unsigned int g_check_first;
#define FCLSH_CHECK(cond, code) ((cond) || (atomicCAS(&fclsh::g_check_first, 0u, (unsigned)(code)), false))
#define FCLSH_CHECK_READER(name)                                             \
    uint32_t name()                                                          \
    {                                                                        \
        unsigned int v = 0, z = 0;                                           \
        if (cudaMemcpyFromSymbol(&v, fclsh::g_check_first, 4) != cudaSuccess) v = 0xFFFFFFFFu; \
        cudaMemcpyToSymbol(fclsh::g_check_first, &z, 4);                     \
        return v;                                                            \
    }
#else
#define FCLSH_CHECK(cond, code) true
#define FCLSH_CHECK_READER(name) \
    uint32_t name() { return 0; }
#endif
// first failed check of each kernel file since the last read (0: none)
uint32_t check_first_query();
uint32_t check_first_hash();
uint32_t check_first_sort();
uint32_t check_first_mma();
uint32_t check_first_noalloc();

// The prime of Eq. (1): 2^50 - 27, the largest prime below 2^50.  Sums of up to
// 2^11 residues stay below 2^61, so Algorithm 2 runs exactly in 64-bit integers.
constexpr uint64_t kP = (1ULL << 50) - 27;
constexpr uint64_t kMask50 = (1ULL << 50) - 1;
constexpr int kMaxLogW = 11;          // W = 2^(r'+1) <= 2048
constexpr uint32_t kMaxD = 262144;    // bits per point
constexpr uint32_t kPackedMaxD = 16384;   // coordinates the packed specific-construction gather can name (14 bits)
// The scatter sketch adds b values (< 2^50) of one column into 64 bits without
// reducing: exact while a column of a part holds at most this many positions.
constexpr uint32_t kScatterMaxPop = 16383;
constexpr uint32_t kS1ScatterPositions = 2048;   // parts at least this long: query sketch by scatter
constexpr uint32_t kDirectMaxPositions = 4096;   // longest part of the direct route (hash_tile 4)
constexpr uint32_t kCsrMinWords = 64;            // points of at least this many words: list set bits once per build
constexpr uint32_t kWarpVerifyWords = 32;        // points of at least this many words: one warp per distance
constexpr uint32_t kSigBlocks = 128;             // blocks of a point's S3 signature (16 bytes)
constexpr int kSortTile = 8192;       // radix-sort items per histogram tile (one block)
constexpr int kSortSub = 2048;        // items per scatter sub-tile (256 threads x 8)
constexpr int kSortThreads = 256;

// Row stride (u32 words) of a table's directory offsets: 2^sb + 1 are used; the row
// is padded to a multiple of 4 words so that every row starts 16-byte aligned.
__host__ __device__ __forceinline__ uint64_t dir_stride(uint32_t sb) { return (1ULL << sb) + 4; }

// x mod P for any 64-bit x, by 2^50 == 27 (mod P): x >> 50 < 2^14, so the folded value is
// below 2^50 + 27 * 2^14 < 2P and one conditional subtraction finishes (the scatter sketch's
// unreduced column sums, up to 16,383 (P - 1) < 2^64, rely on the full range).
__host__ __device__ __forceinline__ uint64_t mod_p(uint64_t x)
{
    uint64_t r = (x & kMask50) + (x >> 50) * 27ULL;   // < 2^50 + 27 * 2^14 < 2P
    return r >= kP ? r - kP : r;
}

// (a + b) mod P for a, b < P.
__host__ __device__ __forceinline__ uint64_t add_mod_p(uint64_t a, uint64_t b)
{
    uint64_t s = a + b;
    return s >= kP ? s - kP : s;
}

// Key from the transform output: h_v = ((S - y_v) / 2) mod P, where S = y_0 is
// the sum of the sketch (||q~||_1 reduced) and S - y_v = 2 * sum_{C(v,j)=1} t_j
// is even and in [0, 2^62).  Arithmetic is mod 2^64, which is exact here.
__host__ __device__ __forceinline__ uint64_t finish_key(uint64_t S, uint64_t y)
{
    return mod_p((S - y) >> 1);
}

// Per-part column lists of the sketch (Algorithm 2): column j of part k receives
// the seed-vector entries b_i of the coordinates i with m_k(i) = j.
struct PartCols {
    const uint32_t *col_off;    // [W+1], absolute offsets into coord/bval
    const uint32_t *coord;      // coordinate (bit index into the point)
    const uint64_t *bval;       // b_i in [0, P)
};

// Coordinate lists of one part for the scatter sketch: the positions of the part
// that read coordinate c are entries off[c] .. off[c+1], each with its code column
// col[e] and seed value b[e] (absolute entry indexes).
struct CoordLists {
    const uint32_t *off;        // [d+1]
    const uint32_t *col;
    const uint64_t *b;
    uint32_t d;                 // bits of a point; set bits past d are ignored
    // optional: the points' set coordinates, point i's at pidx[pstart[i] .. pstart[i] + plen[i])
    // (then the sketch reads these instead of the packed words)
    const uint32_t *pidx = nullptr;
    const uint64_t *pstart = nullptr;
    const uint32_t *plen = nullptr;
    // the part's positions are col/b [pos0, pos0 + npos); stage = 1: a hash block first copies
    // the part's lists into shared memory (scatter_stage_bytes)
    uint32_t pos0 = 0, npos = 0, stage = 0;
};

// Shared memory of a part's staged coordinate lists: seed values, columns, offsets.
__host__ __device__ __forceinline__ size_t scatter_stage_bytes(uint32_t d, uint32_t npos)
{
    return (((size_t)npos * 8 + 15) & ~(size_t)15) + (((size_t)npos * 4 + 15) & ~(size_t)15) + ((size_t)d + 1) * 4;
}
constexpr size_t kScatterStageMaxBytes = 32 * 1024;

struct PhaseTimer;

// Everything the query kernels read: the index, one batch, and its outputs.
struct QueryArgs {
    const uint64_t *points;
    uint64_t n;
    uint32_t words, t, W, T, slot_bits, hset_log2, inline_len;
    uint32_t probe_rows;          // 1: probe only the code rows v < 2^(floor(radius*rep/t)+1) of each part
    uint32_t rep;                 // replication factor of Algorithm 1 (1 = none)
    uint32_t d;                   // bits per point
    uint32_t ent_ib;              // id bits of a directory entry: entry = (key >> slot_bits) << ent_ib | id
    // S1 by scattering the query's set bits through the coordinate lists (long parts),
    // else by walking the column lists
    uint32_t s1_scatter;
    const uint32_t *sc_off, *sc_col;
    const uint64_t *sc_b;
    const uint32_t *col_off, *col_coord;
    const uint64_t *col_b;
    const uint32_t *offs;
    uint64_t offs_stride;
    const uint64_t *ent;
    const uint64_t *queries;
    uint64_t nq;
    uint32_t radius;
    const uint32_t *radii;
    unsigned long long *work;     // next query
    unsigned long long *cursor;   // staging fill
    unsigned long long *staged;   // plain path: hits of one query
    uint32_t *runs;               // batched path: each query's sorted hits, one contiguous run per query
    uint64_t *run_base;           // [nq] start of query i's run in `runs`
    uint64_t cap;
    // 0: a query reserves its run with an atomic on *cursor.  Else a second pass after the
    // runs overflowed a buffer of redo_cap ids: only the queries whose run passed redo_cap run
    // again, into the places they reserved (run_base, res_cnt from the first pass).
    uint64_t redo_cap;
    uint32_t idbits;
    uint32_t *res_cnt;
    unsigned long long *coll, *cand;
    uint32_t *bitmaps;            // [gridDim.x][bm_words]
    uint64_t bm_words;
    // S3 pre-filter (nullptr = off): point id's kSigBlocks-bit signature is the 16 bytes
    // sig[2 id], sig[2 id + 1]; bit j is set when the point has a set coordinate in block j =
    // coordinates [j * sig_block, (j + 1) * sig_block).  A candidate whose distance lower bound
    // from the two signatures passes the radius is rejected without reading it.
    const uint64_t *sig;
    uint32_t sig_block;
    // S1 done by a hash launch before the kernel (classic LSH): the queries' keys [T][nq]
    const uint64_t *qkeys;
    // Very heavy queries handed from the batch kernel to query_heavy_kernel (heavy_q nullptr:
    // the batch kernel sweeps them itself): heavy_q[0 .. *heavy_n) lists them, *heavy_work is
    // the heavy kernel's next list position, win_bits the ids of one shared-memory window
    uint64_t *heavy_q;
    unsigned long long *heavy_n, *heavy_work;
    uint32_t win_bits;
    uint32_t *spill;      // [gridDim.x][spill_cap]: the heavy kernel's ids of later windows
    uint32_t spill_cap;
    uint32_t heavy_from_bitmap;   // 1: every query past the shared-memory set goes to the heavy kernel
    uint64_t *hkeys;              // [heavy list position][T]: the listed queries' keys (S1 done once)
};

// A directory entry holds the key's high 50 - s bits above an ent_ib-bit id: 32 id bits
// from s = 18 on, 14 + s below (so that the entry stays within 64 bits).
__host__ __device__ __forceinline__ uint32_t entry_id_bits(uint32_t slot_bits)
{
    return slot_bits >= 18 ? 32u : 14u + slot_bits;
}
__device__ __forceinline__ uint64_t entry_fp(uint64_t en, uint32_t ib) { return en >> ib; }
__device__ __forceinline__ uint32_t entry_id(uint64_t en, uint32_t ib)
{
    return (uint32_t)(en & ((1ULL << ib) - 1));
}

#if defined(__CUDACC__)   // device intrinsics: CUDA translation units only
// Set coordinates of the packed vector x in [lo, hi) (lo < hi).
// Occupancy levels of a query kept for S3's pre-filter (sig_bound).
constexpr int kSigLevels = 8;

__device__ __forceinline__ uint32_t popc_range(const uint64_t *x, uint32_t lo, uint32_t hi)
{
    const uint32_t w0 = lo >> 6, w1 = (hi - 1) >> 6;
    uint32_t c = 0;
    for (uint32_t w = w0; w <= w1; ++w) {
        uint64_t v = x[w];
        if (w == w0) v &= ~0ULL << (lo & 63);
        if (w == w1 && (hi & 63)) v &= (1ULL << (hi & 63)) - 1;
        c += __popcll(v);
    }
    return c;
}

// Lower bound on the Hamming distance of x and q from their block-occupancy signatures
// (.x: blocks 0-63, .y: blocks 64-127): every block where only x has set coordinates differs
// in at least one, and every block where only q has them differs in all of q's there.
// sigm[t] (t = 1..kSigLevels) marks the blocks where q has at least t set coordinates
// (sigm[1] = sq), so the second term is the sum of min(q's count, kSigLevels) over q's blocks
// that x leaves empty: never above the distance.
__device__ __forceinline__ uint32_t sig_bound(ulonglong2 sx, ulonglong2 sq, const ulonglong2 *sigm)
{
    uint32_t lb = __popcll(sx.x & ~sq.x) + __popcll(sx.y & ~sq.y);
    const uint64_t m0 = sq.x & ~sx.x, m1 = sq.y & ~sx.y;
    for (int t = 1; t <= kSigLevels; ++t) {   // the levels are nested: stop at the first empty one
        const ulonglong2 mt = sigm[t];
        if (!(mt.x | mt.y)) break;
        lb += __popcll(m0 & mt.x) + __popcll(m1 & mt.y);
    }
    return lb;
}

// Point id's signature (one 16-byte load).
__device__ __forceinline__ ulonglong2 sig_of(const uint64_t *sig, uint32_t id)
{
    return __ldg(reinterpret_cast<const ulonglong2 *>(sig) + id);
}
#endif

// Code rows a query of this radius probes in every part: all W-1, or with
// probe_rows only v = 1..2^(floor(radius*rep/t)+1)-1 (a point within the radius is
// within floor(radius/t) of the query on some part, Sec. 3.1, or within radius*rep
// of it after replicating both rep times, and Theorem 1 for the map
// m mod 2^(that radius + 1) makes the two collide on one of those rows).
__device__ __forceinline__ uint32_t rows_per_part(const QueryArgs &a, uint32_t radius)
{
    const uint32_t L = a.W - 1;
    if (!a.probe_rows) return L;
    const uint32_t e = radius * a.rep / a.t + 1;
    const uint32_t rows = e >= 31 ? L : (1u << e) - 1u;
    return rows < L ? rows : L;
}

// Table index of the j-th probed table (parts in order, rows 1..nt in each).
__device__ __forceinline__ uint32_t probed_table(uint32_t j, uint32_t nt, uint32_t L)
{
    const uint32_t k = j / nt;
    return k * L + (j - k * nt);
}

}  // namespace fclsh

// Phases timed by fclsh_timing_read (see include/fclsh.h).
constexpr int kTimedPhases = 9;

// The index (opaque to users).
struct fclsh_index {
    int device = 0;
    uint64_t n = 0;
    uint32_t d = 0, words = 0, r = 0, t = 0, rp = 0, W = 0, T = 0, slot_bits = 0;
    uint32_t rep = 1;                // Algorithm 1 replication: positions D = d * rep, position i reads coordinate perm[i]
    uint32_t ent_ib = 32;            // id bits of a directory entry (entry_id_bits(slot_bits))
    uint64_t P = fclsh::kP;
    // host copy of the random choices, one entry per position ([D])
    std::vector<uint32_t> perm, part_off, m;
    std::vector<uint64_t> b;
    // device arrays
    uint64_t *points = nullptr;      // [n][words]
    uint32_t *col_off = nullptr;     // [t][W+1]  (col_b, col_off, col_coord: one allocation, owned via col_b)
    uint32_t *col_coord = nullptr;   // [D]
    uint64_t *col_b = nullptr;       // [D]
    // coordinate lists of the scatter sketch (hash_tile 3): sc_off [t][d+1], sc_col [D],
    // sc_b [D] (one allocation, owned via sc_b); sc_pop = the fullest column of any part
    uint32_t *sc_off = nullptr, *sc_col = nullptr;
    uint64_t *sc_b = nullptr;
    uint32_t sc_pop = 0;
    uint32_t sc_stage = 0;           // 1: a part's coordinate lists fit the hash blocks' shared memory
    uint32_t *offs = nullptr;        // [T][dir_stride(slot_bits)]: 2^slot_bits + 1 used
    uint64_t *ent = nullptr;         // [T][n]: (key >> slot_bits) << 32 | id
    // tensor-core hash (hash_tile 2): padded coordinates per part, their lists [t][mma_k]
    // and G's fp16 chunks [t][...]; built on first use
    uint32_t mma_k = 0;
    uint32_t *mma_coord = nullptr;
    uint16_t *mma_g = nullptr;
    uint32_t *status = nullptr;      // [1] device word: bit 0 = a kernel's bounded wait ran out
    // classic bit-sampling LSH (the baseline of Sec. 4.1) instead of covering LSH when classic_k > 0:
    // T = t (W - 1) tables, table j keyed by Eq. 1 on classic_k sampled coordinates; per table the
    // distinct coordinates and their summed seed values cl_coord / cl_b [cl_off[j] .. cl_off[j+1])
    uint32_t classic_k = 0;
    double classic_delta = 0.0;
    std::vector<uint32_t> cl_samples;   // host [T][classic_k]
    std::vector<uint64_t> cl_seed;      // host [classic_k]
    uint32_t *cl_off = nullptr, *cl_coord = nullptr;   // one allocation, owned via cl_b
    uint64_t *cl_b = nullptr;
    uint64_t *sig = nullptr;         // [n][2] block-occupancy signature of every point (S3 pre-filter)
    uint32_t sig_block = 1;          // coordinates per signature block: ceil(d / kSigBlocks)
    bool sparse = false;             // the points average at most d/8 set bits
    uint64_t device_bytes = 0;
    fclsh_tuning tune{};
    // timing (CUDA events per phase)
    bool timing = false;
    double ms[kTimedPhases] = {0};
    uint64_t cnt[kTimedPhases] = {0};
    int sm_count = 0;
    size_t smem_optin = 0;

    uint32_t positions() const { return d * rep; }
    uint64_t slots() const { return 1ULL << slot_bits; }
    uint64_t offs_stride() const { return fclsh::dir_stride(slot_bits); }
    fclsh::PartCols part(uint32_t k) const
    {
        return fclsh::PartCols{col_off + (size_t)k * (W + 1), col_coord, col_b};
    }
    fclsh::CoordLists coords(uint32_t k) const
    {
        fclsh::CoordLists cl{sc_off + (size_t)k * (d + 1), sc_col, sc_b, d};
        cl.pos0 = part_off[k];
        cl.npos = part_off[k + 1] - part_off[k];
        cl.stage = sc_stage;
        return cl;
    }
    bool scatter_ok() const { return sc_b != nullptr && sc_pop <= fclsh::kScatterMaxPop; }
};

namespace fclsh {

// ---- error reporting and launch accounting (api.cu)
void set_error(const char *fmt, ...);
void note_launch(uint64_t kernels = 1);   // kernels enqueued by this library
uint64_t launch_count();
int64_t launch_count_adjust(int64_t delta);
fclsh_status cuda_fail(cudaError_t e, const char *what);
// Device or managed memory (cudaPointerGetAttributes; allocates nothing).  Host memory,
// registered or not, and unknown pointers are not.
bool is_device_ptr(const void *p);

#define FCLSH_CUDA(call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return fclsh::cuda_fail(e_, #call); \
    } while (0)

// Query contexts (api.cu) as the server drives them: the device buffers of the last batch
// (result offsets, ids, counters, and the hit count whose excess over `cap` means the ids
// are not complete until fclsh_qctx_wait reruns the overflowed queries), and the device
// bytes a batch of nq queries would add to the context.
void qctx_result_ptrs(const fclsh_qctx *c, const uint64_t **offs, const uint32_t **ids, const uint64_t **coll,
                      const uint64_t **cand, const unsigned long long **hits, uint64_t *cap);
uint64_t qctx_grow_bytes(const fclsh_qctx *c, uint64_t nq);
cudaError_t dev_alloc(void **p, size_t bytes);   // the library's device memory pool
void dev_free(void *p);

// Testing aid (api.cu): c + 1 while the tensor-core hash is told to withhold its operand
// copy of chunk c, so that its bounded waits run out (fclsh_debug_withhold_hash_loads); 0 = off.
uint32_t debug_withhold_loads();

// ---- params.cpp
uint32_t default_parts(uint32_t r);
void algorithm1_rule(uint64_t n, uint32_t r, double c, uint32_t *t, uint32_t *rep);
int derive_params(uint64_t seed, uint32_t d, uint32_t t, uint32_t rep, uint32_t W, std::vector<uint32_t> &perm,
                  std::vector<uint32_t> &part_off, std::vector<uint32_t> &m, std::vector<uint64_t> &b);
uint32_t classic_rule_k(uint32_t L, uint32_t r, uint32_t d, double delta);
void classic_params(uint64_t seed, uint32_t d, uint32_t L, uint32_t k, std::vector<uint32_t> &samples,
                    std::vector<uint64_t> &b);
void classic_lists(uint32_t L, uint32_t k, const std::vector<uint32_t> &samples, const std::vector<uint64_t> &b,
                   std::vector<uint32_t> &off, std::vector<uint32_t> &coord, std::vector<uint64_t> &bsum);
void coord_lists(uint32_t d, uint32_t t, uint32_t W, const std::vector<uint32_t> &perm,
                 const std::vector<uint32_t> &part_off, const std::vector<uint32_t> &m,
                 const std::vector<uint64_t> &b, std::vector<uint32_t> &off, std::vector<uint32_t> &col,
                 std::vector<uint64_t> &bval, uint32_t *max_pop);
void column_lists(uint32_t D, uint32_t t, uint32_t W, const std::vector<uint32_t> &perm,
                  const std::vector<uint32_t> &part_off, const std::vector<uint32_t> &m,
                  const std::vector<uint64_t> &b, std::vector<uint32_t> &col_off,
                  std::vector<uint32_t> &coord, std::vector<uint64_t> &bval);

// ---- hash.cu: keys of `cnt` points for part k into keys[(v-1)*ld + i], v = 1..W-1
// (the Walsh-Hadamard kernels for hash_tile 0/1, hash_mma.cu's contraction for 2)
cudaError_t launch_hash_part(const fclsh_index *idx, uint32_t k, const uint64_t *pts, uint64_t cnt,
                             uint64_t *keys, uint64_t ld, cudaStream_t s,
                             const uint32_t *pidx = nullptr, const uint64_t *pstart = nullptr,
                             const uint32_t *plen = nullptr);
// The points' set coordinates in one pass (warp per point): point i's at idx[start[i] ..
// start[i] + len[i]), ascending, places reserved with an atomic on *cursor (which ends at
// the total).  When the total passes cap, nothing past cap is written and the caller
// keeps to the packed words.
cudaError_t launch_extract_set_bits(const uint64_t *pts, uint64_t n, uint32_t words, uint32_t d, uint64_t cap,
                                   uint32_t *idx, uint64_t *start, uint32_t *len, unsigned long long *cursor,
                                   int sm_count, cudaStream_t s);

// ---- hash_mma.cu
uint32_t hash_mma_k(uint32_t W, uint32_t max_dk);   // 0: the contraction does not apply
uint32_t hash_mma_chunks(uint32_t W);
size_t hash_mma_operand_entries(uint32_t K, uint32_t W);
cudaError_t build_mma_operand(const uint32_t *m, const uint64_t *b, uint32_t dk, uint32_t K, uint32_t W,
                              uint16_t *gmat, cudaStream_t s);
cudaError_t launch_hash_mma(const uint32_t *coord, const uint16_t *gmat, uint32_t K, uint32_t W, const uint64_t *pts,
                            uint64_t cnt, uint32_t words, uint64_t *keys, uint64_t ld, uint32_t *status,
                            cudaStream_t s);

// ---- sort.cu
// Sort `rows` segments of `len` (u64 key, u32 id) pairs by key bits [0, bits) (stable,
// LSD, 8-bit digits).  ids_in == nullptr means id = position in the row.  The result
// is in (keys_a, ids_a) or (keys_b, ids_b); *out_in_b tells which.
struct SortBuffers {
    uint64_t *keys_a, *keys_b;
    uint32_t *ids_a, *ids_b;
    uint32_t *hist;          // [rows * 256 * tiles]
    uint32_t *partials;      // scan scratch
    size_t hist_cap, partials_cap;
    // s <= 20 path: segment bounds [rows][257], bin fills [rows][256], and a status word
    uint32_t *seg_out, *bin_cnt, *status;
};
size_t sort_hist_entries(uint32_t rows, uint64_t len, uint32_t dbits = 8);
size_t scan_partials_entries(size_t count);
cudaError_t radix_sort_rows(const uint64_t *keys_in, uint32_t rows, uint64_t len, uint32_t bits,
                            SortBuffers &buf, bool *out_in_b, cudaStream_t s);
// Single segment of u64 keys whose length is *d_count (device), capacity cap.
cudaError_t radix_sort_keys_dev(uint64_t *keys_a, uint64_t *keys_b, const unsigned long long *d_count,
                                uint64_t cap, uint32_t bits, uint32_t *hist, uint32_t *partials,
                                bool *out_in_b, cudaStream_t s);
size_t sort_keys_hist_entries(uint64_t cap);
// Directory of `rows` tables straight from their keys when 11 <= slot_bits <= 23: one
// partition by the top msd_dbits(slot_bits) slot bits (segments of at most 4,096
// slots), then one block per (segment, table) that groups
// the segment by the remaining slot bits in shared memory and writes the directory
// and the entries (the same buckets as radix_sort_rows + finalize).  Exact form:
// msd_partition_hist (histogram + scan into buf.hist, sized sort_hist_entries(rows,
// len, dbits)), msd_partition_scatter with cap = 0.  Histogram-free form: msd_partition_scatter with
// cap = msd_bin_capacity(len, dbits) (or larger) into bins of buf.keys_a (rows * (2^dbits * cap +
// extra0) entries, extra0 = msd_bin0_extra(len) or more: bin_start, bin_capacity); valid
// when *buf.status reads 0 afterwards, else redo the tables the exact way.  Then
// msd_finish with the same cap; it needs big_cnt [1] and big [rows * 2^dbits] of
// scratch for segments longer than 4096, seg_out [rows * (2^dbits + 1)] and bin_cnt
// [rows * 2^dbits].
bool msd_path_applies(uint32_t slot_bits, uint64_t n);
cudaError_t msd_partition_hist(const uint64_t *keys_in, uint32_t rows, uint64_t len, uint32_t sb, SortBuffers &buf,
                               cudaStream_t s);
cudaError_t msd_partition_scatter(const uint64_t *keys_in, uint32_t rows, uint64_t len, uint32_t sb, uint32_t cap,
                                  uint32_t extra0, SortBuffers &buf, cudaStream_t s);
cudaError_t msd_finish(uint32_t rows, uint64_t len, uint32_t sb, uint32_t cap, uint32_t extra0, SortBuffers &buf,
                       unsigned long long *big_cnt, uint32_t *big, uint64_t *ent, uint32_t *offs, int sm_count,
                       cudaStream_t s);
// Partition digit bits for slot_bits (slot_bits - 12: segments of 4,096 slots) and the bin
// capacity of the histogram-free partition for rows of n entries.
uint32_t msd_dbits(uint32_t slot_bits);
uint32_t msd_bin_capacity(uint64_t n, uint32_t dbits);
// Bin 0 of every row holds msd_bin0_extra(n) entries more than the others: key 0, the empty
// sum of a point with no set coordinate on the table's code row (the common bucket of sparse
// points), lies in slot 0, so in segment 0.
uint32_t msd_bin0_extra(uint64_t n);
// Bins of a row: bin d starts at bin_start(d) and holds bin_capacity(d) entries; a row holds
// 2^dbits * cap + extra0.
__host__ __device__ __forceinline__ uint64_t bin_start(uint32_t d, uint32_t cap, uint32_t extra0)
{
    return d ? (uint64_t)d * cap + extra0 : 0;
}
__host__ __device__ __forceinline__ uint32_t bin_capacity(uint32_t d, uint32_t cap, uint32_t extra0)
{
    return d ? cap : cap + extra0;
}
// Directory of each sorted row: ent = (key >> sb) << 32 | id, offs[slot] = first entry of slot.
cudaError_t launch_finalize_rows(const uint64_t *keys, const uint32_t *ids, uint32_t rows, uint64_t len,
                                 uint32_t slot_bits, uint64_t *ent, uint32_t *offs, cudaStream_t s);
// Keys stored in the directory for sampled point ids: keys[tau * cnt + slot_of_id[id]] for every
// entry of every table whose id has slot_of_id[id] != ~0 (read-back for parity checks).
cudaError_t launch_export_keys(const uint32_t *offs, uint64_t offs_stride, const uint64_t *ent, uint64_t n, uint32_t T,
                               uint32_t sb, uint32_t ib, const uint32_t *slot_of_id, uint64_t cnt, uint64_t *keys,
                               int sm_count, cudaStream_t s);
// Block-occupancy signatures of n points, kSigBlocks bits each in sig[2i], sig[2i + 1] (bit j:
// a set coordinate in [j B, (j + 1) B) with B = sig_block), and the total of their popcounts
// added to *pop_total.
cudaError_t launch_point_sig(const uint64_t *pts, uint64_t n, uint32_t words, uint32_t d, uint32_t sig_block,
                             uint64_t *sig, unsigned long long *pop_total, int sm_count, cudaStream_t s);
// Exclusive scan of u32 values into u64 offsets: out[i] = sum_{j<i} in[j], out[count] = total.
cudaError_t scan_u32_to_u64(const uint32_t *in, uint64_t *out, uint64_t count, uint64_t *partials,
                            cudaStream_t s);

}  // namespace fclsh
