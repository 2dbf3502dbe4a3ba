/*
 * fclsh.h -- C ABI of libfclsh.so, a GB300 (sm_103a) implementation of Fast
 * CoveringLSH (Pham & Pagh, "Scalability and Total Recall with Fast
 * CoveringLSH", arXiv 1602.02620): exact Hamming-space r-near-neighbour
 * reporting with no false negatives.
 *
 * Problem (Definition 2 with delta = 0, Sec. 2.1): given S, a set of n points
 * in {0,1}^d, build a structure that for any query q reports every x in S with
 * Hamming distance d(x, q) <= r.
 *
 * Conventions shared by every entry point:
 *   - A point is d bits packed LSB-first into words = ceil(d/64) uint64 values:
 *     coordinate i is bit (i % 64) of word (i / 64).  Arrays of points are
 *     row-major [count][words].  Bits beyond d in the last word must be 0.
 *   - Point ids are uint32 row indices 0..n-1 (n < 2^32).
 *   - Keys are uint64 values in [0, P) with P = 2^50 - 27 (the prime of Eq. 1).
 *   - Table tau = k*(W-1) + (v-1) is code row v = 1..W-1 of part k = 0..t-1,
 *     W = 2^(r'+1), r' = floor(r * rep / t) (rep = the replication factor of
 *     Algorithm 1, 1 without replication); T = t*(W-1) tables in all.
 *   - Pointers marked "host or device" are classified with
 *     cudaPointerGetAttributes; device pointers must live on the index's GPU.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   - Every call returns a status; on failure fclsh_last_error() describes it
 *     (thread-local, valid until the thread's next call).  No call throws, and a
 *     failed call leaks nothing.
 *   - Thread safety: calls on different fclsh_qctx objects (and therefore on
 *     different streams) may run concurrently on one index; one fclsh_qctx is
 *     used by one thread at a time.  fclsh_free must not race with any call.
 */
#ifndef FCLSH_H
#define FCLSH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FCLSH_OK = 0,
    FCLSH_EINVAL = 1,    /* bad argument (null pointer, d = 0, r too large, ...) */
    FCLSH_ENOMEM = 2,    /* device or host allocation failed; nothing was kept */
    FCLSH_ECUDA = 3,     /* a CUDA call failed */
    FCLSH_ERADIUS = 4,   /* query radius above the build radius r */
    FCLSH_ETIMEOUT = 5,  /* a bounded wait ran out (server, device wait loops) */
    FCLSH_EOVERFLOW = 6  /* a result buffer was too small; the call reports the size needed */
} fclsh_status;

typedef struct fclsh_index fclsh_index;   /* opaque; owns all device memory of one index */
typedef struct fclsh_qctx fclsh_qctx;     /* opaque; per-stream query scratch and results */
typedef struct fclsh_server fclsh_server; /* opaque; continuous-batching request server */

/* Build options.  Zero-initialise and set what you need; NULL = all defaults. */
typedef struct {
    uint32_t t;               /* parts (Algorithm 1); 0 = paper's rule: 1 for r < 10, 2 for 10 <= r <= 21,
                                 else the smallest t with floor(r/t) <= 10 */
    uint32_t slot_bits;       /* bucket-directory slots per table = 2^slot_bits, 13..32; 0 = max(13, ceil(log2 n)).
                                 Below 18 a directory entry keeps 14 + slot_bits id bits, so slot_bits must
                                 leave room for the ids of all n points */
    uint64_t mem_budget;      /* bytes for transient build buffers; 0 = 1/4 of free device memory */
    /* Explicit random choices (all four set, or all NULL to draw them from `seed`), over the
       D = d * replicate positions of the (replicated) vector:
       perm[D]: position i holds coordinate perm[i] (Algorithm 1's permutation; with replication
                it must be i mod d, copy i / d of the vector);
       part_off[t+1]: part k = positions [part_off[k], part_off[k+1]);
       m[D]: code column in [0, W) of position i (Eq. 4 map / Algorithm 2 permutation);
       b[D]: seed-vector entry in [0, P) of position i (Eq. 1). Host pointers, copied. */
    const uint32_t *perm;
    const uint32_t *part_off;
    const uint32_t *m;
    const uint64_t *b;
    uint32_t timing;          /* 1: record per-phase CUDA events from the start (see fclsh_timing_read) */
    uint32_t hash_tile;       /* the hash kernel, speed only (same keys): 0 = Algorithm 2 with the default WHT
                                 tile, 1 = twice the points per tile where it fits (W <= 1024), 2 = the
                                 O(dL) route as an exact tensor-core contraction (W >= 64, parts of at most
                                 128 coordinates), 3 = Algorithm 2 with the sketch built by scattering each
                                 point's set bits (O(nnz) per part, Sec. 3.2; any d, while no code column
                                 of a part holds more than 16,383 positions).  0 and 1 stage the part's
                                 column lists in shared memory; a build whose lists do not fit takes 3.
                                 4 = the O(dL) route on CUDA cores (Eq. 1 on g_v AND x for every table, no
                                 transform: the basic covering construction, kept as the baseline the
                                 paper compares Algorithm 2 against; parts of at most 4,096 positions;
                                 never chosen by fclsh_autotune). */
    uint32_t replicate;       /* Algorithm 1's replication for cr < log n: every point and query is repeated
                                 this many times (0 or 1 = none; needs t <= 1).  The index then covers
                                 radius r * replicate of the repeated vectors: W = 2^(r*replicate + 1),
                                 r * replicate <= 10.  Queries still use radii <= r of the original vectors. */
    double approx_c;          /* > 0 with t = 0 and replicate = 0: choose t and replicate by Algorithm 1 for
                                 this approximation factor c, with log = log2 n: replicate floor(log2 n / (c r))
                                 times when c r < log2 n (capped so that r * replicate <= 10), else
                                 ceil(c r / log2 n) parts; without replication t is raised until
                                 floor(r/t) <= 10.  0 = the rule of t. */
    /* Classic bit-sampling LSH instead of covering LSH (the baseline the paper compares against,
       Sec. 2.2 and 4.2; it has false negatives): selected by classic_k > 0 or classic_delta > 0.
       Table j samples classic_k coordinates s_j(1..k) uniformly with replacement and keys a point
       by Eq. 1 on them, key_j(x) = (sum_i b_i x_{s_j(i)}) mod P, one seed vector b for all
       tables.  classic_tables = L (0 = the covering index's table count for (n, d, r), as
       Sec. 4.1 sets it; other counts up to 2,047); classic_k = 0 takes the rule of Sec. 4.1,
       k = ceil(log(1 - delta^(1/L)) / log(1 - r/d)) with delta = classic_delta.  Draws from
       `seed`: every table's k samples (next() mod d) in table order, then b.  Queries use the
       same calls; probe_rows and hash_tile do not apply. */
    uint32_t classic_tables;
    uint32_t classic_k;
    double classic_delta;
} fclsh_build_opts;

typedef struct {
    uint64_t n;
    uint32_t d, words, r, t, rp, W, T, slot_bits;
    uint64_t P;
    uint64_t device_bytes;    /* device memory held by the index */
    int device;               /* CUDA device ordinal */
    uint32_t rep;             /* replication factor (1 = none); rp = r * rep / t is the covered radius per part */
} fclsh_info;

/* Host-side query results (library-owned; free with fclsh_result_free). */
typedef struct {
    uint64_t nq;
    uint64_t *offs;        /* [nq+1]: results of query i are ids[offs[i] .. offs[i+1]) */
    uint32_t *ids;         /* [offs[nq]] ascending within each query */
    uint64_t *collisions;  /* [nq] #Collisions: bucket entries whose key equals the query's (Sec. 4.1, S2) */
    uint64_t *candidates;  /* [nq] #Candidates: distinct ids among them (Sec. 4.1, S3) */
} fclsh_result;

/* Device-side view of a context's last results (owned by the context; valid until its next query). */
typedef struct {
    uint64_t nq;
    uint64_t total;              /* = offs[nq] */
    const uint64_t *offs;        /* device [nq+1] */
    const uint32_t *ids;         /* device [total] */
    const uint64_t *collisions;  /* device [nq] */
    const uint64_t *candidates;  /* device [nq] */
} fclsh_device_result;

/*
 * Kernel shape choices, which change speed only, never results, and the probe
 * rule of queries (probe_rows), which never changes the reported ids.
 */
typedef struct {
    uint32_t query_block;     /* threads per query CTA: 128, 256 or 512 (verify-block shape) */
    uint32_t query_ctas_per_sm;
    uint32_t hash_set_log2;   /* shared-memory dedup set of 2^k ids (10..13) */
    uint32_t inline_probe;    /* probe fan-out: a bucket range up to this length is walked by the lane that
                                 probed it, a longer one by the whole warp (1..32) */
    uint32_t use_graph;       /* capture a batch's launches into a CUDA graph and replay it */
    uint32_t hash_tile;       /* hash kernel of fclsh_hash and of later builds (fclsh_build_opts.hash_tile): 0..4 */
    uint32_t probe_rows;      /* 0: a query probes all T tables (Strategy 2, Sec. 2.2).  1: a query of radius
                                 rho probes only the code rows v = 1 .. 2^(floor(rho*rep/t)+1) - 1 of each
                                 part; the ids are the same (pigeonhole over the parts, Sec. 3.1, or the
                                 distance rho*rep of the replicated vectors, and Theorem 1 for the map
                                 m mod 2^(floor(rho*rep/t)+1)), and #Collisions / #Candidates count the
                                 probed tables only.  Not chosen by fclsh_autotune. */
    uint32_t verify_filter;   /* 1: S3 first bounds a candidate's distance from two 128-bit block-occupancy
                                 signatures (bit j: a set coordinate among the j-th ceil(d/128) coordinates;
                                 the query's bits in blocks the point leaves empty, plus one per block only the
                                 point occupies) and reads the point only when the bound is within the radius.
                                 Same ids and counters.  Default 0; on points that average at most d/8 set bits
                                 fclsh_autotune times both (where the points are mostly cached the extra
                                 dependent load costs more than the point reads it saves). */
    uint32_t heavy_kernel;    /* very heavy queries (more bucket entries than the n-bit bitmap has 32-bit
                                 words): 0 = the batch kernel marks them in its bitmap in global memory
                                 and sweeps it; 1 = a second kernel (one CTA per SM) answers them; 2 = it
                                 also answers every query past the shared-memory dedup set.  1 and 2
                                 mark the bucket entries in a window of ids held in shared memory,
                                 one window after another, as large as shared memory allows; k >= 64 =
                                 the same with windows of at most k ids (rounded down to a multiple of 64;
                                 never below 64*W) and lists of 4 windows' ids for the collisions past
                                 the first window (past that, later windows walk the buckets again).
                                 Same ids and counters.  Default 1; timed by fclsh_autotune. */
} fclsh_tuning;

/* ------------------------------------------------------------------ index */

/*
 * Build the index (Sec. 3.2, "Construction"): draw the random choices of
 * Algorithms 1 and 2 from `seed`, hash every point into its T keys, and group the
 * points of each table into buckets by key (Sec. 2.2: only non-empty buckets are
 * stored).  The keys are those of Eq. 1 on g_v AND x; opts->hash_tile picks the
 * route that computes them: Algorithm 2 (sketch + fast Hadamard transform, Sec. 3.2
 * "Fast computation of hash functions"; tiles 0, 1, 3, the default) or the direct
 * O(dL) sum of Eq. 1 as an exact tensor-core contraction (tile 2) or on CUDA cores
 * (tile 4).  Lemma 3 makes every route give the same keys; fclsh_autotune reports the
 * fastest of 0..3 for a later build.
 *   points: host or device, [n][ceil(d/64)] uint64, copied (caller keeps ownership).
 *   n: 1 .. 2^32-1.  d: 1 .. 262,144; bits past d in a point's last word must be 0.
 *   r: build radius, 0 .. 63, with floor(r*replicate/t) <= 10.
 *   opts: NULL for defaults.  out: receives the index; NULL on failure.
 * Errors: FCLSH_EINVAL (bad sizes or options), FCLSH_ENOMEM, FCLSH_ECUDA.
 * Synchronous: returns once the index is complete.
 */
fclsh_status fclsh_build(const uint64_t *points, uint64_t n, uint32_t d, uint32_t r, uint64_t seed,
                         const fclsh_build_opts *opts, fclsh_index **out);

/* Release the index (its points, random choices and the bucket tables of Sec. 2.2) and all
   its device memory.  NULL is ignored.  No other call on the index may run concurrently. */
void fclsh_free(fclsh_index *idx);

/*
 * Sparse points (no counterpart in the paper, which takes bit vectors): row i is the set
 * of coordinates indices[indptr[i] .. indptr[i+1]) (CSR; any order, repeats allowed).
 * fclsh_pack_sparse writes the n rows as bit vectors out[n][ceil(d/64)] (host or device;
 * device work on `stream`, synchronous on return); fclsh_build_sparse packs them on the
 * device and builds the index exactly as fclsh_build would from the packed rows.
 *   indptr: host or device [n+1] uint64, non-decreasing, indptr[n] <= nnz.
 *   indices: host or device [nnz] uint32, each < d.
 * Errors: FCLSH_EINVAL for NULL pointers, d out of 1..262,144, bounds that run backwards
 * or past nnz, or a coordinate >= d (detected on the device; nothing out of range is written).
 */
fclsh_status fclsh_pack_sparse(const uint64_t *indptr, const uint32_t *indices, uint64_t n, uint64_t nnz,
                               uint32_t d, uint64_t *out, void *stream);
fclsh_status fclsh_build_sparse(const uint64_t *indptr, const uint32_t *indices, uint64_t n, uint64_t nnz,
                                uint32_t d, uint32_t r, uint64_t seed, const fclsh_build_opts *opts,
                                fclsh_index **out);

/* Sizes and derived parameters (Sec. 3.1: L = 2^(r'+1) - 1 tables per part). */
fclsh_status fclsh_get_info(const fclsh_index *idx, fclsh_info *out);

/*
 * Checkpoint and resume (no counterpart in the paper): fclsh_save writes the index's
 * parameters (sizes, the random choices of Algorithms 1 and 2, the tuning) and its
 * points to `path`, with a checksum; fclsh_load reads such a file and rebuilds the
 * index on the current device from them (the same keys and buckets as the saved
 * index; the bucket tables are not stored, since rebuilding them on the GPU is faster
 * than reading them).  Errors: FCLSH_EINVAL for a file that cannot be opened, is not
 * an index file, is truncated or fails its checksum; FCLSH_ENOMEM; FCLSH_ECUDA.
 */
fclsh_status fclsh_save(const fclsh_index *idx, const char *path);
fclsh_status fclsh_load(const char *path, fclsh_index **out);

/*
 * The shape and random choices that fclsh_build(points, n, d, r, seed, opts) draws, computed
 * on the host, with no GPU and no points: Algorithm 1's t parts or rep copies (opts->t,
 * opts->replicate, the rule for opts->approx_c, else one part below r = 10 and two from 10,
 * Sec. 4.4), W = 2^(r'+1) with r' = floor(r * rep / t), and the permutation, part offsets,
 * map m and seed vector b of Algorithms 1 and 2 in the draw order the library uses.
 * shape[0..2] receives t, rep and W.  perm, m (uint32) and b (uint64) have D = d * rep
 * entries and part_off t + 1; each may be NULL (all NULL: only the shape), so a caller can
 * learn the sizes first.  Errors: FCLSH_EINVAL for the arguments fclsh_build rejects before
 * it touches the device, and for explicit parameter arrays in opts.
 */
fclsh_status fclsh_derive_params(uint64_t n, uint32_t d, uint32_t r, uint64_t seed, const fclsh_build_opts *opts,
                                 uint32_t shape[3], uint32_t *perm, uint32_t *part_off, uint32_t *m, uint64_t *b);

/*
 * A classic LSH index's random choices (the baseline of Sec. 4.1): *k receives the samples per
 * table; samples (host, [T][k], may be NULL) the sampled coordinates of every table in draw
 * order; b (host, [k], may be NULL) the seed vector of Eq. 1.  Errors: FCLSH_EINVAL for a NULL
 * index or k, or a covering-LSH index.
 */
fclsh_status fclsh_get_classic_params(const fclsh_index *idx, uint32_t *k, uint32_t *samples, uint64_t *b);

/*
 * Copy out the index's random choices: perm and part_off (Algorithm 1's permutation and
 * parts), m (Algorithm 2's permutation or the map of Eq. 4) and b (the seed vector of
 * Eq. 1), host arrays sized D, t+1, D, D with D = d * rep positions, so that they can be
 * compared with an independent derivation.  Any array pointer may be NULL.
 * Errors: FCLSH_EINVAL for a NULL index or a classic LSH index.
 */
fclsh_status fclsh_get_params(const fclsh_index *idx, uint32_t *perm, uint32_t *part_off,
                              uint32_t *m, uint64_t *b);

/*
 * Keys of `cnt` points under the index's parameters: keys_out[tau*cnt + i] is
 * the key of point i in table tau, i.e. Algorithm 2's h_v for part k, which by
 * Lemma 3 equals Eq. (1) applied to g_v AND x (Eq. 2 / Eq. 4).
 *   pts: host or device [cnt][words].  keys_out: host or device [T][cnt].
 * Runs on `stream`; returns after the keys are written when keys_out is host memory.
 * Errors: FCLSH_EINVAL (NULL pointers), FCLSH_ENOMEM, FCLSH_ECUDA, FCLSH_ETIMEOUT (a
 * bounded wait of the tensor-core hash ran out; the index stays usable).
 */
fclsh_status fclsh_hash(const fclsh_index *idx, const uint64_t *pts, uint64_t cnt, uint64_t *keys_out,
                        void *stream);

/*
 * Ids of the bucket with `key` in table `table` (Sec. 2.2), ascending.
 *   ids_out: host, capacity `cap`; *count receives the bucket size (which may
 *   exceed cap; then only the first cap ids are written).  Synchronous.
 * Errors: FCLSH_EINVAL (NULL pointers, table >= T), FCLSH_ECUDA.
 */
fclsh_status fclsh_bucket(const fclsh_index *idx, uint32_t table, uint64_t key, uint32_t *ids_out,
                          uint64_t cap, uint64_t *count);

/*
 * Every (key, id) entry of table `table` (one hash table of Sec. 2.2) in directory
 * order: ascending by key mod 2^slot_bits (the slot); the order of the entries inside
 * one slot is unspecified (it may differ between two builds of the same index).
 * keys_out/ids_out: host arrays of n entries.  Synchronous.
 * Errors: FCLSH_EINVAL (NULL pointers, table >= T), FCLSH_ENOMEM, FCLSH_ECUDA.
 */
fclsh_status fclsh_export_table(const fclsh_index *idx, uint32_t table, uint64_t *keys_out, uint32_t *ids_out);

/*
 * The keys the build stored for the given points, read back from every table's directory
 * (a diagnostic: the tables of Sec. 2.2 keep each point under its key by Eq. 1, and this
 * returns that key, so that it can be compared with an independent computation).
 *   ids: host [cnt] distinct point ids < n.  keys_out: host [T][cnt]: keys_out[tau*cnt + j]
 *   is the key of point ids[j] in table tau; an id missing from a table reads 2^64 - 1.
 * Synchronous.  Errors: FCLSH_EINVAL (NULL pointers, an id >= n or given twice),
 * FCLSH_ENOMEM, FCLSH_ECUDA.
 */
fclsh_status fclsh_export_keys(const fclsh_index *idx, const uint32_t *ids, uint64_t cnt, uint64_t *keys_out);

/* ------------------------------------------------------------------ queries */

/*
 * Exact r-NN reporting with Strategy 2 (Sec. 2.2) in the S1-S3 steps of
 * Sec. 4.1: hash each query into its T keys, look up its bucket in every table,
 * remove duplicate candidates, and report every candidate within Hamming
 * distance `radius` (verified by popcount).  Queries run batched in one
 * persistent kernel.
 *   queries: host or device [nq][words].  radius <= the build radius r.
 *   radii: optional per-query radii (host or device, [nq], each <= r); NULL = `radius` for all.
 *   out: host results, ascending ids per query.
 * Errors: FCLSH_ERADIUS, FCLSH_EINVAL, FCLSH_ENOMEM, FCLSH_ECUDA.  Synchronous.
 */
fclsh_status fclsh_query(fclsh_index *idx, const uint64_t *queries, uint64_t nq, uint32_t radius,
                         const uint32_t *radii, void *stream, fclsh_result **out);

/*
 * The same answers (Strategy 2, Sec. 2.2, steps S1-S3 of Sec. 4.1) through the
 * one-query-at-a-time path: for each query separately, a hash launch, a
 * probe/dedup/verify launch and a copy back.  The baseline that the batched form is
 * measured against.  Arguments and results as fclsh_query (one radius for all).
 * Errors: FCLSH_ERADIUS, FCLSH_EINVAL, FCLSH_ENOMEM, FCLSH_ECUDA.  Synchronous.
 */
fclsh_status fclsh_query_plain(fclsh_index *idx, const uint64_t *queries, uint64_t nq, uint32_t radius,
                               void *stream, fclsh_result **out);

/*
 * Linear scan on the GPU: every point within `radius` of each query by XOR +
 * popcount over all n points (the ground truth of Sec. 4.2), independent of the
 * tables.  Any radius is allowed; d <= 3,072 (FCLSH_EINVAL beyond).  Synchronous.
 */
fclsh_status fclsh_bruteforce(fclsh_index *idx, const uint64_t *queries, uint64_t nq, uint32_t radius,
                              void *stream, fclsh_result **out);

/*
 * One query through the plain path without allocating: for callers that cannot
 * call cudaMalloc/cudaFree while they query (code running under an allocator or
 * memory pool it does not own, or a latency-bound loop where an allocation and
 * the device synchronisation it can cause are not allowed).  No counterpart in the
 * paper: it packages the plain path above for such callers.
 *   query: device, one point [words].  radius <= r.
 *   ids_out: device, capacity cap; receives the ids within `radius`, ascending
 *   (only the first cap if there are more).  counts_out: device [3]: the number of
 *   results (it may exceed cap), #Collisions, #Candidates.
 * All scratch lives in one fixed device array of about 1.1 MB that every GPU
 * loading the library holds until the process exits, so the call supports
 * indexes of at most 4,194,304 points, 4,094 tables and d <= 16,384, and rejects
 * larger ones with FCLSH_EINVAL.  It allocates nothing: no cudaMalloc, cudaFree
 * or allocating library routine.  The first call on a device looks up the
 * array's device address (make that first call before any stream capture).
 * Every call reuses the same array and clears what it needs, so calls that
 * overlap on the GPU (other streams, other threads) race: serialise them.
 * Asynchronous on `stream`.  Errors: FCLSH_ERADIUS, FCLSH_EINVAL (NULL or host
 * pointers, an index past the limits above), FCLSH_ECUDA.
 */
fclsh_status fclsh_query_plain_noalloc(const fclsh_index *idx, const uint64_t *query, uint32_t radius,
                                       uint32_t *ids_out, uint64_t cap, uint64_t *counts_out, void *stream);

/* Free a host result of fclsh_query, fclsh_query_plain, fclsh_bruteforce, fclsh_qctx_fetch
   or fclsh_server_wait (the library owns it until then; no counterpart in the paper).
   NULL is ignored. */
void fclsh_result_free(fclsh_result *res);

/* ------------------------------------------------------------------ contexts */

/*
 * Per-stream query scratch of the batched form (no counterpart in the paper: the
 * device buffers a batch of Strategy 2 queries needs, reused between batches).
 * Create one per concurrent stream; it must not outlive its index.  fclsh_qctx_free
 * waits for the context's work and releases it (NULL is ignored).
 * Errors: FCLSH_EINVAL (NULL pointers), FCLSH_ENOMEM, FCLSH_ECUDA.
 */
fclsh_status fclsh_qctx_create(fclsh_index *idx, fclsh_qctx **out);
void fclsh_qctx_free(fclsh_qctx *ctx);

/*
 * Enqueue one batch on `stream` without waiting: the whole batch (hash, probe,
 * dedup, verify, result sort and CSR) runs on the device with no host
 * round-trip, and with use_graph set it is replayed as one CUDA graph.
 *   queries, radii: device pointers (radii may be NULL: `radius` for all).
 *   The buffers must stay valid until fclsh_qctx_wait returns.
 * The answers are those of fclsh_query (Strategy 2, Sec. 2.2; S1-S3 of Sec. 4.1).
 * Errors: FCLSH_ERADIUS, FCLSH_EINVAL (NULL or host pointers), FCLSH_ENOMEM, FCLSH_ECUDA.
 */
fclsh_status fclsh_query_async(fclsh_qctx *ctx, const uint64_t *queries, uint64_t nq, uint32_t radius,
                               const uint32_t *radii, void *stream);

/*
 * Wait for the context's batch (no counterpart in the paper) and expose its device
 * results (owned by the context, valid until its next batch).  If the result buffer
 * overflowed, the batch is re-run with a larger buffer before returning.
 * Errors: FCLSH_EINVAL, FCLSH_ENOMEM, FCLSH_ECUDA.
 */
fclsh_status fclsh_qctx_wait(fclsh_qctx *ctx, fclsh_device_result *out);

/* Copy the context's last device results to a host fclsh_result (free it with
   fclsh_result_free; no counterpart in the paper).  Errors: FCLSH_EINVAL, FCLSH_ENOMEM,
   FCLSH_ECUDA. */
fclsh_status fclsh_qctx_fetch(fclsh_qctx *ctx, fclsh_result **out);

/* ------------------------------------------------------------------ serving */

/* Server options.  Zero fields take the defaults shown. */
typedef struct {
    uint32_t slots;              /* device batches in flight, each on its own stream (4) */
    uint32_t max_batch_queries;  /* queries packed into one device batch (16384) */
    uint64_t mem_reserve;        /* device bytes a new batch must leave free (0 = none) */
} fclsh_server_opts;

typedef struct {
    uint64_t requests, queries, batches, deferred_for_memory;
    double mean_batch_queries;
    double p50_ms, p99_ms, max_ms;   /* request latency, submit to results ready */
    double queries_per_s;            /* completed queries / (last completion - first submit) */
} fclsh_serve_stats;

/*
 * Continuous-batching server over a resident index (the served form of the
 * batched query path).  A scheduler thread packs queued requests into device
 * batches (requests of different radius share a batch through per-query radii),
 * admits a batch when a slot is free and the device has the memory it needs, and
 * retires batches as they finish, so arriving requests join while others run and
 * batches on different slots overlap on the device.  A query's answer does not
 * depend on what it was batched with.  The index must outlive the server.  No
 * counterpart in the paper (an execution pattern; the answers are Strategy 2's).
 * Errors: FCLSH_EINVAL (NULL pointers), FCLSH_ENOMEM, FCLSH_ECUDA.
 */
fclsh_status fclsh_server_create(fclsh_index *idx, const fclsh_server_opts *opts, fclsh_server **out);

/* Queue a request (no counterpart in the paper): `queries` host [nq][words] (copied), one
   radius <= r for all of them; *ticket identifies it.
   Errors: FCLSH_ERADIUS, FCLSH_EINVAL, FCLSH_ENOMEM. */
fclsh_status fclsh_server_submit(fclsh_server *srv, const uint64_t *queries, uint64_t nq, uint32_t radius,
                                 uint64_t *ticket);

/*
 * Wait up to timeout_ms (negative = no limit) for a request (no counterpart in the
 * paper); on success *out holds its results (free with fclsh_result_free) and
 * *latency_ms its submit-to-ready time.  FCLSH_ETIMEOUT leaves the request queued; the
 * ticket stays valid.  Other errors: FCLSH_EINVAL (NULL pointers, unknown ticket),
 * FCLSH_ENOMEM, or the status of the request's batch if that failed.
 */
fclsh_status fclsh_server_wait(fclsh_server *srv, uint64_t ticket, int timeout_ms, fclsh_result **out,
                               double *latency_ms);

/* Counters and latency percentiles of completed requests (no counterpart in the paper);
   reset = 1 starts a new window.  Errors: FCLSH_EINVAL (NULL pointers). */
fclsh_status fclsh_server_stats(fclsh_server *srv, fclsh_serve_stats *out, int reset);

/* Drain the queue, stop the scheduler and free the server (no counterpart in the paper).
   NULL is ignored. */
void fclsh_server_free(fclsh_server *srv);

/* ------------------------------------------------------------------ tuning */

/*
 * Read or set the index's kernel shapes and probe rule (fclsh_tuning; no counterpart in
 * the paper: they change speed only, never the reported ids).  fclsh_set_tuning checks
 * every field (ranges above; a hash tile the index's parts cannot use) and returns
 * FCLSH_EINVAL without changing anything if one is out of range.
 */
fclsh_status fclsh_get_tuning(const fclsh_index *idx, fclsh_tuning *out);
fclsh_status fclsh_set_tuning(fclsh_index *idx, const fclsh_tuning *tune);

/*
 * Time the kernel shapes on a sample: the query kernel's (verify-block shape,
 * blocks per SM, dedup set, probe fan-out) on a batch of queries (device or
 * host), and the hash kernel (WHT tiles, and the tensor-core contraction where it
 * applies) on the index's first points; keep the fastest.  The choice is cached in `cache_path` (JSON, may be NULL) keyed by
 * (n, d, r, t, W).  Results never depend on the choice; probe_rows is kept as
 * set.  A later build takes the hash tile through fclsh_build_opts.hash_tile.
 * No counterpart in the paper (results never depend on it).  Synchronous.
 * Errors: FCLSH_ERADIUS, FCLSH_EINVAL, FCLSH_ENOMEM, FCLSH_ECUDA.
 */
fclsh_status fclsh_autotune(fclsh_index *idx, const uint64_t *queries, uint64_t nq, uint32_t radius,
                            const char *cache_path, fclsh_tuning *chosen);

/* ------------------------------------------------------------------ timing */

/*
 * Per-phase device time (milliseconds, CUDA events on the launching stream)
 * accumulated since the last reset: [0] build hash kernel, [1] build sort and
 * directory kernels (all of them), [2] batched query kernels, [3] result CSR,
 * [4] fclsh_hash kernel, [5] build partition scatter kernel, [6] build
 * segment-finish kernels, [7] build partition histogram + scan ([5]-[7] are
 * parts of [1]), [8] heavy-query kernel (part of [2]).  counts[i] = timed launches of phase i.  Timing is off until enabled;
 * enabling adds one event pair per phase and runs query batches without graphs.
 * Measurement aid (no counterpart in the paper).  Errors: FCLSH_EINVAL, FCLSH_ECUDA.
 */
fclsh_status fclsh_timing_enable(fclsh_index *idx, int on);
fclsh_status fclsh_timing_read(fclsh_index *idx, double ms[9], uint64_t counts[9], int reset);

/* Kernels this library has enqueued in this process (a replayed CUDA graph counts its kernel
   nodes).  Measurement aid (no counterpart in the paper). */
uint64_t fclsh_kernel_launches(void);

/*
 * Testing aids for the out-of-memory paths (no counterpart in the paper).
 * fclsh_debug_fail_alloc(k): the k-th device allocation of this library from now on
 * (k = 0: the next one) fails as if the device were out of memory, once; k < 0 turns
 * the injection off.  Calls then return FCLSH_ENOMEM and must release what they took.
 * fclsh_debug_pool_used: bytes of the current device's library memory pool in use,
 * after a device synchronisation (freed memory stays reserved by the pool but is not
 * counted), so that a test can check that a failed call leaked nothing.
 */
fclsh_status fclsh_debug_fail_alloc(int64_t after);
fclsh_status fclsh_debug_pool_used(uint64_t *bytes);

/*
 * Testing aid for the bounded waits (no counterpart in the paper): while on = c + 1 > 0,
 * the tensor-core hash kernel (hash_tile 2) never requests its operand chunk c (on = 1:
 * the first), so its wait for that chunk runs out after about two seconds; the kernel
 * then waits (bounded) for the tensor-core work and copies it already issued, releases
 * its tensor memory and flags the index, and the call returns FCLSH_ETIMEOUT.  The
 * device stays usable.  on <= 0 turns it off.
 */
fclsh_status fclsh_debug_withhold_hash_loads(int on);

/*
 * Checked builds (no counterpart in the paper; the library compiled with -DFCLSH_CHECKED, the
 * stand-in for a memory checker): the kernels bounds-check their computed indexes, skip an
 * access that fails and record the check's code.  *checked = 1 in such a build (0 otherwise);
 * *first = the first failed check's code since the last call (0: none; always 0 in a normal
 * build).  Waits for the device.  Errors: FCLSH_EINVAL (NULL pointers), FCLSH_ECUDA.
 */
fclsh_status fclsh_debug_check_status(int *checked, uint32_t *first);

/* Thread-local description of the calling thread's last failure (no counterpart in the
   paper).  The string is owned by the library and valid until the thread's next call. */
const char *fclsh_last_error(void);

/* Library version string (static; no counterpart in the paper). */
const char *fclsh_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FCLSH_H */
