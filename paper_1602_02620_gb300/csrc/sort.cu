// sort.cu -- the bucket build (Sec. 2.2: only non-empty buckets are kept, one
// table per hash function) and the device-wide scans.
//
// Directory of a table: entries (key >> slot_bits) << entry_id_bits(slot_bits) | id grouped by slot
// (key mod 2^slot_bits) and, for every slot, the index of its first entry.  A
// query reads its slot, compares the stored high key bits and takes the ids of
// equal keys: its bucket.  Two builds give it:
//   * slot_bits <= 23 (MSD): a partition of each table by the top slot_bits - 12 slot
//     bits (segments of 4,096 slots), into fixed-capacity bins or, where a bin would
//     overflow, by an exact histogram; then one block per (segment, table) that counts
//     the segment into its slots in shared memory.  The order inside a slot's run is
//     the order its shared-memory atomics returned (a run is a set).
//   * otherwise (LSD): a stable radix sort by the slot bits (8-bit digits) and a
//     finalize pass; the input is in id order, so a slot's run is ordered by id.
//
// Radix pass = per-tile digit histogram -> one exclusive scan over
// (row, digit, tile) -> stable scatter.  Scanning in (row, digit, tile) order
// gives each tile's digit run its final position, rows included, in one scan.
// Stable ranks inside a tile come from digit-bit ballots + per-warp digit counts.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace fclsh {

namespace {

constexpr int kIPT = kSortSub / kSortThreads;    // items per thread per sub-tile (8)
constexpr int kWarps = kSortThreads / 32;

struct RadixArgs {
    const uint64_t *keys_in;
    const uint32_t *ids_in;       // nullptr: id = position in the row
    uint64_t *keys_out;
    uint32_t *ids_out;            // nullptr: keys only
    uint64_t len;                 // items per row (capacity when d_count is set)
    const unsigned long long *d_count;   // single row whose length is min(*d_count, len)
    uint32_t tiles;               // tiles per row
    uint32_t shift;
    uint32_t dmask;               // digit = (key >> shift) & dmask: the last pass may have fewer than 8 bits
    uint32_t *hist;               // [rows][256][tiles]
    uint32_t rows;
    uint32_t pack_sb;             // partition kernels: slot bits of the directory
    uint32_t pack_idbits;         // partition kernels: bits of an id
    uint32_t cap;                 // partition kernels: 0 = places from hist; else bins of cap entries
    uint32_t extra0;              //   (bin 0: cap + extra0; a row's bins: 2^D * cap + extra0)
    uint32_t *bin_cnt;            //   [rows][256] entries reserved in each bin (cap > 0)
    uint32_t *status;             //   bit 0 set when a bin overflowed (cap > 0)
    uint64_t out_cap = 0;         // partition kernels: entries keys_out holds (bounds of the checked build)
};

// Packed partition output for the MSD directory path (partition digit = the slot's
// top dbits bits, implied by the segment):
//   bits [52, 52+sub)   the slot's low sub = sb-dbits <= 12 bits
//   bits [idbits, 52)   the key's high bits key >> sb (50-sb bits; idbits <= sb + 2)
//   bits [0, idbits)    the id
__device__ __forceinline__ uint64_t pack_entry(uint64_t key, uint32_t id, uint32_t sb, uint32_t idbits, uint32_t dbits)
{
    const uint64_t sub = key & ((1ULL << (sb - dbits)) - 1);
    return (sub << 52) | ((key >> sb) << idbits) | id;
}

__device__ __forceinline__ uint64_t row_len(const RadixArgs &a)
{
    if (a.d_count) {
        unsigned long long c = *a.d_count;
        return c < a.len ? c : a.len;
    }
    return a.len;
}

__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(RadixArgs a)
{
    __shared__ uint32_t cnt[256];
    const uint32_t row = blockIdx.y, tile = blockIdx.x, tid = threadIdx.x;
    cnt[tid] = 0;
    __syncthreads();
    const uint64_t len = row_len(a);
    const uint64_t *K = a.keys_in + (uint64_t)row * a.len;
    const uint64_t base = (uint64_t)tile * kSortTile;
    constexpr int kBatch = 16;   // loads in flight per thread before their shared-memory counts
#pragma unroll
    for (int b = 0; b < kSortTile / (kSortThreads * kBatch); ++b) {
        uint32_t dg[kBatch];
#pragma unroll
        for (int i = 0; i < kBatch; ++i) {
            const uint64_t idx = base + (uint64_t)(b * kBatch + i) * kSortThreads + tid;
            dg[i] = idx < len ? ((uint32_t)(K[idx] >> a.shift) & a.dmask) : 0xFFFFFFFFu;
        }
#pragma unroll
        for (int i = 0; i < kBatch; ++i)
            if (dg[i] != 0xFFFFFFFFu) atomicAdd(&cnt[dg[i]], 1u);
    }
    __syncthreads();
    a.hist[((uint64_t)row * 256 + tid) * a.tiles + tile] = cnt[tid];
}

template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T *total);

// Lanes of the warp whose B-bit digit equals this lane's, among the lanes with
// `valid` set: one ballot per digit bit narrows the set (a warp-level multisplit).
template <int B>
__device__ __forceinline__ uint32_t same_digit_lanes(uint32_t digit, bool valid)
{
    uint32_t m = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const bool one = (digit >> b) & 1u;
        const uint32_t v = __ballot_sync(0xffffffffu, one);
        m &= one ? v : ~v;
    }
    return m;
}

// Stable scatter of one tile, in sub-tiles of kSortSub items taken in order.  In a
// sub-tile, warp w owns the items [w*256, (w+1)*256), taken in rounds of 32 in
// index order: ballots over the digit bits give each item its rank among equal
// digits in the round, and a warp-private counter per digit carries the rank
// across rounds (no block barrier).  One block-wide prefix over (digit, warp) then
// fixes every item's place in the sub-tile's digit-sorted order in shared memory,
// and the sub-tile's digit runs are written out as contiguous, coalesced runs.
// Each digit's global cursor starts at the tile's place from the scanned
// (row, digit, tile) histogram and advances by the digit's count per sub-tile.
template <bool IDS, bool IMPLICIT>
__global__ void __launch_bounds__(kSortThreads, 4) radix_scatter_kernel(RadixArgs a)
{
    constexpr int R = kIPT;   // rounds per warp and sub-tile: 8 x 32 = 256 items
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *sk = reinterpret_cast<uint64_t *>(smem_raw);        // [kSortSub] keys in digit order
    uint32_t *sg = reinterpret_cast<uint32_t *>(sk + kSortSub);   // [kSortSub] their global positions
    uint32_t *si = sg + kSortSub;                                 // [kSortSub] ids, when IDS
    __shared__ uint32_t global_off[256];
    __shared__ uint32_t warp_hist[kWarps][256];                   // counts, then each warp's base
    const uint32_t row = blockIdx.y, tile = blockIdx.x, tid = threadIdx.x;
    const uint32_t lane = tid & 31, warp = tid >> 5;
    const uint64_t len = row_len(a);
    const uint64_t base = (uint64_t)tile * kSortTile;
    if (base >= len) return;   // uniform: an empty tile has no items
    // digit tid's cursor: the tile's first global place for it
    uint32_t cursor = a.hist[((uint64_t)row * 256 + tid) * a.tiles + tile];
    const uint64_t *K = a.keys_in + (uint64_t)row * a.len;
    const uint32_t *I = IMPLICIT ? nullptr : a.ids_in + (uint64_t)row * a.len;
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t *wh = warp_hist[warp];
    for (uint64_t sbase = base; sbase < len && sbase < base + kSortTile; sbase += kSortSub) {
        const uint64_t wbase = sbase + (uint64_t)warp * (32 * R);
        // every load of the warp's part is issued before the ranking loop, whose
        // __syncwarp()s would otherwise keep the next round's load from being hoisted
        uint64_t key[R];
        uint32_t id[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint64_t idx = wbase + (uint64_t)r * 32 + lane;
            key[r] = idx < len ? K[idx] : 0;
            if (IDS) id[r] = IMPLICIT ? (uint32_t)idx : (idx < len ? I[idx] : 0u);
        }
#pragma unroll
        for (int w = 0; w < kWarps; ++w) warp_hist[w][tid] = 0;
        __syncthreads();   // (also: the previous sub-tile's output is read out)
        uint32_t lr[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint64_t idx = wbase + (uint64_t)r * 32 + lane;
            const bool valid = idx < len;
            const uint32_t digit = valid ? ((uint32_t)(key[r] >> a.shift) & a.dmask) : 0u;
            const uint32_t peers = same_digit_lanes<8>(digit, valid);
            const uint32_t before = valid ? wh[digit] : 0u;
            lr[r] = before + __popc(peers & lt_mask);
            __syncwarp();
            if (valid && (peers & lt_mask) == 0) wh[digit] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        {   // thread tid owns digit tid: its count, its place in the sub-tile, each warp's first place
            uint32_t c = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) c += warp_hist[w][tid];
            uint32_t tot;
            uint32_t run = block_excl_scan<uint32_t>(c, &tot);   // barriers inside
            global_off[tid] = cursor - run;   // global place of sub-tile position p of digit tid: global_off + p
            cursor += c;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t cw = warp_hist[w][tid];
                warp_hist[w][tid] = run;
                run += cw;
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint64_t idx = wbase + (uint64_t)r * 32 + lane;
            if (idx < len) {
                const uint32_t digit = (uint32_t)(key[r] >> a.shift) & a.dmask;
                const uint32_t lp = wh[digit] + lr[r];
                sk[lp] = key[r];
                sg[lp] = global_off[digit] + lp;
                if (IDS) si[lp] = id[r];
            }
        }
        __syncthreads();
        const uint32_t sub_n = (uint32_t)((len - sbase) < (uint64_t)kSortSub ? (len - sbase) : (uint64_t)kSortSub);
        for (uint32_t i = tid; i < sub_n; i += kSortThreads) {
            const uint32_t g = sg[i];
            a.keys_out[g] = sk[i];
            if (IDS) a.ids_out[g] = si[i];
        }
    }
}

// Partition of every table by the top 8 slot bits for the s <= 20 directory path,
// packed output.  It need not be stable: segment_one_kernel and
// segment_finish_kernel group a segment by slot whatever its order, and the order
// inside a slot is not part of the directory.  So a sub-tile is ranked with
// shared-memory atomics on one counter per digit (no warp-level multisplit),
// reordered by digit in shared memory and written as contiguous digit runs.
// Where the runs go: with cap = 0 each digit's global cursor starts at the tile's
// place from the scanned (row, digit, tile) histogram and advances by the digit's
// count per sub-tile.  With cap > 0 (no histogram pass) segment (row, digit) is a
// bin of cap entries and each sub-tile reserves its run in the bin with one global
// atomic; a run that would pass the bin's end is dropped and flagged in *status
// (the caller then rebuilds these tables the exact way).
__global__ void __launch_bounds__(kSortThreads, 4) partition_scatter_kernel(RadixArgs a)
{
    constexpr int R = kIPT;   // items per thread and sub-tile
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *sk = reinterpret_cast<uint64_t *>(smem_raw);        // [kSortSub] packed entries in digit order
    uint32_t *sg = reinterpret_cast<uint32_t *>(sk + kSortSub);   // [kSortSub] their global positions
    __shared__ uint32_t cnt[256], gofs[256];
    const uint32_t row = blockIdx.y, tile = blockIdx.x, tid = threadIdx.x;
    const uint64_t len = a.len;
    const uint64_t base = (uint64_t)tile * kSortTile;
    if (base >= len) return;   // uniform: an empty tile has no items
    uint32_t cursor = a.cap ? 0u : a.hist[((uint64_t)row * 256 + tid) * a.tiles + tile];   // digit tid's next place
    const uint64_t *K = a.keys_in + (uint64_t)row * len;
    uint64_t nxt[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint64_t idx = base + (uint64_t)r * kSortThreads + tid;
        nxt[r] = idx < len ? K[idx] : 0;
    }
    for (uint64_t sbase = base; sbase < len && sbase < base + kSortTile; sbase += kSortSub) {
        uint64_t key[R];
#pragma unroll
        for (int r = 0; r < R; ++r) key[r] = nxt[r];
        if (sbase + kSortSub < base + kSortTile) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint64_t idx = sbase + kSortSub + (uint64_t)r * kSortThreads + tid;
                nxt[r] = idx < len ? K[idx] : 0;
            }
        }
        cnt[tid] = 0;
        __syncthreads();   // (also: the previous sub-tile's output is read out)
        uint32_t rk[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint64_t idx = sbase + (uint64_t)r * kSortThreads + tid;
            if (idx < len) rk[r] = atomicAdd(&cnt[(uint32_t)(key[r] >> a.shift) & 255u], 1u);
        }
        __syncthreads();
        {   // thread tid owns digit tid: its place in the sub-tile and its global offset
            const uint32_t c = cnt[tid];
            uint32_t tot;
            const uint32_t start = block_excl_scan<uint32_t>(c, &tot);   // barriers inside
            if (a.cap == 0) {
                gofs[tid] = cursor - start;   // global place of sub-tile position p of digit tid: gofs + p
                cursor += c;
            } else {
                const uint32_t at = c ? atomicAdd(a.bin_cnt + (uint64_t)row * 256 + tid, c) : 0u;
                if (at + c <= bin_capacity(tid, a.cap, a.extra0)) {
                    gofs[tid] = (uint32_t)((uint64_t)row * (256ull * a.cap + a.extra0) + bin_start(tid, a.cap, a.extra0) +
                                           at) - start;
                } else {
                    gofs[tid] = 0xFFFFFFFFu;   // dropped: the bin is full
                    atomicOr(a.status, 1u);
                }
            }
            cnt[tid] = start;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint64_t idx = sbase + (uint64_t)r * kSortThreads + tid;
            if (idx < len) {
                const uint32_t digit = (uint32_t)(key[r] >> a.shift) & 255u;
                const uint32_t lp = cnt[digit] + rk[r];
                const uint32_t go = gofs[digit];
                sk[lp] = pack_entry(key[r], (uint32_t)idx, a.pack_sb, a.pack_idbits, 8);
                sg[lp] = go == 0xFFFFFFFFu ? go : go + lp;
            }
        }
        __syncthreads();
        const uint32_t sub_n = (uint32_t)((len - sbase) < (uint64_t)kSortSub ? (len - sbase) : (uint64_t)kSortSub);
        for (uint32_t i = tid; i < sub_n; i += kSortThreads) {
            const uint32_t g = sg[i];
            if (g != 0xFFFFFFFFu && FCLSH_CHECK(!a.out_cap || g < a.out_cap, 0x0301)) a.keys_out[g] = sk[i];
        }
    }
}

// Partition of every table by the slot's top D = 9..11 bits (slot_bits 21..23),
// packed output; segments then hold 2^(slot_bits-D) = 4,096 slots, as at
// slot_bits = 20.  Into fixed-capacity bins (cap > 0): with 2^D digits a sub-tile's
// runs are short, so a block first counts its whole tile of kWideTile keys and
// reserves each digit's run in its bin with one global atomic (the keys are read
// twice; the second time they come from L2); a run that would pass its bin's end is
// dropped and flagged.  Exact form (cap = 0): the tile's places come from the
// scanned per-tile histogram of wide_hist_kernel.  Either way the tile is ranked,
// reordered and written in sub-tiles of kWideSub.
constexpr int kWideThreads = 512;
constexpr int kWideSub = 4096;                 // 8 keys per thread
constexpr int kWideSubs = 4;
constexpr int kWideTile = kWideSub * kWideSubs;

// Exact form's digit counts of one wide tile: hist[(row * 2^D + d) * tiles + tile].
template <int D>
__global__ void __launch_bounds__(kWideThreads) wide_hist_kernel(RadixArgs a)
{
    constexpr uint32_t ND = 1u << D;
    constexpr int R = kWideSub / kWideThreads;
    __shared__ uint32_t cnt[ND];
    const uint32_t row = blockIdx.y, tile = blockIdx.x, tid = threadIdx.x;
    const uint64_t len = a.len;
    const uint64_t base = (uint64_t)tile * kWideTile;
    const uint64_t *K = a.keys_in + (uint64_t)row * len;
    for (uint32_t d = tid; d < ND; d += kWideThreads) cnt[d] = 0;
    __syncthreads();
    for (int sbk = 0; sbk < kWideSubs; ++sbk) {
        uint32_t dg[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint64_t idx = base + (uint64_t)sbk * kWideSub + (uint64_t)r * kWideThreads + tid;
            dg[r] = idx < len ? ((uint32_t)(K[idx] >> a.shift) & (ND - 1)) : 0xFFFFFFFFu;
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (dg[r] != 0xFFFFFFFFu) atomicAdd(&cnt[dg[r]], 1u);
    }
    __syncthreads();
    for (uint32_t d = tid; d < ND; d += kWideThreads) a.hist[(((uint64_t)row << D) + d) * a.tiles + tile] = cnt[d];
}

template <int D>
__global__ void __launch_bounds__(kWideThreads, 2) partition_wide_kernel(RadixArgs a)
{
    constexpr uint32_t ND = 1u << D;
    constexpr int R = kWideSub / kWideThreads;
    constexpr uint32_t PER = ND >= kWideThreads ? ND / kWideThreads : 1;   // digits per thread in the scans
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *sk = reinterpret_cast<uint64_t *>(smem_raw);        // [kWideSub] packed entries in digit order
    uint32_t *sg = reinterpret_cast<uint32_t *>(sk + kWideSub);   // [kWideSub] their global positions
    __shared__ uint32_t cnt[ND], st[ND], cur[ND], gofs[ND];
    const uint32_t row = blockIdx.y, tid = threadIdx.x;
    const bool owner = tid * PER < ND;   // thread tid takes digits [tid*PER, tid*PER + PER) in the scans
    const uint64_t len = a.len;
    const uint64_t base = (uint64_t)blockIdx.x * kWideTile;
    if (base >= len) return;   // uniform
    const uint64_t *K = a.keys_in + (uint64_t)row * len;
    const uint32_t shift = a.shift;
    for (uint32_t d = tid; d < ND; d += kWideThreads) {
        cnt[d] = 0;
        cur[d] = 0;
    }
    __syncthreads();
    for (int sbk = 0; a.cap && sbk < kWideSubs; ++sbk) {   // bins: the tile's digit counts
        uint32_t dg[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint64_t idx = base + (uint64_t)sbk * kWideSub + (uint64_t)r * kWideThreads + tid;
            dg[r] = idx < len ? ((uint32_t)(K[idx] >> shift) & (ND - 1)) : 0xFFFFFFFFu;
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (dg[r] != 0xFFFFFFFFu) atomicAdd(&cnt[dg[r]], 1u);
    }
    __syncthreads();
    for (uint32_t d = tid; d < ND; d += kWideThreads) {   // reserve the tile's runs in the bins
        if (a.cap == 0) {   // exact form: the tile's places from the scanned histogram
            gofs[d] = a.hist[(((uint64_t)row << D) + d) * a.tiles + blockIdx.x];
            continue;
        }
        const uint32_t c = cnt[d];
        const uint32_t at = c ? atomicAdd(a.bin_cnt + (uint64_t)row * ND + d, c) : 0u;
        if (at + c <= bin_capacity(d, a.cap, a.extra0)) {
            gofs[d] = (uint32_t)((uint64_t)row * ((uint64_t)ND * a.cap + a.extra0) + bin_start(d, a.cap, a.extra0) + at);
        } else {
            gofs[d] = 0xFFFFFFFFu;   // dropped: the bin is full
            atomicOr(a.status, 1u);
        }
    }
    for (uint64_t sbase = base; sbase < len && sbase < base + kWideTile; sbase += kWideSub) {
        uint64_t key[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint64_t idx = sbase + (uint64_t)r * kWideThreads + tid;
            key[r] = idx < len ? K[idx] : 0;
        }
        for (uint32_t d = tid; d < ND; d += kWideThreads) cnt[d] = 0;
        __syncthreads();   // (also: the previous sub-tile's output is read out, cur advanced)
        uint32_t rk[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint64_t idx = sbase + (uint64_t)r * kWideThreads + tid;
            if (idx < len) rk[r] = atomicAdd(&cnt[(uint32_t)(key[r] >> shift) & (ND - 1)], 1u);
        }
        __syncthreads();
        {   // thread tid owns digits [tid*PER, tid*PER + PER): their first places in the sub-tile
            uint32_t c[PER], mine = 0;
#pragma unroll
            for (uint32_t i = 0; i < PER; ++i) {
                c[i] = owner ? cnt[tid * PER + i] : 0u;
                mine += c[i];
            }
            uint32_t tot;
            uint32_t run = block_excl_scan<uint32_t>(mine, &tot);   // barriers inside
#pragma unroll
            for (uint32_t i = 0; i < PER; ++i) {
                if (owner) st[tid * PER + i] = run;
                run += c[i];
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint64_t idx = sbase + (uint64_t)r * kWideThreads + tid;
            if (idx < len) {
                const uint32_t digit = (uint32_t)(key[r] >> shift) & (ND - 1);
                const uint32_t lp = st[digit] + rk[r];
                const uint32_t go = gofs[digit];
                sk[lp] = pack_entry(key[r], (uint32_t)idx, a.pack_sb, a.pack_idbits, D);
                sg[lp] = go == 0xFFFFFFFFu ? go : go + cur[digit] + rk[r];
            }
        }
        __syncthreads();
        const uint32_t sub_n = (uint32_t)((len - sbase) < (uint64_t)kWideSub ? (len - sbase) : (uint64_t)kWideSub);
        for (uint32_t i = tid; i < sub_n; i += kWideThreads) {
            const uint32_t g = sg[i];
            if (g != 0xFFFFFFFFu && FCLSH_CHECK(!a.out_cap || g < a.out_cap, 0x0302)) a.keys_out[g] = sk[i];
        }
        for (uint32_t d = tid; d < ND; d += kWideThreads) cur[d] += cnt[d];
    }
}

// ---------------------------------------------------------------- scans

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) >= (unsigned)o) v += u;
    }
    return v;
}

// Exclusive block scan of one value per thread (256 threads); returns the block total in *total.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T *total)
{
    __shared__ T wsum[32];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nw = blockDim.x >> 5;
    T incl = warp_incl_scan(v);
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? wsum[lane] : T(0);
        T wi = warp_incl_scan(w);
        if (lane < nw) wsum[lane] = wi - w;
        if (lane == nw - 1) wsum[31] = wi;
    }
    __syncthreads();
    T res = incl - v + wsum[warp];
    *total = wsum[31];
    __syncthreads();
    return res;
}

constexpr int kScanChunk = 256 * 16;

template <typename Tin, typename Tacc>
__global__ void __launch_bounds__(256) scan_reduce_kernel(const Tin *in, uint64_t count, Tacc *partials)
{
    const uint64_t base = (uint64_t)blockIdx.x * kScanChunk;
    Tacc s = 0;
    for (int i = 0; i < 16; ++i) {
        const uint64_t idx = base + (uint64_t)i * 256 + threadIdx.x;
        if (idx < count) s += (Tacc)in[idx];
    }
    Tacc total;
    block_excl_scan<Tacc>(s, &total);
    if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

template <typename Tacc>
__global__ void __launch_bounds__(256) scan_partials_kernel(Tacc *partials, uint64_t count)
{
    Tacc carry = 0;
    for (uint64_t base = 0; base < count; base += 256) {
        const uint64_t idx = base + threadIdx.x;
        Tacc v = idx < count ? partials[idx] : Tacc(0);
        Tacc total;
        Tacc ex = block_excl_scan<Tacc>(v, &total);
        if (idx < count) partials[idx] = ex + carry;
        carry += total;
    }
    if (threadIdx.x == 0) partials[count] = carry;
}

template <typename Tin, typename Tout, typename Tacc>
__global__ void __launch_bounds__(256) scan_down_kernel(const Tin *in, Tout *out, uint64_t count, const Tacc *partials,
                                                        bool write_total)
{
    const uint64_t base = (uint64_t)blockIdx.x * kScanChunk;
    // each thread owns 16 consecutive items
    Tacc v[16];
    Tacc s = 0;
    const uint64_t my = base + (uint64_t)threadIdx.x * 16;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        v[i] = (my + i < count) ? (Tacc)in[my + i] : Tacc(0);
        s += v[i];
    }
    Tacc total;
    Tacc run = block_excl_scan<Tacc>(s, &total) + partials[blockIdx.x];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        if (my + i < count) out[my + i] = (Tout)run;
        run += v[i];
    }
    if (write_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[count] = (Tout)partials[gridDim.x];
}

template <typename Tin, typename Tout, typename Tacc>
cudaError_t scan_exclusive(const Tin *in, Tout *out, uint64_t count, Tacc *partials, bool write_total, cudaStream_t s)
{
    const uint64_t chunks = (count + kScanChunk - 1) / kScanChunk;
    if (chunks == 0) {
        if (write_total) return cudaMemsetAsync(out, 0, sizeof(Tout), s);
        return cudaSuccess;
    }
    scan_reduce_kernel<Tin, Tacc><<<(unsigned)chunks, 256, 0, s>>>(in, count, partials);
    note_launch();
    scan_partials_kernel<Tacc><<<1, 256, 0, s>>>(partials, chunks);
    note_launch();
    scan_down_kernel<Tin, Tout, Tacc><<<(unsigned)chunks, 256, 0, s>>>(in, out, count, partials, write_total);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- directory

__global__ void __launch_bounds__(256) finalize_kernel(const uint64_t *__restrict__ keys,
                                                       const uint32_t *__restrict__ ids, uint64_t len,
                                                       uint32_t sb, uint64_t *__restrict__ ent,
                                                       uint32_t *__restrict__ offs)
{
    const uint32_t row = blockIdx.y;
    const uint64_t e = (uint64_t)blockIdx.x * 256 + threadIdx.x;
    if (e >= len) return;
    const uint64_t nslots = 1ULL << sb;
    const uint64_t mask = nslots - 1;
    const uint64_t *Kr = keys + (uint64_t)row * len;
    uint32_t *O = offs + (uint64_t)row * dir_stride(sb);
    const uint64_t key = Kr[e];
    const uint64_t sl = key & mask;
    ent[(uint64_t)row * len + e] = ((key >> sb) << entry_id_bits(sb)) | ids[(uint64_t)row * len + e];
    const uint64_t first = (e == 0) ? 0 : (Kr[e - 1] & mask) + 1;
    for (uint64_t s2 = first; s2 <= sl; ++s2) O[s2] = (uint32_t)e;
    if (e == len - 1)
        for (uint64_t s2 = sl + 1; s2 <= nslots; ++s2) O[s2] = (uint32_t)len;
}



// ---------------------------------------------------------------- directory, second half (MSD path)

constexpr int kSegThreads = 512;
constexpr int kSegItems = 4;                          // entries per thread in flight per round
constexpr int kSubMaxBits = 12;                       // slot bits below the partition digit

// One shared-memory atomic add of 1 per lane on cnt[j], aggregated over the lanes of the
// warp that take the same j (valid lanes only; every lane of the warp calls it): the
// lowest lane of each group adds the group's size once.  Returns the counter's value
// before the lane's own unit, i.e. the lane's place among the entries counted so far.
__device__ __forceinline__ uint32_t warp_aggregated_add(uint32_t *cnt, uint32_t j, bool valid)
{
    const uint32_t act = __ballot_sync(0xffffffffu, valid);
    if (!valid) return 0;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t peers = __match_any_sync(act, j);
    const uint32_t leader = (uint32_t)__ffs(peers) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&cnt[j], (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
}

// Exclusive scan in place of v[0..cnt) (cnt <= 4096) by the whole block; optionally
// also writes out[j] = base + prefix.
__device__ __forceinline__ void seg_scan(uint32_t *v, uint32_t cnt, uint32_t *wsum, uint32_t *out, uint32_t base)
{
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t per = (cnt + kSegThreads - 1) / kSegThreads;
    const uint32_t j0 = tid * per;
    uint32_t loc = 0;
    for (uint32_t j = j0; j < j0 + per && j < cnt; ++j) loc += v[j];
    uint32_t incl = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += u;
    }
    __syncthreads();
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t run = incl - loc;
    for (uint32_t w = 0; w < warp; ++w) run += wsum[w];
    for (uint32_t j = j0; j < j0 + per && j < cnt; ++j) {
        const uint32_t c = v[j];
        v[j] = run;
        if (out) out[j] = base + run;
        run += c;
    }
    __syncthreads();
}

constexpr int kOneThreads = 512;
constexpr int kOneWarps = kOneThreads / 32;
constexpr int kOneItems = 9;                         // entries per thread
constexpr int kOneCap = kOneThreads * kOneItems;     // 4,608 entries: a full bin of a 4,096-slot segment
constexpr int kOneSlots = 8;                         // directory slots owned per thread (2^12 / 512)

// Padded index of per-slot counters: four spare words after every 32, so that the
// eight consecutive counters a thread owns start on a 16-byte boundary and the
// vector accesses of a quarter-warp fall on distinct banks.
__device__ __forceinline__ uint32_t pj(uint32_t j) { return j + ((j >> 5) << 2); }

// seg_out[row][g] = first directory entry of segment (row, g) within its row, for
// the 2^dbits segments g of a row, and seg_out[row][2^dbits] = n: from the scanned
// (row, digit, tile) histogram (bin_cnt == nullptr) or by a prefix over
// the bins' fills.  One block of 256 threads per row; thread t takes 2^dbits/256
// consecutive segments.
__global__ void __launch_bounds__(256) segment_bounds_kernel(const uint32_t *__restrict__ hist, uint32_t tiles,
                                                             uint64_t n, const uint32_t *__restrict__ bin_cnt,
                                                             uint32_t dbits, uint32_t *__restrict__ seg_out)
{
    const uint32_t row = blockIdx.x, tid = threadIdx.x;
    const uint32_t nd = 1u << dbits, per = nd >= 256 ? nd / 256 : 1;
    const bool owner = tid * per < nd;   // fewer segments than threads: the first nd threads take one each
    uint32_t *out = seg_out + (uint64_t)row * (nd + 1);
    if (bin_cnt) {
        const uint32_t *c = bin_cnt + (uint64_t)row * nd + tid * per;
        uint32_t mine = 0;
        if (owner)
            for (uint32_t i = 0; i < per; ++i) mine += c[i];
        uint32_t tot;
        uint32_t run = block_excl_scan<uint32_t>(mine, &tot);
        if (owner)
            for (uint32_t i = 0; i < per; ++i) {
                out[tid * per + i] = run;
                run += c[i];
            }
    } else if (owner) {
        for (uint32_t i = 0; i < per; ++i)
            out[tid * per + i] = hist[(((uint64_t)row << dbits) + tid * per + i) * tiles] - (uint32_t)((uint64_t)row * n);
    }
    if (tid == 0) out[nd] = (uint32_t)n;
}

// One block per (segment, table) for segments of at most kOneCap = 4,608 entries
// (the common case: a segment of 4,096 slots holds ~n/2^dbits of them).  Entries are counted into their slots with shared-memory
// atomics; thread i owns the eight consecutive slots [8i, 8i+8): it scans their
// counts in registers and writes their directory words with two vector stores.
// Each entry is then placed in its slot's run at the place its atomic returned
// (the order inside a run is not part of the directory), and the segment's
// entries are written with coalesced stores.  Larger segments are listed for
// segment_finish_kernel.
// Segment (row, g) of the partition: seg_out[row][g] .. seg_out[row][g+1] in the row's
// directory entries; its packed input starts at row * in_stride + (cap ? bin_start(g) : seg_out[row][g]).
__global__ void __launch_bounds__(kOneThreads, 3) segment_one_kernel(const uint64_t *__restrict__ packed, uint64_t n,
                                                                     uint64_t in_stride, uint32_t cap, uint32_t extra0,
                                                                     uint32_t sb,
                                                                     uint32_t idbits, uint32_t dbits,
                                                                     const uint32_t *__restrict__ seg_out,
                                                                     uint64_t *__restrict__ ent,
                                                                     uint32_t *__restrict__ offs,
                                                                     unsigned long long *big_cnt, uint32_t *big)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *ck = reinterpret_cast<uint64_t *>(smem_raw);             // [kOneCap]
    uint32_t *cnt = reinterpret_cast<uint32_t *>(ck + kOneCap);         // [pj(nsub)]
    __shared__ uint32_t wsum[kOneWarps];
    const uint32_t g = blockIdx.x, row = blockIdx.y, tid = threadIdx.x;
    const uint32_t lane = tid & 31, warp = tid >> 5;
    const uint32_t nd = 1u << dbits, subb = sb - dbits, nsub = 1u << subb, smask = nsub - 1;
    const uint64_t low52 = (1ULL << 52) - 1, idmask = (1ULL << idbits) - 1;
    const uint32_t lo = seg_out[(uint64_t)row * (nd + 1) + g], hi = seg_out[(uint64_t)row * (nd + 1) + g + 1];
    const uint32_t len = hi - lo;
    if (len > (uint32_t)kOneCap) {
        if (tid == 0) big[atomicAdd(big_cnt, 1ULL)] = (row << dbits) | g;
        return;
    }
    const uint32_t cn = len;
    if (!FCLSH_CHECK((uint64_t)lo + cn <= n, 0x0303)) return;   // block-uniform, before any barrier
    const uint64_t rowbase = (uint64_t)row * n;
    const uint64_t *Pk = packed + (uint64_t)row * in_stride + (cap ? bin_start(g, cap, extra0) : (uint64_t)lo);
    uint64_t *E = ent + rowbase + lo;
    uint32_t *O = offs + (uint64_t)row * dir_stride(sb) + (uint64_t)g * nsub;   // 16-byte aligned (nsub >= 8)
    if (g == nd - 1 && tid == 0) O[nsub] = (uint32_t)n;
    uint64_t v[kOneItems];
    uint32_t rk[kOneItems];
#pragma unroll
    for (int r = 0; r < kOneItems; ++r) {
        const uint32_t idx = tid + r * kOneThreads;
        v[r] = idx < cn ? Pk[idx] : 0;
    }
    uint4 *cnt4 = reinterpret_cast<uint4 *>(cnt);
    for (uint32_t i = tid; i < pj(nsub) / 4; i += kOneThreads) cnt4[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kOneItems; ++r)
        if (tid + r * kOneThreads < cn) rk[r] = atomicAdd(&cnt[pj((uint32_t)(v[r] >> 52) & smask)], 1u);
    __syncthreads();

    // counts of the owned slots -> their first entries
    const uint32_t j0 = tid * kOneSlots;
    const bool owner = j0 < nsub;
    uint32_t c[kOneSlots], st[kOneSlots];
    if (owner) {
        const uint4 x = cnt4[pj(j0) / 4], y = cnt4[pj(j0) / 4 + 1];
        c[0] = x.x, c[1] = x.y, c[2] = x.z, c[3] = x.w, c[4] = y.x, c[5] = y.y, c[6] = y.z, c[7] = y.w;
    } else {
#pragma unroll
        for (int i = 0; i < kOneSlots; ++i) c[i] = 0;
    }
    uint32_t tot = 0;
#pragma unroll
    for (int i = 0; i < kOneSlots; ++i) {
        st[i] = tot;
        tot += c[i];
    }
    uint32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t wv = lane < (uint32_t)kOneWarps ? wsum[lane] : 0u, wincl = wv;
#pragma unroll
    for (int o = 1; o < kOneWarps; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, wincl, o);
        if (lane >= (uint32_t)o) wincl += u;
    }
    const uint32_t before = __shfl_sync(0xffffffffu, wincl - wv, warp) + incl - tot;
#pragma unroll
    for (int i = 0; i < kOneSlots; ++i) st[i] += before;
    if (owner && FCLSH_CHECK((uint64_t)g * nsub + j0 + 8 <= dir_stride(sb), 0x0304)) {
        // the owned slots' first entries, for the placement and the directory
        cnt4[pj(j0) / 4] = make_uint4(st[0], st[1], st[2], st[3]);
        cnt4[pj(j0) / 4 + 1] = make_uint4(st[4], st[5], st[6], st[7]);
        const uint32_t l = (uint32_t)lo;
        uint4 *O4 = reinterpret_cast<uint4 *>(O + j0);
        O4[0] = make_uint4(l + st[0], l + st[1], l + st[2], l + st[3]);
        O4[1] = make_uint4(l + st[4], l + st[5], l + st[6], l + st[7]);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kOneItems; ++r)
        if (tid + r * kOneThreads < cn) ck[cnt[pj((uint32_t)(v[r] >> 52) & smask)] + rk[r]] = v[r];
    __syncthreads();
    for (uint32_t i = tid; i < cn; i += kOneThreads) {
        const uint64_t x = ck[i];
        E[i] = ((x & low52) >> idbits) << entry_id_bits(sb) | (x & idmask);
    }
}

// Segments longer than kOneCap entries (listed by segment_one_kernel; a key that
// repeats in many points, such as the empty sum of sparse points, puts thousands of
// entries into one slot): blocks take the listed segments in turn.  The segment's
// entries are counted into their slots with warp-aggregated shared-memory atomics, the
// counts are scanned into each slot's first entry (written to the directory), and each
// entry goes to its slot's run at the place a second aggregated atomic returns.  The
// order inside a run is not part of the directory; the lanes of a warp that share a slot
// take consecutive places, so the heavy slot is written with coalesced stores.
__global__ void __launch_bounds__(kSegThreads, 3) segment_finish_kernel(const uint64_t *__restrict__ packed,
                                                                        uint64_t n, uint64_t in_stride, uint32_t cap,
                                                                        uint32_t extra0,
                                                                        uint32_t sb, uint32_t idbits, uint32_t dbits,
                                                                        const uint32_t *__restrict__ seg_out,
                                                                        uint64_t *__restrict__ ent,
                                                                        uint32_t *__restrict__ offs,
                                                                        const unsigned long long *big_cnt,
                                                                        const uint32_t *big)
{
    __shared__ uint32_t sub_off[1u << kSubMaxBits];
    __shared__ uint32_t wsum[32];
    const unsigned long long nbig = *big_cnt;
    const uint32_t nd = 1u << dbits, tid = threadIdx.x;
    const uint32_t subb = sb - dbits, nsub = 1u << subb, smask = nsub - 1;
    const uint64_t low52 = (1ULL << 52) - 1, idmask = (1ULL << idbits) - 1;
    auto sub_of = [&](uint64_t v) { return (uint32_t)(v >> 52) & smask; };
    auto ent_of = [&](uint64_t v) { return ((v & low52) >> idbits) << entry_id_bits(sb) | (v & idmask); };
    for (unsigned long long bi = blockIdx.x; bi < nbig; bi += gridDim.x) {
        const uint32_t g = big[bi] & (nd - 1), row = big[bi] >> dbits;
        const uint32_t seg_lo = seg_out[(uint64_t)row * (nd + 1) + g], seg_hi = seg_out[(uint64_t)row * (nd + 1) + g + 1];
        const uint64_t seg_len = seg_hi - seg_lo;
        if (!FCLSH_CHECK((uint64_t)seg_lo + seg_len <= n && seg_lo <= seg_hi, 0x0306)) return;   // block-uniform
        const uint64_t *Pk = packed + (uint64_t)row * in_stride + (cap ? bin_start(g, cap, extra0) : (uint64_t)seg_lo);
        uint64_t *E = ent + (uint64_t)row * n + seg_lo;
        uint32_t *O = offs + (uint64_t)row * dir_stride(sb) + (uint64_t)g * nsub;
        if (g == nd - 1 && tid == 0) O[nsub] = (uint32_t)n;

        for (uint32_t j = tid; j < nsub; j += kSegThreads) sub_off[j] = 0;
        __syncthreads();
        // every lane runs the same rounds (the aggregated atomics need whole warps)
        for (uint64_t e0 = 0; e0 < seg_len; e0 += (uint64_t)kSegThreads * kSegItems) {
            uint64_t v[kSegItems];
#pragma unroll
            for (int r = 0; r < kSegItems; ++r) {
                const uint64_t e = e0 + (uint64_t)r * kSegThreads + tid;
                v[r] = e < seg_len ? Pk[e] : 0;
            }
#pragma unroll
            for (int r = 0; r < kSegItems; ++r)
                warp_aggregated_add(sub_off, sub_of(v[r]), e0 + (uint64_t)r * kSegThreads + tid < seg_len);
        }
        __syncthreads();
        seg_scan(sub_off, nsub, wsum, O, seg_lo);   // sub_off[j]: slot j's first entry in the segment
        for (uint64_t e0 = 0; e0 < seg_len; e0 += (uint64_t)kSegThreads * kSegItems) {
            uint64_t v[kSegItems];
#pragma unroll
            for (int r = 0; r < kSegItems; ++r) {
                const uint64_t e = e0 + (uint64_t)r * kSegThreads + tid;
                v[r] = e < seg_len ? Pk[e] : 0;
            }
#pragma unroll
            for (int r = 0; r < kSegItems; ++r) {
                const bool valid = e0 + (uint64_t)r * kSegThreads + tid < seg_len;
                const uint32_t at = warp_aggregated_add(sub_off, sub_of(v[r]), valid);
                if (valid && FCLSH_CHECK(at < seg_len, 0x0305)) E[at] = ent_of(v[r]);
            }
        }
        __syncthreads();
    }
}

}  // namespace

constexpr size_t kScatterSmemIds = (size_t)kSortSub * 16;
constexpr size_t kScatterSmemKeys = (size_t)kSortSub * 12;

// The scatter kernels use more than 48 KB of shared memory; raise their limit once.
static cudaError_t scatter_smem_init()
{
    static cudaError_t once = [] {
        cudaError_t e = cudaFuncSetAttribute(radix_scatter_kernel<true, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmemIds);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(radix_scatter_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kScatterSmemIds);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(radix_scatter_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kScatterSmemKeys);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(partition_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kScatterSmemKeys);
        return e;
    }();
    return once;
}

size_t sort_hist_entries(uint32_t rows, uint64_t len, uint32_t dbits)
{
    const uint64_t tiles = (len + kSortTile - 1) / kSortTile;
    const uint64_t wide = dbits != 8 ? ((uint64_t)1 << dbits) * ((len + kWideTile - 1) / kWideTile) : 0;
    return (size_t)rows * std::max<uint64_t>(256 * tiles, wide);
}

// Histogram tiles per row of the partition with dbits-bit digits.
static uint32_t msd_tiles(uint64_t len, uint32_t dbits)
{
    const uint64_t t = dbits == 8 ? kSortTile : kWideTile;
    return (uint32_t)((len + t - 1) / t);
}

size_t sort_keys_hist_entries(uint64_t cap) { return sort_hist_entries(1, cap, 8); }

size_t scan_partials_entries(size_t count) { return (count + kScanChunk - 1) / kScanChunk + 2; }

cudaError_t radix_sort_rows(const uint64_t *keys_in, uint32_t rows, uint64_t len, uint32_t bits, SortBuffers &buf,
                            bool *out_in_b, cudaStream_t s)
{
    cudaError_t e0 = scatter_smem_init();
    if (e0 != cudaSuccess) return e0;
    const uint32_t tiles = (uint32_t)((len + kSortTile - 1) / kSortTile);
    const uint32_t passes = (bits + 7) / 8;
    const uint64_t hcount = (uint64_t)rows * 256 * tiles;
    dim3 grid(tiles, rows);
    const uint64_t *kin = keys_in;
    const uint32_t *iin = nullptr;
    for (uint32_t p = 0; p < passes; ++p) {
        const bool to_b = (p % 2) == 1;
        const uint32_t nb = bits - 8 * p < 8 ? bits - 8 * p : 8;
        RadixArgs a{kin, iin, to_b ? buf.keys_b : buf.keys_a, to_b ? buf.ids_b : buf.ids_a, len, nullptr, tiles,
                    8 * p, (1u << nb) - 1u, buf.hist, rows};
        radix_hist_kernel<<<grid, kSortThreads, 0, s>>>(a);
        note_launch();
        cudaError_t e = scan_exclusive<uint32_t, uint32_t, uint32_t>(buf.hist, buf.hist, hcount, buf.partials, false, s);
        if (e != cudaSuccess) return e;
        if (p == 0)
            radix_scatter_kernel<true, true><<<grid, kSortThreads, kScatterSmemIds, s>>>(a);
        else
            radix_scatter_kernel<true, false><<<grid, kSortThreads, kScatterSmemIds, s>>>(a);
        note_launch();
        kin = a.keys_out;
        iin = a.ids_out;
    }
    *out_in_b = passes % 2 == 0;
    return cudaGetLastError();
}

cudaError_t radix_sort_keys_dev(uint64_t *keys_a, uint64_t *keys_b, const unsigned long long *d_count, uint64_t cap,
                                uint32_t bits, uint32_t *hist, uint32_t *partials, bool *out_in_b, cudaStream_t s)
{
    cudaError_t e0 = scatter_smem_init();
    if (e0 != cudaSuccess) return e0;
    const uint32_t tiles = (uint32_t)((cap + kSortTile - 1) / kSortTile);
    const uint32_t passes = (bits + 7) / 8;
    const uint64_t hcount = (uint64_t)256 * tiles;
    dim3 grid(tiles, 1);
    for (uint32_t p = 0; p < passes; ++p) {
        const bool from_b = (p % 2) == 1;
        const uint32_t nb = bits - 8 * p < 8 ? bits - 8 * p : 8;
        RadixArgs a{from_b ? keys_b : keys_a, nullptr, from_b ? keys_a : keys_b, nullptr, cap, d_count, tiles, 8 * p,
                    (1u << nb) - 1u, hist, 1};
        radix_hist_kernel<<<grid, kSortThreads, 0, s>>>(a);
        note_launch();
        cudaError_t e = scan_exclusive<uint32_t, uint32_t, uint32_t>(hist, hist, hcount, partials, false, s);
        if (e != cudaSuccess) return e;
        radix_scatter_kernel<false, false><<<grid, kSortThreads, kScatterSmemKeys, s>>>(a);
        note_launch();
    }
    *out_in_b = passes % 2 == 1;
    return cudaGetLastError();
}

cudaError_t launch_finalize_rows(const uint64_t *keys, const uint32_t *ids, uint32_t rows, uint64_t len,
                                 uint32_t slot_bits, uint64_t *ent, uint32_t *offs, cudaStream_t s)
{
    dim3 grid((unsigned)((len + 255) / 256), rows);
    finalize_kernel<<<grid, 256, 0, s>>>(keys, ids, len, slot_bits, ent, offs);
    note_launch();
    return cudaGetLastError();
}

cudaError_t scan_u32_to_u64(const uint32_t *in, uint64_t *out, uint64_t count, uint64_t *partials, cudaStream_t s)
{
    return scan_exclusive<uint32_t, uint64_t, uint64_t>(in, out, count, partials, true, s);
}

}  // namespace fclsh


namespace fclsh {

size_t segment_one_smem() { return (size_t)kOneCap * 8 + ((1u << kSubMaxBits) + (1u << kSubMaxBits) / 8 + 4) * 4; }

static uint32_t id_bits(uint64_t len)
{
    uint32_t b = 1;
    while ((1ULL << b) < len) ++b;
    return b;
}

bool msd_path_applies(uint32_t slot_bits, uint64_t n)
{
    // the packed entry holds sb - dbits <= 12 slot bits, 50 - sb key bits and the id
    return slot_bits >= 11 && slot_bits <= 23 && id_bits(n) <= slot_bits + 2;
}

// Partition digits: a segment always spans 2^12 = 4,096 directory slots (s = 13..23: 1..11 digit
// bits; 8-bit digits take partition_scatter_kernel, the others partition_wide_kernel).
uint32_t msd_dbits(uint32_t slot_bits) { return slot_bits - (uint32_t)kSubMaxBits; }

cudaError_t msd_partition_hist(const uint64_t *keys_in, uint32_t rows, uint64_t len, uint32_t sb, SortBuffers &buf,
                               cudaStream_t s)
{
    const uint32_t dbits = msd_dbits(sb);
    const uint32_t tiles = msd_tiles(len, dbits);
    const uint64_t hcount = ((uint64_t)rows << dbits) * tiles;
    RadixArgs a{keys_in, nullptr, buf.keys_a, nullptr, len, nullptr, tiles, sb - dbits, (1u << dbits) - 1, buf.hist,
                rows, sb, id_bits(len)};
    const dim3 grid(tiles, rows);
    switch (dbits) {
    case 1: wide_hist_kernel<1><<<grid, kWideThreads, 0, s>>>(a); break;
    case 2: wide_hist_kernel<2><<<grid, kWideThreads, 0, s>>>(a); break;
    case 3: wide_hist_kernel<3><<<grid, kWideThreads, 0, s>>>(a); break;
    case 4: wide_hist_kernel<4><<<grid, kWideThreads, 0, s>>>(a); break;
    case 5: wide_hist_kernel<5><<<grid, kWideThreads, 0, s>>>(a); break;
    case 6: wide_hist_kernel<6><<<grid, kWideThreads, 0, s>>>(a); break;
    case 7: wide_hist_kernel<7><<<grid, kWideThreads, 0, s>>>(a); break;
    case 8: radix_hist_kernel<<<grid, kSortThreads, 0, s>>>(a); break;
    case 9: wide_hist_kernel<9><<<grid, kWideThreads, 0, s>>>(a); break;
    case 10: wide_hist_kernel<10><<<grid, kWideThreads, 0, s>>>(a); break;
    case 11: wide_hist_kernel<11><<<grid, kWideThreads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    note_launch();
    return scan_exclusive<uint32_t, uint32_t, uint32_t>(buf.hist, buf.hist, hcount, buf.partials, false, s);
}

// Partition of every table by the slot's top msd_dbits(sb) bits, packed output: into
// places from the scanned histogram (cap = 0), or into bins of
// cap entries per (row, digit) (no histogram; buf.status bit 0 reports a full bin).
cudaError_t msd_partition_scatter(const uint64_t *keys_in, uint32_t rows, uint64_t len, uint32_t sb, uint32_t cap,
                                  uint32_t extra0, SortBuffers &buf, cudaStream_t s)
{
    cudaError_t e = scatter_smem_init();
    if (e != cudaSuccess) return e;
    const uint32_t dbits = msd_dbits(sb);
    const uint32_t tiles = msd_tiles(len, dbits);
    if (!cap) extra0 = 0;
    RadixArgs a{keys_in, nullptr, buf.keys_a, nullptr, len, nullptr, tiles, sb - dbits, (1u << dbits) - 1, buf.hist,
                rows, sb, id_bits(len), cap, extra0, buf.bin_cnt, buf.status};
    a.out_cap = (uint64_t)rows * (cap ? ((uint64_t)1 << dbits) * cap + extra0 : len);
    if (cap) {
        if ((e = cudaMemsetAsync(buf.bin_cnt, 0, ((size_t)rows << dbits) * 4, s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(buf.status, 0, 4, s)) != cudaSuccess) return e;
    }
    if (dbits == 8) {
        partition_scatter_kernel<<<dim3(tiles, rows), kSortThreads, kScatterSmemKeys, s>>>(a);
    } else {
        const dim3 grid(tiles, rows);
        constexpr size_t smem = (size_t)kWideSub * 12;
        static cudaError_t once = [] {   // static digit tables + dynamic sub-tile exceed 48 KB
            cudaError_t r = cudaSuccess;
            auto allow = [&](auto kern) {
                if (r == cudaSuccess) r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            };
            allow(partition_wide_kernel<1>);
            allow(partition_wide_kernel<2>);
            allow(partition_wide_kernel<3>);
            allow(partition_wide_kernel<4>);
            allow(partition_wide_kernel<5>);
            allow(partition_wide_kernel<6>);
            allow(partition_wide_kernel<7>);
            allow(partition_wide_kernel<9>);
            allow(partition_wide_kernel<10>);
            allow(partition_wide_kernel<11>);
            return r;
        }();
        if (once != cudaSuccess) return once;
        switch (dbits) {
        case 1: partition_wide_kernel<1><<<grid, kWideThreads, smem, s>>>(a); break;
        case 2: partition_wide_kernel<2><<<grid, kWideThreads, smem, s>>>(a); break;
        case 3: partition_wide_kernel<3><<<grid, kWideThreads, smem, s>>>(a); break;
        case 4: partition_wide_kernel<4><<<grid, kWideThreads, smem, s>>>(a); break;
        case 5: partition_wide_kernel<5><<<grid, kWideThreads, smem, s>>>(a); break;
        case 6: partition_wide_kernel<6><<<grid, kWideThreads, smem, s>>>(a); break;
        case 7: partition_wide_kernel<7><<<grid, kWideThreads, smem, s>>>(a); break;
        case 9: partition_wide_kernel<9><<<grid, kWideThreads, smem, s>>>(a); break;
        case 10: partition_wide_kernel<10><<<grid, kWideThreads, smem, s>>>(a); break;
        case 11: partition_wide_kernel<11><<<grid, kWideThreads, smem, s>>>(a); break;
        default: return cudaErrorInvalidValue;
        }
    }
    note_launch();
    return cudaGetLastError();
}

cudaError_t msd_finish(uint32_t rows, uint64_t len, uint32_t sb, uint32_t cap, uint32_t extra0, SortBuffers &buf,
                       unsigned long long *big_cnt, uint32_t *big, uint64_t *ent, uint32_t *offs, int sm_count,
                       cudaStream_t s)
{
    const uint32_t dbits = msd_dbits(sb);
    static cudaError_t once = [] {
        return cudaFuncSetAttribute(segment_one_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)segment_one_smem());
    }();
    if (once != cudaSuccess) return once;
    if (reinterpret_cast<uintptr_t>(offs) & 15) return cudaErrorMisalignedAddress;   // vector stores of offsets
    const uint32_t tiles = msd_tiles(len, dbits);
    const uint32_t idb = id_bits(len);
    if (!cap) extra0 = 0;
    const uint64_t in_stride = cap ? ((uint64_t)1 << dbits) * cap + extra0 : len;
    segment_bounds_kernel<<<rows, 256, 0, s>>>(buf.hist, tiles, len, cap ? buf.bin_cnt : nullptr, dbits, buf.seg_out);
    note_launch();
    cudaError_t e = cudaMemsetAsync(big_cnt, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    segment_one_kernel<<<dim3(1u << dbits, rows), kOneThreads, segment_one_smem(), s>>>(
        buf.keys_a, len, in_stride, cap, extra0, sb, idb, dbits, buf.seg_out, ent, offs, big_cnt, big);
    note_launch();
    segment_finish_kernel<<<3 * sm_count, kSegThreads, 0, s>>>(
        buf.keys_a, len, in_stride, cap, extra0, sb, idb, dbits, buf.seg_out, ent, offs, big_cnt, big);
    note_launch();
    return cudaGetLastError();
}

// Entries per bin of the histogram-free partition: the mean segment n/2^dbits plus
// eight standard deviations of its binomial count, an eighth of the mean for keys
// that repeat (a clustered data set puts tens of points on one key in every table;
// its fullest bins run ~10 standard deviations over the mean), and a margin.  Bins
// still overflow when a few keys carry a large share of a table (e.g. the empty sum
// of sparse points); those tables take the exact histogram path.
uint32_t msd_bin0_extra(uint64_t n) { return (uint32_t)((n / 16 + 3) & ~3ULL); }

uint32_t msd_bin_capacity(uint64_t n, uint32_t dbits)
{
    const double mean = (double)n / (double)(1u << dbits);
    const uint64_t c = (uint64_t)(mean + mean / 8.0 + 8.0 * sqrt(mean) + 64.0);
    return (uint32_t)((c + 3) & ~3ULL);
}

// ---------------------------------------------------------------- directory read-back

// The keys the build stored for sampled points (a diagnostic): every (table, slot) walks
// its run, and an entry whose id is sampled (slot_of_id[id] = its place in the sample, else
// ~0) writes its key, the stored high bits above the slot bits, to keys[table][place].
__global__ void __launch_bounds__(256) export_keys_kernel(const uint32_t *__restrict__ offs, uint64_t offs_stride,
                                                          const uint64_t *__restrict__ ent, uint64_t n, uint32_t T,
                                                          uint32_t sb, uint32_t ib,
                                                          const uint32_t *__restrict__ slot_of_id, uint64_t cnt,
                                                          uint64_t *__restrict__ keys)
{
    const uint64_t slots = 1ULL << sb, total = (uint64_t)T * slots;
    const uint64_t idmask = (1ULL << ib) - 1;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t tau = i >> sb, sl = i & (slots - 1);
        const uint32_t *O = offs + tau * offs_stride + sl;
        const uint32_t lo = O[0], hi = O[1];
        const uint64_t *row = ent + tau * n;
        for (uint32_t e = lo; e < hi && e < n; ++e) {
            const uint64_t en = row[e];
            const uint64_t id = en & idmask;
            if (id >= n) continue;
            const uint32_t j = slot_of_id[id];
            if (j != 0xFFFFFFFFu && j < cnt) keys[tau * cnt + j] = ((en >> ib) << sb) | sl;
        }
    }
}

cudaError_t launch_export_keys(const uint32_t *offs, uint64_t offs_stride, const uint64_t *ent, uint64_t n, uint32_t T,
                               uint32_t sb, uint32_t ib, const uint32_t *slot_of_id, uint64_t cnt, uint64_t *keys,
                               int sm_count, cudaStream_t s)
{
    export_keys_kernel<<<(unsigned)(sm_count * 8), 256, 0, s>>>(offs, offs_stride, ent, n, T, sb, ib, slot_of_id, cnt,
                                                                 keys);
    note_launch();
    return cudaGetLastError();
}

FCLSH_CHECK_READER(check_first_sort)

}  // namespace fclsh
