// Single-instance RASTER on one GB300: the contraction, agglomeration and
// labelling kernels, and the C ABI declared in include/raster.h.
//
// Pipeline (Alg. 1), one handle, one device-resident tile table:
//   contraction   k_part (exact integer projection of 16-byte loads, sort by
//                 table region), k_bucket (sort each region's keys by
//                 4096-slot bucket), k_insert_bucket (insert a bucket's keys
//                 into its copy in shared memory, write it back); small
//                 rounds into a live table use k_insert (global atomics).
//                 Alg. 1 first loop; chunked processing, Sect. 3.6.
//   agglomeration k_select (tiles with count >= tau, rows in their slots),
//                 k_hook (union-find over the forward half of
//                 neighbors(u, delta)), k_flatten_stats (root, size and
//                 smallest tile per component), k_emit (components of >= mu tiles:
//                 result rows and label codes).  Alg. 1 second loop, while
//                 loop, mu test.
//   per point     k_labels (RASTER*, Sect. 4.1) and the RASTER' groups
//                 (Sect. 3.4).
// The kernels live in raster_single_contract.cuh, raster_single_agglomerate.cuh
// and raster_single_labels.cuh; this file holds the host side.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <new>

#include <cuda_runtime.h>

#include "../../include/raster.h"
#include "raster_device.cuh"
#include "raster_host.h"
#include "raster_block.cuh"
#include "raster_region.cuh"

using namespace raster;

namespace {

constexpr int kBlock = 256;
// Table load: lookups (neighbour probes, labels) touch fewer sectors in a
// sparse table, which outweighs the larger clear and scan; measured best
// around 0.25-0.35 on the 500M-point workload.
constexpr double kMaxLoad = 0.5;      // grow after a round that leaves the table fuller than this
constexpr double kGrowLoad = 0.3;     // target load after growing
constexpr int kUnionLimit = 1 << 30;

// ---------------------------------------------------------------------------
// Kernels

#include "raster_single_contract.cuh"
#include "raster_single_agglomerate.cuh"
#include "raster_single_labels.cuh"

// ---------------------------------------------------------------------------
// Host side

std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_probe_limit{-1};
std::atomic<int> g_union_limit{-1};

}  // namespace

namespace raster {
void note_launch(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
TestLimits test_limits() { return TestLimits{g_probe_limit.load(), g_union_limit.load()}; }
}  // namespace raster

namespace {

int grid_for(const void* kernel, int block, size_t smem = 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
    return std::max(1, sms * std::max(1, per_sm));
}

}  // namespace

struct raster_handle {
    double precision = 0, scale = 0;
    unsigned int tau = 1, mu = 1;
    // neighbors(u, delta): forward offsets; `general` unless Chebyshev 1
    NbrSet nbr{};
    NbrSet* d_nbr = nullptr;  // device copy, read by the hook kernel
    bool general = false;
    bool groups = false;  // the 2 x 2 group rule of Sect. 3.6
    int dims = 2;         // coordinates per point: 2 or 3
    int probe_limit = -1;  // test bound of an insertion's probes (negative: the library's own)
    unsigned long long* d_sum = nullptr;  // scratch of raster_contract_tiles
    int union_limit = kUnionLimit;
    bool round_grew = false;  // the table was grown at the start of the current round
    // device copy of the points of raster_cluster_host (kept for the labels)
    double* res_xy = nullptr;
    size_t res_bytes = 0;
    ProjParams pp{};
    bool wide = false;
    cudaStream_t stream = nullptr;
    int status = RASTER_OK;  // sticky
    enum { kContracting, kAgglomerated } state = kContracting;

    Slot* tab = nullptr;
    unsigned long long cap = 0;  // regions << region_bits
    unsigned int regions = 1, region_bits = 12;
    long long d_bound = 0;       // upper bound on distinct tiles
    long long points = 0;        // points submitted (incl. invalid ones)

    // device counters: [0] tiles in the table (D), [1] significant (S),
    // [2] kept rows, [3] clusters, [4] export rows, [5] overflow entries,
    // [6] keys refused by a full bucket
    unsigned long long* d_ctr = nullptr;
    unsigned int* d_status = nullptr;
    unsigned long long* h_ctr = nullptr;  // pinned mirror: 8 counters, then the status word

    // agglomeration scratch and results (capacity in rows)
    long long agg_cap = 0;
    unsigned long long* sig_key = nullptr;
    unsigned int* sig_cnt = nullptr;
    unsigned int* sig_slot = nullptr;
    int* parent = nullptr;
    unsigned int* csize = nullptr;
    unsigned long long* cmin = nullptr;
    unsigned long long* out_key = nullptr;
    unsigned int* out_cnt = nullptr;
    unsigned long long* out_cid = nullptr;
    unsigned int* out_slot = nullptr;  // table slot of each result row
    raster_clusters result{};
    // RASTER' point groups: row of each point, per-row counters
    unsigned long long* point_rr = nullptr;  // (row << 32 | rank within the row) per point
    long long point_row_cap = 0;
    unsigned int* row_count = nullptr;
    long long* scan_sums = nullptr;
    long long row_count_cap = 0;

    // contraction staging: per-region key segments and cursors
    unsigned long long* stage_keys = nullptr;
    unsigned long long stage_cap = 0;  // keys
    unsigned int* cursor = nullptr;
    long long* item_start = nullptr;
    unsigned int cursor_cap = 0;       // regions
    unsigned long long* ovf_key = nullptr;
    unsigned int* ovf_cnt = nullptr;
    unsigned long long ovf_cap = 0;    // entries (one per point of a round)
    // per-bucket key segments of pass 1b and their cursors
    unsigned long long* stage2 = nullptr;
    unsigned long long stage2_cap = 0;  // keys
    unsigned int* bcursor = nullptr;
    unsigned long long bcursor_cap = 0; // buckets
    // the table's contents are void (after a reset): the next contraction
    // round starts its buckets empty instead of reading them
    bool fresh = false;
    // the significant tiles were selected while the last round wrote the
    // table (k_insert_fresh): rows in sig_key/sig_cnt/sig_slot, their count in
    // d_ctr[7], aux set; valid until the table changes again
    bool presel = false;

    unsigned long long* d_work = nullptr;  // work counters of the ordered kernels (8)

    // block index of the kept tiles for the labels (two coordinates): rebuilt
    // by the first labels call after each agglomeration
    int lidx_mode = 0;         // 0: when the tile table outgrows L2; 1: always; -1: never
    bool lidx_stale = true;
    bool lidx_on = false;
    unsigned long long* lidx = nullptr;   // 32-byte buckets of two entries
    unsigned long long lidx_alloc = 0;    // buckets
    unsigned long long lidx_buckets = 0;  // buckets in use: regions x share
    unsigned long long lidx_share = 0;
    unsigned int* lbitmap = nullptr;    // linear-counting bitmap
    unsigned long long lbitmap_words = 0;
    unsigned long long* d_lidx = nullptr;  // [0] zero bits of the bitmap, [1] build failure flag

    // host staging (contract_host / labels_host)
    cudaStream_t copy_stream = nullptr;
    double* stage_xy[2] = {nullptr, nullptr};
    long long* stage_lab[2] = {nullptr, nullptr};
    long long stage_points = 0;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};
    cudaEvent_t ev_done[2] = {nullptr, nullptr};
};

namespace {

int cuda_fail(raster_handle* h, cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        if (h) h->status = RASTER_E_OOM;
        return RASTER_E_OOM;
    }
    if (h) h->status = RASTER_E_CUDA;
    return RASTER_E_CUDA;
}

#define RCHECK(h, call)                                   \
    do {                                                  \
        cudaError_t _e = (call);                          \
        if (_e != cudaSuccess) return cuda_fail((h), _e); \
    } while (0)

bool hard_error(int s) { return s != RASTER_OK && s != RASTER_E_RANGE; }

int status_from_bits(unsigned int bits) {
    if (bits & kStInternal) return RASTER_E_INTERNAL;
    if (bits & kStFull) return RASTER_E_TABLE_FULL;
    if (bits & kStRange) return RASTER_E_RANGE;
    return RASTER_OK;
}

void merge_status(raster_handle* h, int s) {
    if (s == RASTER_OK) return;
    if (h->status == RASTER_OK || (h->status == RASTER_E_RANGE && s != RASTER_E_RANGE)) h->status = s;
}

unsigned int max_probe_for(unsigned long long cap) {
    return (unsigned int)std::min<unsigned long long>(cap, kBucketSlots);  // probing wraps within a bucket
}

// The probe bound of an insertion: `bound`, or a test's lower one.  Lookups
// always take the full bound, so a lowered limit can only make insertions
// fail (RASTER_E_TABLE_FULL), never hide a tile.
unsigned int insert_probe(const raster_handle* h, unsigned int bound) {
    return h->probe_limit >= 0 ? std::min<unsigned int>(bound, (unsigned int)h->probe_limit) : bound;
}

RegionTable table_of(const raster_handle* h) {
    RegionTable t;
    t.tab = h->tab;
    t.cap = h->cap;
    t.regions = h->regions;
    t.region_bits = h->region_bits;
    t.max_probe = max_probe_for(h->cap);
    t.dims = h->dims;
    return t;
}

constexpr unsigned int kRegionBits = 20;  // 1M slots (16 MiB) per region

// Table geometry for at least `need` slots: one power-of-two region up to
// 2^kRegionBits slots, otherwise a whole number of 2^kRegionBits-slot regions.
void geometry_for(double need, unsigned int* regions, unsigned int* bits) {
    if (need <= (double)(1ull << kRegionBits)) {
        unsigned int b = 12;
        while ((double)(1ull << b) < need) ++b;
        *regions = 1;
        *bits = b;
    } else {
        *regions = (unsigned int)std::ceil(need / (double)(1ull << kRegionBits));
        *bits = kRegionBits;
    }
}

int fill_table(raster_handle* h, Slot* tab, unsigned long long cap, cudaStream_t s) {
    static int grid = grid_for((const void*)k_fill_table, kBlock);
    k_fill_table<<<grid, kBlock, 0, s>>>(tab, cap);
    note_launch();
    RCHECK(h, cudaGetLastError());
    return RASTER_OK;
}

// Read the device counters and status into h_ctr (synchronises the stream).
int read_counters(raster_handle* h) {
    RCHECK(h, cudaMemcpyAsync(h->h_ctr, h->d_ctr, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
    h->h_ctr[8] = 0;
    RCHECK(h, cudaMemcpyAsync(h->h_ctr + 8, h->d_status, sizeof(unsigned int), cudaMemcpyDeviceToHost, h->stream));
    RCHECK(h, cudaStreamSynchronize(h->stream));
    merge_status(h, status_from_bits((unsigned int)h->h_ctr[8]));
    return RASTER_OK;
}

// Replace the table by one of `regions` x 2^bits slots, re-inserting every tile.
int grow_table(raster_handle* h, unsigned int regions, unsigned int bits) {
    // capacity is at most 2^32 slots, so at most 4096 regions: k_part keeps
    // region indices in 16 bits
    if (regions > 0xFFFFu) return RASTER_E_OOM;
    h->presel = false;  // slots move
    const unsigned long long new_cap = (unsigned long long)regions << bits;
    Slot* nt = nullptr;
    RCHECK(h, cudaMalloc(&nt, new_cap * sizeof(Slot)));
    int rc = fill_table(h, nt, new_cap, h->stream);
    if (rc) {
        cudaFree(nt);
        return rc;
    }
    RegionTable t;
    t.tab = nt;
    t.cap = new_cap;
    t.regions = regions;
    t.region_bits = bits;
    t.dims = h->dims;
    t.max_probe = insert_probe(h, max_probe_for(new_cap));
    if (h->tab && h->cap && !h->fresh) {
        static int grid = grid_for((const void*)k_rehash, kBlock);
        k_rehash<<<grid, kBlock, 0, h->stream>>>(h->tab, h->cap, t, h->d_status);
        note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            cudaFree(nt);
            return cuda_fail(h, e);
        }
    }
    RCHECK(h, cudaStreamSynchronize(h->stream));
    if (h->tab) cudaFree(h->tab);
    h->tab = nt;
    h->cap = new_cap;
    h->regions = regions;
    h->region_bits = bits;
    h->fresh = false;  // the new table is filled
    h->lidx_stale = true;  // its home buckets follow the regions
    if (h->state == raster_handle::kAgglomerated && h->result.n_tiles > 0) {
        // results are live (a reserve after the agglomeration): their slots
        // moved, and the rehash kept no label codes
        static int g_rst = grid_for((const void*)k_restore_rows, kBlock);
        const int lim = (int)std::max<long long>(1, (h->result.n_tiles + kBlock - 1) / kBlock);
        k_restore_rows<<<std::min(g_rst, lim), kBlock, 0, h->stream>>>(h->d_ctr + 2, h->out_key, h->out_cid,
                                                                      table_of(h), h->out_slot, h->d_status);
        note_launch();
        RCHECK(h, cudaGetLastError());
        RCHECK(h, cudaStreamSynchronize(h->stream));
    }
    return RASTER_OK;
}

// Make a void table (after a reset) readable: fill it with empty slots.
int ensure_clean(raster_handle* h) {
    if (!h->fresh) return RASTER_OK;
    int rc = fill_table(h, h->tab, h->cap, h->stream);
    if (rc) return rc;
    h->fresh = false;
    return RASTER_OK;
}

size_t part_smem(unsigned int regions) {
    return (size_t)kPartTile * (8 + 2) + (size_t)regions * 12;
}

int ensure_staging(raster_handle* h, long long n) {
    const unsigned long long seg = (unsigned long long)std::ceil((double)n / h->regions * 1.25) + 2 * kPartTile;
    const unsigned long long need = seg * h->regions;
    if (need > h->stage_cap) {
        RCHECK(h, cudaStreamSynchronize(h->stream));
        if (h->stage_keys) cudaFree(h->stage_keys);
        h->stage_keys = nullptr;
        h->stage_cap = 0;
        const unsigned long long cap = need + need / 8;
        RCHECK(h, cudaMalloc(&h->stage_keys, cap * sizeof(unsigned long long)));
        h->stage_cap = cap;
    }
    if ((unsigned long long)n > h->ovf_cap) {
        RCHECK(h, cudaStreamSynchronize(h->stream));
        if (h->ovf_key) cudaFree(h->ovf_key);
        if (h->ovf_cnt) cudaFree(h->ovf_cnt);
        h->ovf_key = nullptr;
        h->ovf_cnt = nullptr;
        h->ovf_cap = 0;
        RCHECK(h, cudaMalloc(&h->ovf_key, sizeof(unsigned long long) * (size_t)n));
        RCHECK(h, cudaMalloc(&h->ovf_cnt, sizeof(unsigned int) * (size_t)n));
        h->ovf_cap = (unsigned long long)n;
    }
    // pass 1b: per-bucket segments, 1.25x a bucket's share of a region segment
    const unsigned long long nb_region = 1ull << (h->region_bits - kBucketBits);
    const unsigned long long n_buckets = h->cap >> kBucketBits;
    const unsigned long long seg2 = ((seg + seg / 4) / nb_region + 64 + 1) & ~1ull;
    if (seg2 * n_buckets > h->stage2_cap) {
        RCHECK(h, cudaStreamSynchronize(h->stream));
        if (h->stage2) cudaFree(h->stage2);
        h->stage2 = nullptr;
        h->stage2_cap = 0;
        const unsigned long long cap = seg2 * n_buckets + (seg2 * n_buckets) / 8;
        RCHECK(h, cudaMalloc(&h->stage2, cap * sizeof(unsigned long long)));
        h->stage2_cap = cap;
    }
    if (n_buckets > h->bcursor_cap) {
        RCHECK(h, cudaStreamSynchronize(h->stream));
        if (h->bcursor) cudaFree(h->bcursor);
        h->bcursor = nullptr;
        h->bcursor_cap = 0;
        RCHECK(h, cudaMalloc(&h->bcursor, sizeof(unsigned int) * n_buckets));
        h->bcursor_cap = n_buckets;
    }
    if (h->regions > h->cursor_cap) {
        RCHECK(h, cudaStreamSynchronize(h->stream));
        if (h->cursor) cudaFree(h->cursor);
        if (h->item_start) cudaFree(h->item_start);
        h->cursor = nullptr;
        h->item_start = nullptr;
        h->cursor_cap = 0;
        RCHECK(h, cudaMalloc(&h->cursor, sizeof(unsigned int) * h->regions));
        RCHECK(h, cudaMalloc(&h->item_start, sizeof(long long) * (h->regions + 1)));
        h->cursor_cap = h->regions;
    }
    return RASTER_OK;
}

constexpr long long kRoundPoints = 1ll << 30;    // points per contraction round
constexpr long long kClusterChunk = 16ll << 20;  // points per copy of raster_cluster_host
constexpr double kNewLimit = 0.8;                // no new tiles beyond this load within a round
constexpr unsigned int kInsertProbe = 1024;      // global insert: longer probe sequences go to the overflow list
constexpr double kBucketRound = 0.25;            // rounds of fewer points per table slot insert globally
constexpr double kRefitRatio = 1.5;              // a grown table this much larger than needed is rebuilt
constexpr double kPreGrow = 4.0;                 // grow before a round whose estimate is this far past kMaxLoad
constexpr bool kLabelsQueued = true;             // labels with the block index: k_labels_idx (queued fallbacks)
constexpr bool kInsertSplit = true;              // pass 2 into a void table: split key/count buckets (k_insert_fresh)
constexpr bool kPreSelect = true;                // k_insert_fresh selects the significant tiles as it writes

// One contraction round of n points: pass 1, item prefix, pass 1b, pass 2
// (all asynchronous), then one synchronisation to read the table's tile count
// and the overflow counts.  If keys overflowed or the table is too full, grow
// it and re-insert the overflow list.  Pass 1 may run chunk by chunk (as host
// copies arrive): round_begin, round_part for each chunk, round_finish.
int round_begin(raster_handle* h, long long n) {
    // A round far larger than the table (the first call into the initial
    // table, say) grows it first: a full bucket would pass its remaining keys
    // to the overflow list one block at a time.  D + n/2 estimates the tiles
    // after the round; a table that turns out far too large is rebuilt
    // smaller in round_finish.
    int rc;
    h->round_grew = false;
    h->presel = false;  // this round changes counts; round_finish may select again
    const double est = (double)h->d_bound + 0.5 * (double)n;
    if (est > kPreGrow * kMaxLoad * (double)h->cap) {
        unsigned int regions, bits;
        geometry_for(est / kGrowLoad, &regions, &bits);
        if (((unsigned long long)regions << bits) <= (1ull << 32)) {
            rc = grow_table(h, regions, bits);
            if (rc) return rc;
            h->round_grew = true;
        }
    }
    rc = ensure_staging(h, n);
    if (rc) return rc;
    RCHECK(h, cudaMemsetAsync(h->cursor, 0, sizeof(unsigned int) * h->regions, h->stream));
    RCHECK(h, cudaMemsetAsync(h->d_ctr + 5, 0, sizeof(unsigned long long), h->stream));
    return RASTER_OK;
}

// Pass 1 over m points of the round (appends to the staging segments).
template <bool WIDE>
int round_part(raster_handle* h, const double* xy, long long m, unsigned long long* keys_out = nullptr) {
    if (m <= 0) return RASTER_OK;
    const unsigned long long seg = (h->stage_cap / h->regions) & ~1ull;  // even: 16-byte aligned item starts
    RegionTable t = table_of(h);
    const size_t smem = part_smem(h->regions);
    const void* part = h->dims == 3 ? (const void*)k_part<WIDE, 3> : (const void*)k_part<WIDE, 2>;
    static bool attr_set[2] = {false, false};
    if (!attr_set[h->dims - 2]) {
        RCHECK(h, cudaFuncSetAttribute(part, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr_set[h->dims - 2] = true;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, part, kBlock, smem);
    const long long tiles = (m + kPartTile - 1) / kPartTile;
    const int g1 = (int)std::max<long long>(1, std::min<long long>((long long)sms * std::max(per_sm, 1), tiles));
    if (h->dims == 3)
        k_part<WIDE, 3><<<g1, kBlock, smem, h->stream>>>(xy, m, h->pp, t, h->stage_keys, seg, h->cursor, h->ovf_key,
                                                         h->ovf_cnt, h->d_ctr + 5, h->d_status, keys_out);
    else
        k_part<WIDE, 2><<<g1, kBlock, smem, h->stream>>>(xy, m, h->pp, t, h->stage_keys, seg, h->cursor, h->ovf_key,
                                                         h->ovf_cnt, h->d_ctr + 5, h->d_status, keys_out);
    note_launch();
    RCHECK(h, cudaGetLastError());
    return RASTER_OK;
}

int round_finish(raster_handle* h, long long n) {
    int rc;
    const bool grew_before = h->round_grew;
    bool presel_tried = false;
    const unsigned long long seg = (h->stage_cap / h->regions) & ~1ull;  // even: 16-byte aligned item starts
    RegionTable t = table_of(h);
    k_region_items<<<1, kBlock, 0, h->stream>>>(h->cursor, (int)h->regions, seg, h->item_start);
    // pass 2: whole buckets in shared memory, unless the round is much smaller
    // than the table (and the table is live), where rewriting every bucket
    // would cost more than inserting with global atomics
    const bool by_bucket = h->fresh || (double)n >= kBucketRound * (double)h->cap;
    RCHECK(h, cudaMemsetAsync(h->d_ctr + 6, 0, sizeof(unsigned long long), h->stream));
    if (!by_bucket) {
        static int g2 = grid_for((const void*)k_insert, kBlock);
        RegionTable ti = t;
        ti.max_probe = insert_probe(h, std::min<unsigned int>(t.max_probe, kInsertProbe));
        RCHECK(h, cudaMemsetAsync(h->d_work, 0, sizeof(unsigned long long), h->stream));
        k_insert<<<g2, kBlock, 0, h->stream>>>(ti, h->stage_keys, seg, h->cursor, h->item_start, (int)h->regions,
                                              (unsigned long long)((double)h->cap * kNewLimit), h->d_ctr,
                                              h->ovf_key, h->ovf_cnt, h->d_ctr + 5, h->d_work);
        note_launch(2);
        RCHECK(h, cudaGetLastError());
    } else {
        // pass 1b: by bucket within each region
        const unsigned long long n_buckets = h->cap >> kBucketBits;
        const unsigned long long seg2 = (h->stage2_cap / n_buckets) & ~1ull;
        RCHECK(h, cudaMemsetAsync(h->bcursor, 0, sizeof(unsigned int) * n_buckets, h->stream));
        RCHECK(h, cudaMemsetAsync(h->d_work, 0, 2 * sizeof(unsigned long long), h->stream));
        static bool bkattr = false;
        if (!bkattr) {
            RCHECK(h, cudaFuncSetAttribute(k_bucket, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBucketSmem));
            bkattr = true;
        }
        static int gb = grid_for((const void*)k_bucket, kBlock, kBucketSmem);
        // pass 2: bucket by bucket in shared memory
        const size_t bsmem = sizeof(Slot) * kBucketSlots;
        static bool battr = false;
        if (!battr) {
            RCHECK(h, cudaFuncSetAttribute(k_insert_bucket<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)bsmem));
            RCHECK(h, cudaFuncSetAttribute(k_insert_bucket<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)bsmem));
            battr = true;
        }
        static int gi = grid_for((const void*)k_insert_bucket<false>, kInsBlock, bsmem);
        const unsigned int probe = insert_probe(h, kBucketProbe);
        auto ins = probe < kBucketProbe ? k_insert_bucket<true> : k_insert_bucket<false>;
        const size_t fsmem = (sizeof(unsigned long long) + sizeof(unsigned int)) * kBucketSlots;
        static bool fattr = false;
        if (kInsertSplit && !fattr) {
            RCHECK(h, cudaFuncSetAttribute(k_insert_fresh<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)fsmem));
            RCHECK(h, cudaFuncSetAttribute(k_insert_fresh<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)fsmem));
            fattr = true;
        }
        static int gf = kInsertSplit ? grid_for((const void*)k_insert_fresh<false>, kInsBlock, fsmem) : 0;
        auto ins_fresh = probe < kBucketProbe ? k_insert_fresh<true> : k_insert_fresh<false>;
        k_bucket<<<gb, kBlock, kBucketSmem, h->stream>>>(t, h->stage_keys, seg, h->cursor, h->item_start, (int)h->regions,
                                                         h->stage2, seg2, h->bcursor, h->ovf_key, h->ovf_cnt,
                                                         h->d_ctr + 5, h->d_work);
        // the selection of significant tiles rides along when the rows have
        // room (the 2 x 2 group rule marks tiles first, so it selects later)
        presel_tried = kInsertSplit && h->fresh && kPreSelect && !h->groups && h->agg_cap > 0;
        PreSelect sel{0u, nullptr, nullptr, nullptr, nullptr, 0ull};
        if (presel_tried) {
            RCHECK(h, cudaMemsetAsync(h->d_ctr + 7, 0, sizeof(unsigned long long), h->stream));
            sel = PreSelect{h->tau, h->sig_key, h->sig_cnt, h->sig_slot, h->d_ctr + 7,
                            (unsigned long long)h->agg_cap};
        }
        if (kInsertSplit && h->fresh)
            ins_fresh<<<(int)std::min<unsigned long long>((unsigned long long)gf, n_buckets), kInsBlock, fsmem,
                        h->stream>>>(h->tab, n_buckets, h->stage2, seg2, h->bcursor,
                                     (unsigned int)(kNewLimit * kBucketSlots), probe, h->d_ctr, h->d_ctr + 6,
                                     h->ovf_key, h->ovf_cnt, h->d_ctr + 5, h->d_work + 1, sel);
        else
            ins<<<(int)std::min<unsigned long long>((unsigned long long)gi, n_buckets), kInsBlock, bsmem, h->stream>>>(
                h->tab, n_buckets, h->stage2, seg2, h->bcursor, h->fresh ? 1 : 0,
                (unsigned int)(kNewLimit * kBucketSlots), probe, h->d_ctr, h->d_ctr + 6, h->ovf_key, h->ovf_cnt,
                h->d_ctr + 5, h->d_work + 1);
        h->fresh = false;  // every bucket has been written
        note_launch(3);
        RCHECK(h, cudaGetLastError());
    }
    rc = read_counters(h);
    if (rc) return rc;
    const unsigned long long D = h->h_ctr[0], ovf = h->h_ctr[5], full = h->h_ctr[6];
    // the selection holds only if no count or slot changes after it: no
    // overflow to re-insert, no growth before or after, every row written
    const bool presel_ok = presel_tried && !grew_before && ovf == 0 && h->h_ctr[7] <= (unsigned long long)h->agg_cap;
    // D + ovf bounds the tile count; a bucket that refused new tiles needs room too
    bool grew = grew_before;
    if ((double)(D + ovf) > kMaxLoad * (double)h->cap || full > 0) {
        const double need = std::max((double)(D + ovf) / kGrowLoad, 1.5 * (double)h->cap);
        unsigned int regions, bits;
        geometry_for(need, &regions, &bits);
        if (((unsigned long long)regions << bits) > (1ull << 32)) return RASTER_E_OOM;
        rc = grow_table(h, regions, bits);
        if (rc) return rc;
        grew = true;
    }
    if (ovf > 0) {
        static int g3 = grid_for((const void*)k_reinsert, kBlock);
        RegionTable tr = table_of(h);
        tr.max_probe = insert_probe(h, tr.max_probe);
        k_reinsert<<<g3, kBlock, 0, h->stream>>>(tr, h->ovf_key, h->ovf_cnt, ovf, h->d_ctr, h->d_status);
        note_launch();
        RCHECK(h, cudaGetLastError());
        rc = read_counters(h);
        if (rc) return rc;
    }
    // the growth estimates counted overflowed points, or half the round's
    // points, as new tiles: rebuild a grown table that ended up far larger
    // than the tiles need (a table the caller reserved is left alone)
    const double fit = (double)h->h_ctr[0] / kGrowLoad;
    if (grew && (double)h->cap > kRefitRatio * fit && (double)h->cap > (double)(1ull << 20)) {
        unsigned int regions, bits;
        geometry_for(fit, &regions, &bits);
        rc = grow_table(h, regions, bits);
        if (rc) return rc;
    }
    h->d_bound = (long long)h->h_ctr[0];
    h->presel = presel_ok && !grew;
    return RASTER_OK;
}

template <bool WIDE>
int contract_round(raster_handle* h, const double* xy, long long n, unsigned long long* keys_out) {
    int rc = round_begin(h, n);
    if (rc) return rc;
    rc = round_part<WIDE>(h, xy, n, keys_out);
    if (rc) return rc;
    return round_finish(h, n);
}

// keys_out (optional): every point's tile key, in point order
int contract_device(raster_handle* h, const double* xy, long long n, unsigned long long* keys_out = nullptr) {
    for (long long off = 0; off < n; off += kRoundPoints) {
        const long long m = std::min(n - off, kRoundPoints);
        const double* p = xy + (long long)h->dims * off;
        unsigned long long* k = keys_out ? keys_out + off : nullptr;
        const int rc = h->wide ? contract_round<true>(h, p, m, k) : contract_round<false>(h, p, m, k);
        if (rc) return rc;
    }
    return RASTER_OK;
}

int ensure_agg_capacity(raster_handle* h, long long rows) {
    if (rows <= h->agg_cap) return RASTER_OK;
    const long long cap = std::max<long long>(rows + rows / 4, 1 << 16);
    void** bufs[] = {(void**)&h->sig_key, (void**)&h->sig_cnt, (void**)&h->sig_slot, (void**)&h->parent,
                     (void**)&h->csize,   (void**)&h->cmin,    (void**)&h->out_key,  (void**)&h->out_cnt,
                     (void**)&h->out_cid, (void**)&h->out_slot};
    const size_t sizes[] = {8, 4, 4, 4, 4, 8, 8, 4, 8, 4};
    RCHECK(h, cudaStreamSynchronize(h->stream));
    for (int i = 0; i < 10; ++i) {
        if (*bufs[i]) cudaFree(*bufs[i]);
        *bufs[i] = nullptr;
    }
    h->agg_cap = 0;
    for (int i = 0; i < 10; ++i) RCHECK(h, cudaMalloc(bufs[i], (size_t)cap * sizes[i]));
    h->agg_cap = cap;
    return RASTER_OK;
}

int ensure_stage(raster_handle* h) {
    if (h->stage_points) return RASTER_OK;
    const long long pts = 64ll << 20;  // 64M points = 1 GiB of xy per buffer
    RCHECK(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
        RCHECK(h, cudaMalloc(&h->stage_xy[b], (size_t)pts * 8 * h->dims));
        RCHECK(h, cudaMalloc(&h->stage_lab[b], (size_t)pts * 8));
        RCHECK(h, cudaEventCreateWithFlags(&h->ev_copied[b], cudaEventDisableTiming));
        RCHECK(h, cudaEventCreateWithFlags(&h->ev_done[b], cudaEventDisableTiming));
    }
    h->stage_points = pts;
    return RASTER_OK;
}

constexpr double kLidxMinTableBytes = 64.0 * (1 << 20);  // a smaller tile table stays in L2 by itself

// Build the block index of the kept tiles (raster_single_labels.cuh) for the
// labels, once per agglomeration: estimate the number of blocks by linear
// counting (one synchronisation), size the index for kLidxLoad, insert.  An
// index that would not be much smaller than the tile table, or that finds no
// memory, is left out: the labels then read the table.
int ensure_label_index(raster_handle* h) {
    if (!h->lidx_stale) return RASTER_OK;
    h->lidx_stale = false;
    h->lidx_on = false;
    const long long K = h->result.n_tiles;
    if (h->dims != 2 || h->lidx_mode < 0 || K <= 0) return RASTER_OK;
    const double table_bytes = (double)h->cap * sizeof(Slot);
    if (h->lidx_mode == 0 && table_bytes <= kLidxMinTableBytes) return RASTER_OK;
    int lb = 10;  // bitmap of 2^lb bits, at least 8 per kept tile up to 32 MiB
    while (lb < 28 && (1ull << lb) < 8ull * (unsigned long long)K) ++lb;
    const unsigned long long words = (1ull << lb) >> 5;
    if (words > h->lbitmap_words) {
        if (h->lbitmap) cudaFree(h->lbitmap);
        h->lbitmap = nullptr;
        h->lbitmap_words = 0;
        if (cudaMalloc(&h->lbitmap, words * 4) != cudaSuccess) {
            cudaGetLastError();
            h->lbitmap = nullptr;
            return RASTER_OK;
        }
        h->lbitmap_words = words;
    }
    if (!h->d_lidx) RCHECK(h, cudaMalloc(&h->d_lidx, 2 * sizeof(unsigned long long)));
    cudaStream_t s = h->stream;
    RCHECK(h, cudaMemsetAsync(h->lbitmap, 0, words * 4, s));
    RCHECK(h, cudaMemsetAsync(h->d_lidx, 0, 2 * sizeof(unsigned long long), s));
    static int g_cnt = grid_for((const void*)k_lidx_count, kBlock);
    static int g_zer = grid_for((const void*)k_lidx_zeros, kBlock);
    static int g_bld = grid_for((const void*)k_lidx_build, kBlock);
    const int lim = (int)std::max<long long>(1, (K + kBlock - 1) / kBlock);
    k_lidx_count<<<std::min(g_cnt, lim), kBlock, 0, s>>>(h->d_ctr + 2, h->out_key, h->lbitmap, lb);
    k_lidx_zeros<<<(int)std::min<unsigned long long>(g_zer, (words + kBlock - 1) / kBlock), kBlock, 0, s>>>(
        h->lbitmap, words, h->d_lidx);
    note_launch(2);
    RCHECK(h, cudaGetLastError());
    unsigned long long zeros = 0;
    RCHECK(h, cudaMemcpyAsync(&zeros, h->d_lidx, sizeof(zeros), cudaMemcpyDeviceToHost, s));
    RCHECK(h, cudaStreamSynchronize(s));
    const double M = (double)(1ull << lb);
    double blocks = zeros > 0 ? -M * std::log((double)zeros / M) : (double)K;
    blocks = std::min(blocks * 1.02 + 16.0, (double)K);
    const unsigned long long share = (unsigned long long)std::ceil(blocks / kLidxLoad / 2.0 / h->regions) + 1;
    const unsigned long long buckets = share * h->regions;
    if (h->lidx_mode == 0 && (double)buckets * 32.0 > 0.5 * table_bytes) return RASTER_OK;
    if (buckets > h->lidx_alloc) {
        if (h->lidx) cudaFree(h->lidx);
        h->lidx = nullptr;
        h->lidx_alloc = 0;
        if (cudaMalloc(&h->lidx, buckets * 32) != cudaSuccess) {  // 256-byte aligned
            cudaGetLastError();
            h->lidx = nullptr;
            return RASTER_OK;
        }
        h->lidx_alloc = buckets;
    }
    RCHECK(h, cudaMemsetAsync(h->lidx, 0, buckets * 32, s));
    k_lidx_build<<<std::min(g_bld, lim), kBlock, 0, s>>>(h->d_ctr + 2, h->out_key, h->out_cid, table_of(h),
                                                         h->lidx, buckets, share,
                                                         reinterpret_cast<unsigned int*>(h->d_lidx + 1));
    note_launch();
    RCHECK(h, cudaGetLastError());
    h->lidx_buckets = buckets;
    h->lidx_share = share;
    h->lidx_on = true;
    return RASTER_OK;
}

// Labels of n points given by their coordinates (xy), or (KEYS) by the tile
// keys that contraction stored for them.
template <bool WIDE, int DIMS, bool KEYS = false>
void launch_labels(raster_handle* h, const double* xy, long long n, int64_t* labels,
                   const unsigned long long* keys = nullptr) {
    static int grid = grid_for((const void*)k_labels<WIDE, DIMS, KEYS>, kBlock);
    LabelIndex li{nullptr, 0, 0, nullptr};
    if (DIMS == 2 && h->lidx_on)
        li = LabelIndex{h->lidx, h->lidx_buckets, h->lidx_share, reinterpret_cast<unsigned int*>(h->d_lidx + 1)};
    if (DIMS == 2 && h->lidx_on && kLabelsQueued) {
        static int gq = grid_for((const void*)k_labels_idx<WIDE, KEYS>, kBlock);
        k_labels_idx<WIDE, KEYS><<<(int)std::min<long long>(gq, (n + kBlock - 1) / kBlock), kBlock, 0, h->stream>>>(
            xy, keys, n, h->pp, table_of(h), reinterpret_cast<const long long*>(h->out_cid),
            reinterpret_cast<long long*>(labels), h->d_status, li);
        return;
    }
    k_labels<WIDE, DIMS, KEYS><<<(int)std::min<long long>(grid, (n + kBlock - 1) / kBlock), kBlock, 0, h->stream>>>(
        xy, keys, n, h->pp, table_of(h), h->tau, reinterpret_cast<const long long*>(h->out_cid),
        reinterpret_cast<long long*>(labels), h->d_status, li);
}

template <bool WIDE, int DIMS>
void launch_group_count(raster_handle* h, const double* xy, long long n) {
    static int grid = grid_for((const void*)k_group_count<WIDE, DIMS>, kBlock);
    k_group_count<WIDE, DIMS><<<(int)std::min<long long>(grid, (n + kBlock - 1) / kBlock), kBlock, 0, h->stream>>>(
        xy, n, h->pp, table_of(h), h->tau, h->row_count, h->point_rr, h->d_status);
}

bool misaligned(const void* p, int dims = 2) { return ((uintptr_t)p & (dims == 3 ? 7u : 15u)) != 0; }

}  // namespace

// ---------------------------------------------------------------------------
// Shared with the batched and serving code.
namespace raster {

int make_proj_params(double scale, ProjParams* pp, bool* wide) {
    if (!(scale > 0.0) || !std::isfinite(scale) || !std::isnormal(scale)) return RASTER_E_ARG;
    uint64_t b;
    std::memcpy(&b, &scale, 8);
    const int e = (int)((b >> 52) & 0x7FF);
    uint64_t m = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    int tz = 0;
    while (!(m & 1ull)) {
        m >>= 1;
        ++tz;
    }
    int bits = 0;
    while ((m >> bits) != 0ull) ++bits;
    pp->s_odd = m;
    pp->s_exp = e - 1075 + tz;
    pp->s_bits = bits;
    pp->d0 = 1075 - pp->s_exp;
    pp->top = 52 + bits;
    pp->scale = scale;
    pp->half_lo = bits >= 2 ? 1ull << (bits - 2) : 0ull;  // P of top bits: rounding at bit bits-1
    pp->half_hi = 1ull << (bits - 1);                    // P of top+1 bits: rounding at bit bits
    pp->thr = bits <= 10 ? 1ull << pp->top : 0ull;
    pp->dmax = pp->top + 1021;
    *wide = bits > 10;
    return RASTER_OK;
}

double scale_of_precision(double precision) {
    static const double exact[] = {1e0,  1e1,  1e2,  1e3,  1e4,  1e5,  1e6,  1e7,  1e8,  1e9,  1e10, 1e11,
                                   1e12, 1e13, 1e14, 1e15, 1e16, 1e17, 1e18, 1e19, 1e20, 1e21, 1e22};
    if (precision == std::floor(precision) && precision >= 0.0 && precision <= 22.0) return exact[(int)precision];
    return std::pow(10.0, precision);
}

}  // namespace raster

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

const char* raster_strerror(int status) {
    switch (status) {
        case RASTER_OK: return "ok";
        case RASTER_E_ARG: return "invalid argument";
        case RASTER_E_RANGE: return "coordinate not finite or tile index out of int32 range";
        case RASTER_E_OOM: return "out of memory";
        case RASTER_E_TABLE_FULL: return "tile table full (bounded probe exhausted)";
        case RASTER_E_CUDA: return "CUDA runtime error";
        case RASTER_E_INTERNAL: return "bounded device iteration did not converge";
        case RASTER_E_STATE: return "call not valid in the handle's current state";
        case RASTER_E_LIMIT: return "input larger than the fixed capacity of this entry point";
        default: return "unknown status";
    }
}

int raster_create(double precision, uint32_t tau, uint32_t mu, raster_handle** out) {
    raster_params p;
    p.precision = precision;
    p.tau = tau;
    p.mu = mu;
    p.metric = RASTER_CHEBYSHEV;
    p.delta = 1;
    p.groups = 0;
    p.dims = 2;
    return raster_create_ex(&p, out);
}

int raster_create_ex(const raster_params* params, raster_handle** out) {
    if (!out || !params) return RASTER_E_ARG;
    const double precision = params->precision;
    const uint32_t tau = params->tau, mu = params->mu;
    if (tau == 0 || mu == 0 || !std::isfinite(precision)) return RASTER_E_ARG;
    if (params->metric != RASTER_CHEBYSHEV && params->metric != RASTER_MANHATTAN) return RASTER_E_ARG;
    if (params->delta < 1 || params->delta > RASTER_MAX_DELTA || params->groups > 1) return RASTER_E_ARG;
    const int dims = params->dims == 0 ? 2 : (int)params->dims;
    if (dims != 2 && dims != 3) return RASTER_E_ARG;
    if (dims == 3 && params->groups) return RASTER_E_ARG;  // the group rule is defined for 2 x 2 tiles
    *out = nullptr;
    raster_handle* h = new (std::nothrow) raster_handle();
    if (!h) return RASTER_E_OOM;
    h->precision = precision;
    h->scale = scale_of_precision(precision);
    h->tau = tau;
    h->mu = mu;
    h->groups = params->groups != 0;
    h->dims = dims;
    {
        const TestLimits lim = test_limits();
        h->probe_limit = lim.probe;
        if (lim.unions >= 0) h->union_limit = lim.unions;
    }
    if (const char* m = std::getenv("RASTER_LABEL_INDEX")) h->lidx_mode = m[0] == '0' ? -1 : m[0] == '1' ? 1 : 0;
    h->general = dims == 3 || !(params->metric == RASTER_CHEBYSHEV && params->delta == 1);
    {
        // forward half of the ball: the first nonzero offset is positive
        const int d = (int)params->delta, dz_max = dims == 3 ? d : 0;
        int n = 0;
        for (int dx = 0; dx <= d; ++dx)
            for (int dy = -d; dy <= d; ++dy)
                for (int dz = -dz_max; dz <= dz_max; ++dz) {
                    if (dx == 0 && (dy < 0 || (dy == 0 && dz <= 0))) continue;
                    if (params->metric == RASTER_MANHATTAN && dx + std::abs(dy) + std::abs(dz) > d) continue;
                    if (n == kMaxFwd) {
                        delete h;
                        return RASTER_E_ARG;  // neighbourhood larger than the kernels take
                    }
                    h->nbr.dx[n] = (signed char)dx;
                    h->nbr.dy[n] = (signed char)dy;
                    h->nbr.dz[n] = (signed char)dz;
                    ++n;
                }
        h->nbr.n = n;
        h->nbr.dims = dims;
    }
    if (make_proj_params(h->scale, &h->pp, &h->wide) != RASTER_OK) {
        delete h;
        return RASTER_E_ARG;
    }
    cudaError_t e = cudaMalloc(&h->d_ctr, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_work, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_status, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMallocHost(&h->h_ctr, 9 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(h->d_ctr, 0, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_nbr, sizeof(NbrSet));
    if (e == cudaSuccess) e = cudaMemcpy(h->d_nbr, &h->nbr, sizeof(NbrSet), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        raster_destroy(h);
        return e == cudaErrorMemoryAllocation ? RASTER_E_OOM : RASTER_E_CUDA;
    }
    int rc = grow_table(h, 1, 16);
    if (rc) {
        raster_destroy(h);
        return rc;
    }
    *out = h;
    return RASTER_OK;
}

int raster_reserve(raster_handle* h, int64_t n_tiles) {
    if (!h || n_tiles < 0) return RASTER_E_ARG;
    if (hard_error(h->status)) return h->status;
    int rc = read_counters(h);
    if (rc) return rc;
    h->d_bound = (long long)h->h_ctr[0];
    const double need = (double)std::max<long long>(n_tiles, h->d_bound) / kGrowLoad;
    if (need <= (double)h->cap) return RASTER_OK;
    unsigned int regions, bits;
    geometry_for(need, &regions, &bits);
    if (((unsigned long long)regions << bits) > (1ull << 32)) return RASTER_E_OOM;
    return grow_table(h, regions, bits);
}

int raster_contract_tiles(raster_handle* h, const int64_t* key, const uint32_t* count, int64_t n, void* stream) {
    if (!h || n < 0 || (n > 0 && (!key || !count || ((uintptr_t)key & 7u) || ((uintptr_t)count & 3u))))
        return RASTER_E_ARG;
    if (hard_error(h->status)) return h->status;
    h->stream = (cudaStream_t)stream;
    if (n == 0) return RASTER_OK;
    // the points these tiles stand for, against the 32-bit count limit
    if (!h->d_sum) RCHECK(h, cudaMalloc(&h->d_sum, sizeof(unsigned long long)));
    RCHECK(h, cudaMemsetAsync(h->d_sum, 0, sizeof(unsigned long long), h->stream));
    const int gs = (int)std::min<long long>(1024, (n + kBlock - 1) / kBlock);
    k_sum_counts<<<gs, kBlock, 0, h->stream>>>(count, n, h->d_sum);
    note_launch();
    unsigned long long points = 0;
    RCHECK(h, cudaMemcpyAsync(&points, h->d_sum, sizeof(points), cudaMemcpyDeviceToHost, h->stream));
    RCHECK(h, cudaStreamSynchronize(h->stream));
    if ((unsigned long long)h->points + points > 0xFFFFFFFFull) return RASTER_E_ARG;
    // room for every key as a new tile at the growth load, then one pass of inserts
    int rc = raster_reserve(h, (int64_t)std::min<unsigned long long>((unsigned long long)h->d_bound + (unsigned long long)n,
                                                                     0x7FFFFFFFull));
    if (rc) return rc;
    rc = ensure_clean(h);
    if (rc) return rc;
    h->state = raster_handle::kContracting;
    h->presel = false;  // counts change
    h->points += (long long)points;
    RegionTable t = table_of(h);
    t.max_probe = insert_probe(h, t.max_probe);
    static int g_add = grid_for((const void*)k_add_tiles, kBlock);
    k_add_tiles<<<(int)std::min<long long>(g_add, (n + kBlock - 1) / kBlock), kBlock, 0, h->stream>>>(
        t, reinterpret_cast<const unsigned long long*>(key), count, n, h->d_ctr, h->d_status);
    note_launch();
    RCHECK(h, cudaGetLastError());
    rc = read_counters(h);
    if (rc) return rc;
    h->d_bound = (long long)h->h_ctr[0];
    return RASTER_OK;
}

int raster_contract(raster_handle* h, const double* xy, int64_t n, void* stream) {
    if (!h || n < 0 || (n > 0 && (!xy || misaligned(xy, h->dims)))) return RASTER_E_ARG;
    if (hard_error(h->status)) return h->status;
    if (h->points + n > 0xFFFFFFFFll) return RASTER_E_ARG;  // per-tile counts are 32-bit
    h->stream = (cudaStream_t)stream;
    h->state = raster_handle::kContracting;
    h->points += n;
    if (n == 0) return RASTER_OK;
    return contract_device(h, xy, n);
}

int raster_contract_keys(raster_handle* h, const double* xy, int64_t n, int64_t* keys, void* stream) {
    if (!h || n < 0 || (n > 0 && (!xy || !keys || misaligned(xy, h->dims) || ((uintptr_t)keys & 7u))))
        return RASTER_E_ARG;
    if (hard_error(h->status)) return h->status;
    if (h->points + n > 0xFFFFFFFFll) return RASTER_E_ARG;  // per-tile counts are 32-bit
    h->stream = (cudaStream_t)stream;
    h->state = raster_handle::kContracting;
    h->points += n;
    if (n == 0) return RASTER_OK;
    return contract_device(h, xy, n, reinterpret_cast<unsigned long long*>(keys));
}

int raster_contract_host(raster_handle* h, const double* xy_host, int64_t n, void* stream) {
    if (!h || n < 0 || (n > 0 && !xy_host)) return RASTER_E_ARG;
    if (hard_error(h->status)) return h->status;
    if (h->points + n > 0xFFFFFFFFll) return RASTER_E_ARG;
    h->stream = (cudaStream_t)stream;
    h->state = raster_handle::kContracting;
    if (n == 0) return RASTER_OK;
    int rc = ensure_stage(h);
    if (rc) return rc;
    h->points += n;
    RCHECK(h, cudaEventRecord(h->ev_done[0], h->stream));
    RCHECK(h, cudaEventRecord(h->ev_done[1], h->stream));
    const long long nchunks = (n + h->stage_points - 1) / h->stage_points;
    auto issue_copy = [&](long long c) -> int {
        const int b = (int)(c & 1);
        const long long off = c * h->stage_points;
        const long long m = std::min(n - off, h->stage_points);
        RCHECK(h, cudaStreamWaitEvent(h->copy_stream, h->ev_done[b], 0));
        RCHECK(h, cudaMemcpyAsync(h->stage_xy[b], xy_host + (long long)h->dims * off, (size_t)m * 8 * h->dims,
                                  cudaMemcpyHostToDevice,
                                  h->copy_stream));
        RCHECK(h, cudaEventRecord(h->ev_copied[b], h->copy_stream));
        return RASTER_OK;
    };
    rc = issue_copy(0);
    if (rc) return rc;
    for (long long c = 0; c < nchunks; ++c) {
        const int b = (int)(c & 1);
        const long long m = std::min(n - c * h->stage_points, h->stage_points);
        RCHECK(h, cudaStreamWaitEvent(h->stream, h->ev_copied[b], 0));
        if (c + 1 < nchunks) {  // the next copy overlaps this chunk's contraction
            rc = issue_copy(c + 1);
            if (rc) return rc;
        }
        rc = contract_device(h, h->stage_xy[b], m);
        if (rc) return rc;
        RCHECK(h, cudaEventRecord(h->ev_done[b], h->stream));
    }
    RCHECK(h, cudaStreamSynchronize(h->stream));
    return RASTER_OK;
}

int raster_agglomerate(raster_handle* h, raster_clusters* out) {
    if (!h || !out) return RASTER_E_ARG;
    if (hard_error(h->status)) return h->status;
    int rc = read_counters(h);
    if (rc) return rc;
    if (hard_error(h->status)) return h->status;
    const long long D = (long long)h->h_ctr[0];
    h->d_bound = D;
    if (D >= 0x7FFFFFFFll) return RASTER_E_OOM;
    rc = ensure_clean(h);
    if (rc) return rc;
    // the significant tiles selected during contraction, unless the row
    // buffers are about to be replaced by larger ones
    const bool presel = h->presel && !h->groups && std::max<long long>(D, 1) <= h->agg_cap;
    h->presel = false;  // the aux fields are rewritten below
    rc = ensure_agg_capacity(h, std::max<long long>(D, 1));
    if (rc) return rc;
    cudaStream_t s = h->stream;
    RCHECK(h, cudaMemsetAsync(h->d_ctr + 1, 0, 4 * sizeof(unsigned long long), s));
    unsigned long long* d_nsig = h->d_ctr + 1;
    static int g_sel = grid_for((const void*)k_select, kBlock);
    if (h->groups) {  // Sect. 3.6: mark tiles of 2 x 2 groups holding >= tau points
        static int g_grp = grid_for((const void*)k_groups, kBlock);
        RCHECK(h, cudaMemsetAsync(h->d_work + 6, 0, sizeof(unsigned long long), s));
        k_groups<<<g_grp, kBlock, 0, s>>>(h->tab, table_of(h), h->tau, h->d_work + 6);
        note_launch();
    }
    if (presel) {
        RCHECK(h, cudaMemcpyAsync(d_nsig, h->d_ctr + 7, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
    } else {
        RCHECK(h, cudaMemsetAsync(h->d_work + 3, 0, sizeof(unsigned long long), s));
        k_select<<<g_sel, kBlock, 0, s>>>(h->tab, h->cap, h->tau, h->sig_key, h->sig_cnt, h->sig_slot, d_nsig,
                                          (unsigned long long)h->agg_cap, 1, h->groups ? 1 : 0, h->d_work + 3);
        note_launch();
    }
    k_clamp_rows<<<1, 1, 0, s>>>(d_nsig, (unsigned long long)h->agg_cap, h->d_status);
    note_launch();
    RCHECK(h, cudaGetLastError());
    static int g_init = grid_for((const void*)k_uf_init, kBlock);
    static int g_hook = grid_for((const void*)k_hook<false>, kBlock);
    static int g_flat = grid_for((const void*)k_flatten_stats, kBlock);
    static int g_emit = grid_for((const void*)k_emit, kBlock);
    const int lim = (int)std::max<long long>(1, (D + kBlock - 1) / kBlock);
    k_uf_init<<<std::min(g_init, lim), kBlock, 0, s>>>(d_nsig, h->parent, h->csize, h->cmin);
    RCHECK(h, cudaMemsetAsync(h->d_work, 0, 8 * sizeof(unsigned long long), s));
    const long long F = h->general ? h->nbr.n : 1;  // threads per significant tile
    if (h->general)
        k_hook<true><<<std::min<long long>(g_hook, F * lim), kBlock, 0, s>>>(d_nsig, h->sig_key, table_of(h), h->d_nbr,
                                                                           h->nbr.n, h->dims, h->parent,
                                                                           h->union_limit, h->d_work + 1,
                                                                           h->d_status);
    else
        k_hook<false><<<std::min<long long>(g_hook, F * lim), kBlock, 0, s>>>(d_nsig, h->sig_key, table_of(h), h->d_nbr,
                                                                            4, 2, h->parent, h->union_limit,
                                                                            h->d_work + 1, h->d_status);
    const unsigned long long order_xor = h->dims == 3 ? kOrderXor3 : kOrderXor2;
    k_flatten_stats<<<std::min(g_flat, lim), kBlock, 0, s>>>(d_nsig, h->parent, h->sig_key, h->csize, h->cmin,
                                                             h->d_work + 2, order_xor);
    k_emit<<<std::min(g_emit, lim), kBlock, 0, s>>>(d_nsig, h->sig_key, h->sig_cnt, h->sig_slot, h->parent, h->csize,
                                                    h->cmin, h->mu, h->tab, h->out_key, h->out_cnt, h->out_cid,
                                                    h->out_slot, h->d_ctr + 2, h->d_ctr + 3, h->d_work + 4, order_xor,
                                                    h->dims);
    note_launch(4);
    RCHECK(h, cudaGetLastError());
    rc = read_counters(h);
    if (rc) return rc;
    h->result.key = reinterpret_cast<const int64_t*>(h->out_key);
    h->result.count = h->out_cnt;
    h->result.cid = reinterpret_cast<const int64_t*>(h->out_cid);
    h->result.n_tiles = (int64_t)h->h_ctr[2];
    h->result.n_clusters = (int64_t)h->h_ctr[3];
    h->result.n_distinct = D;
    h->result.n_significant = (int64_t)h->h_ctr[1];
    h->result.n_points = (int64_t)h->points;
    *out = h->result;
    if (hard_error(h->status)) return h->status;
    h->state = raster_handle::kAgglomerated;
    h->lidx_stale = true;
    return h->status;
}

int raster_point_labels(raster_handle* h, const double* xy, int64_t n, int64_t* labels, void* stream) {
    if (!h || n < 0 || (n > 0 && (!xy || !labels || misaligned(xy, h->dims)))) return RASTER_E_ARG;
    if (hard_error(h->status)) return h->status;
    if (h->state != raster_handle::kAgglomerated) return RASTER_E_STATE;
    h->stream = (cudaStream_t)stream;
    if (n == 0) return RASTER_OK;
    const int rc = ensure_label_index(h);
    if (rc) return rc;
    if (h->dims == 3)
        h->wide ? launch_labels<true, 3>(h, xy, n, labels) : launch_labels<false, 3>(h, xy, n, labels);
    else
        h->wide ? launch_labels<true, 2>(h, xy, n, labels) : launch_labels<false, 2>(h, xy, n, labels);
    note_launch();
    RCHECK(h, cudaGetLastError());
    return RASTER_OK;
}

int raster_key_labels(raster_handle* h, const int64_t* keys, int64_t n, int64_t* labels, void* stream) {
    if (!h || n < 0 || (n > 0 && (!keys || !labels || ((uintptr_t)keys & 7u) || ((uintptr_t)labels & 7u))))
        return RASTER_E_ARG;
    if (hard_error(h->status)) return h->status;
    if (h->state != raster_handle::kAgglomerated) return RASTER_E_STATE;
    h->stream = (cudaStream_t)stream;
    if (n == 0) return RASTER_OK;
    const int rc = ensure_label_index(h);
    if (rc) return rc;
    const unsigned long long* k = reinterpret_cast<const unsigned long long*>(keys);
    if (h->dims == 3)
        launch_labels<false, 3, true>(h, nullptr, n, labels, k);
    else
        launch_labels<false, 2, true>(h, nullptr, n, labels, k);
    note_launch();
    RCHECK(h, cudaGetLastError());
    return RASTER_OK;
}

int raster_point_labels_host(raster_handle* h, const double* xy_host, int64_t n, int64_t* labels_host,
                             void* stream) {
    if (!h || n < 0 || (n > 0 && (!xy_host || !labels_host))) return RASTER_E_ARG;
    if (hard_error(h->status)) return h->status;
    if (h->state != raster_handle::kAgglomerated) return RASTER_E_STATE;
    h->stream = (cudaStream_t)stream;
    if (n == 0) return RASTER_OK;
    int rc = ensure_stage(h);
    if (rc) return rc;
    RCHECK(h, cudaEventRecord(h->ev_done[0], h->stream));
    RCHECK(h, cudaEventRecord(h->ev_done[1], h->stream));
    long long off = 0;
    for (int c = 0; off < n; ++c) {
        const int b = c & 1;
        const long long m = std::min(n - off, h->stage_points);
        RCHECK(h, cudaStreamWaitEvent(h->copy_stream, h->ev_done[b], 0));
        RCHECK(h, cudaMemcpyAsync(h->stage_xy[b], xy_host + (long long)h->dims * off, (size_t)m * 8 * h->dims,
                                  cudaMemcpyHostToDevice,
                                  h->copy_stream));
        RCHECK(h, cudaEventRecord(h->ev_copied[b], h->copy_stream));
        RCHECK(h, cudaStreamWaitEvent(h->stream, h->ev_copied[b], 0));
        rc = raster_point_labels(h, h->stage_xy[b], m, reinterpret_cast<int64_t*>(h->stage_lab[b]), stream);
        if (rc) return rc;
        RCHECK(h, cudaMemcpyAsync(labels_host + off, h->stage_lab[b], (size_t)m * 8, cudaMemcpyDeviceToHost,
                                  h->stream));
        RCHECK(h, cudaEventRecord(h->ev_done[b], h->stream));
        off += m;
    }
    RCHECK(h, cudaStreamSynchronize(h->stream));
    return RASTER_OK;
}

int raster_point_groups(raster_handle* h, const double* xy, int64_t n, int64_t* row_start, int64_t* point_index,
                        int64_t capacity, int64_t* n_grouped, void* stream) {
    if (!h || n < 0 || !n_grouped || !row_start || capacity < 0 || (n > 0 && (!xy || misaligned(xy, h->dims))))
        return RASTER_E_ARG;
    if (hard_error(h->status)) return h->status;
    if (h->state != raster_handle::kAgglomerated) return RASTER_E_STATE;
    if (n > 0xFFFFFFFFll) return RASTER_E_LIMIT;  // per-row counters are 32-bit
    h->stream = (cudaStream_t)stream;
    cudaStream_t s = h->stream;
    const long long K = h->result.n_tiles;
    // scratch: (row, rank) per point, a counter per result row
    if (n > h->point_row_cap) {
        RCHECK(h, cudaStreamSynchronize(s));
        if (h->point_rr) cudaFree(h->point_rr);
        h->point_rr = nullptr;
        h->point_row_cap = 0;
        RCHECK(h, cudaMalloc(&h->point_rr, sizeof(unsigned long long) * (size_t)std::max<long long>(n, 1)));
        h->point_row_cap = std::max<long long>(n, 1);
    }
    if (K + 1 > h->row_count_cap) {
        RCHECK(h, cudaStreamSynchronize(s));
        if (h->row_count) cudaFree(h->row_count);
        if (h->scan_sums) cudaFree(h->scan_sums);
        h->row_count = nullptr;
        h->scan_sums = nullptr;
        h->row_count_cap = 0;
        const long long cap = K + 1;
        RCHECK(h, cudaMalloc(&h->row_count, sizeof(unsigned int) * (size_t)cap));
        RCHECK(h, cudaMalloc(&h->scan_sums, sizeof(long long) * (size_t)(cap / kScanTile + 2)));
        h->row_count_cap = cap;
    }
    const unsigned long long* d_nkept = h->d_ctr + 2;
    static int g = grid_for((const void*)k_aux_rows, kBlock);
    const int gk = (int)std::max<long long>(1, std::min<long long>(g, (K + kBlock - 1) / kBlock));
    RCHECK(h, cudaMemsetAsync(h->row_count, 0, sizeof(unsigned int) * (size_t)(K + 1), s));
    k_aux_rows<<<gk, kBlock, 0, s>>>(d_nkept, h->out_slot, h->tab);
    if (n > 0) {
        if (h->dims == 3)
            h->wide ? launch_group_count<true, 3>(h, xy, n) : launch_group_count<false, 3>(h, xy, n);
        else
            h->wide ? launch_group_count<true, 2>(h, xy, n) : launch_group_count<false, 2>(h, xy, n);
    }
    const int gs = (int)std::max<long long>(1, std::min<long long>(1024, (K + kScanTile - 1) / kScanTile));
    long long* rs = reinterpret_cast<long long*>(row_start);
    k_scan_tiles<<<gs, kBlock, 0, s>>>(d_nkept, h->row_count, rs, h->scan_sums);
    k_scan_sums<<<1, kBlock, 0, s>>>(d_nkept, h->scan_sums, rs);
    k_scan_add<<<gk, kBlock, 0, s>>>(d_nkept, h->scan_sums, rs);
    k_aux_codes<<<gk, kBlock, 0, s>>>(d_nkept, h->out_slot, h->out_key, h->out_cid, h->tab, h->dims);
    note_launch(n > 0 ? 6 : 5);
    RCHECK(h, cudaGetLastError());
    long long m = 0;
    RCHECK(h, cudaMemcpyAsync(&m, row_start + K, sizeof(long long), cudaMemcpyDeviceToHost, s));
    RCHECK(h, cudaStreamSynchronize(s));
    *n_grouped = m;
    if (m > capacity || (m > 0 && !point_index)) return RASTER_E_ARG;
    if (m > 0) {
        static int g2 = grid_for((const void*)k_group_scatter, kBlock);
        k_group_scatter<<<(int)std::min<long long>(g2, (n + kBlock - 1) / kBlock), kBlock, 0, s>>>(
            n, h->point_rr, rs, reinterpret_cast<long long*>(point_index));
        note_launch();
        RCHECK(h, cudaGetLastError());
    }
    return RASTER_OK;
}

int raster_export_tiles(raster_handle* h, int64_t* key, uint32_t* count, int64_t capacity, int64_t* n_out) {
    if (!h || !n_out || capacity < 0) return RASTER_E_ARG;
    if (hard_error(h->status)) return h->status;
    int rc = read_counters(h);
    if (rc) return rc;
    const long long D = (long long)h->h_ctr[0];
    *n_out = D;
    if (capacity < D || (D > 0 && (!key || !count))) return RASTER_E_ARG;
    rc = ensure_clean(h);
    if (rc) return rc;
    RCHECK(h, cudaMemsetAsync(h->d_ctr + 4, 0, sizeof(unsigned long long), h->stream));
    static int g_sel = grid_for((const void*)k_select, kBlock);
    k_select<<<g_sel, kBlock, 0, h->stream>>>(h->tab, h->cap, 1u, reinterpret_cast<unsigned long long*>(key), count,
                                              nullptr, h->d_ctr + 4, (unsigned long long)capacity, 0, 0);
    note_launch();
    RCHECK(h, cudaGetLastError());
    rc = read_counters(h);
    if (rc) return rc;
    if ((long long)h->h_ctr[4] != D) {  // rows beyond the capacity were not written
        merge_status(h, RASTER_E_INTERNAL);
        return RASTER_E_INTERNAL;
    }
    return RASTER_OK;
}

int raster_cluster_host(raster_handle* h, const double* xy_host, int64_t n, int64_t* labels_host,
                        raster_clusters* out, void* stream) {
    if (!h || !out || n < 0 || (n > 0 && (!xy_host || !labels_host))) return RASTER_E_ARG;
    if (hard_error(h->status)) return h->status;
    if (h->points + n > 0xFFFFFFFFll) return RASTER_E_ARG;
    h->stream = (cudaStream_t)stream;
    h->state = raster_handle::kContracting;
    int rc = ensure_stage(h);
    if (rc) return rc;
    const size_t bytes = (size_t)n * 8 * (size_t)h->dims;
    if (bytes > h->res_bytes) {
        RCHECK(h, cudaStreamSynchronize(h->stream));
        if (h->res_xy) cudaFree(h->res_xy);
        h->res_xy = nullptr;
        h->res_bytes = 0;
        if (cudaMalloc(&h->res_xy, bytes) != cudaSuccess) {
            // no room to keep the points: copy them twice instead
            cudaGetLastError();
            h->res_xy = nullptr;
            rc = raster_contract_host(h, xy_host, n, stream);
            if (rc) return rc;
            rc = raster_agglomerate(h, out);
            if (hard_error(rc)) return rc;
            const int rl = raster_point_labels_host(h, xy_host, n, labels_host, stream);
            return rl ? rl : rc;
        }
        h->res_bytes = bytes;
    }
    h->points += n;
    // contraction: rounds of at most kRoundPoints; within a round, pass 1 runs
    // on each chunk as soon as its copy has landed, while later copies proceed
    const int dims = h->dims;
    for (long long r0 = 0; r0 < n; r0 += kRoundPoints) {
        const long long mr = std::min(n - r0, kRoundPoints);
        rc = round_begin(h, mr);
        if (rc) return rc;
        for (long long c0 = 0, c = 0; c0 < mr; c0 += kClusterChunk, ++c) {
            const int b = (int)(c & 1);
            const long long m = std::min(mr - c0, kClusterChunk);
            const long long off = (r0 + c0) * dims;
            RCHECK(h, cudaMemcpyAsync(h->res_xy + off, xy_host + off, (size_t)m * 8 * dims, cudaMemcpyHostToDevice,
                                      h->copy_stream));
            RCHECK(h, cudaEventRecord(h->ev_copied[b], h->copy_stream));
            RCHECK(h, cudaStreamWaitEvent(h->stream, h->ev_copied[b], 0));
            rc = h->wide ? round_part<true>(h, h->res_xy + off, m) : round_part<false>(h, h->res_xy + off, m);
            if (rc) return rc;
        }
        rc = round_finish(h, mr);
        if (rc) return rc;
    }
    rc = raster_agglomerate(h, out);
    if (hard_error(rc)) return rc;
    // labels of the resident points, copied back chunk by chunk behind the kernels
    RCHECK(h, cudaEventRecord(h->ev_done[0], h->copy_stream));
    RCHECK(h, cudaEventRecord(h->ev_done[1], h->copy_stream));
    for (long long c0 = 0, c = 0; c0 < n; c0 += kClusterChunk, ++c) {
        const int b = (int)(c & 1);
        const long long m = std::min(n - c0, kClusterChunk);
        RCHECK(h, cudaStreamWaitEvent(h->stream, h->ev_done[b], 0));  // the buffer's previous copy is done
        const int rl = raster_point_labels(h, h->res_xy + c0 * dims, m, reinterpret_cast<int64_t*>(h->stage_lab[b]),
                                           stream);
        if (rl) return rl;
        RCHECK(h, cudaEventRecord(h->ev_copied[b], h->stream));
        RCHECK(h, cudaStreamWaitEvent(h->copy_stream, h->ev_copied[b], 0));
        RCHECK(h, cudaMemcpyAsync(labels_host + c0, h->stage_lab[b], (size_t)m * 8, cudaMemcpyDeviceToHost,
                                  h->copy_stream));
        RCHECK(h, cudaEventRecord(h->ev_done[b], h->copy_stream));
    }
    RCHECK(h, cudaStreamSynchronize(h->copy_stream));
    RCHECK(h, cudaStreamSynchronize(h->stream));
    return rc;
}

int raster_table_stats(raster_handle* h, raster_table_stats_t* out) {
    if (!h || !out) return RASTER_E_ARG;
    if (hard_error(h->status)) return h->status;
    int rc = ensure_clean(h);
    if (rc) return rc;
    unsigned long long* d = h->d_work + 5;  // three counters, free outside the kernels that use them
    RCHECK(h, cudaMemsetAsync(d, 0, 3 * sizeof(unsigned long long), h->stream));
    static int grid = grid_for((const void*)k_probe_stats, kBlock);
    k_probe_stats<<<grid, kBlock, 0, h->stream>>>(h->tab, table_of(h), d);
    note_launch();
    RCHECK(h, cudaGetLastError());
    unsigned long long v[3];
    RCHECK(h, cudaMemcpyAsync(v, d, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
    RCHECK(h, cudaStreamSynchronize(h->stream));
    out->capacity = (int64_t)h->cap;
    out->occupied = (int64_t)v[0];
    out->probe_sum = (int64_t)v[1];
    out->probe_max = (int64_t)v[2];
    return RASTER_OK;
}

int raster_reset(raster_handle* h, void* stream) {
    if (!h) return RASTER_E_ARG;
    h->stream = (cudaStream_t)stream;
    if (h->status == RASTER_E_CUDA) {
        // a failed CUDA call may have left the context unusable; try anyway
        cudaGetLastError();
    }
    // the table's contents become void; the next contraction round writes
    // every bucket, and any other reader fills the table first
    h->fresh = true;
    h->presel = false;
    RCHECK(h, cudaMemsetAsync(h->d_ctr, 0, 8 * sizeof(unsigned long long), h->stream));
    RCHECK(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned int), h->stream));
    h->d_bound = 0;
    h->points = 0;
    h->status = RASTER_OK;
    h->state = raster_handle::kContracting;
    return RASTER_OK;
}

int raster_status(raster_handle* h) {
    if (!h) return RASTER_E_ARG;
    int rc = read_counters(h);
    if (rc) return rc;
    return h->status;
}

double raster_get_scale(const raster_handle* h) { return h ? h->scale : 0.0; }

int64_t raster_table_capacity(const raster_handle* h) { return h ? (int64_t)h->cap : 0; }

uint64_t raster_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int raster_set_test_limits(int32_t probe_limit, int32_t union_limit) {
    g_probe_limit.store(probe_limit < 0 ? -1 : probe_limit);
    g_union_limit.store(union_limit < 0 ? -1 : union_limit);
    return RASTER_OK;
}

int raster_destroy(raster_handle* h) {
    if (!h) return RASTER_E_ARG;
    if (h->stream) cudaStreamSynchronize(h->stream);
    void* bufs[] = {h->tab,    h->d_ctr,   h->d_status, h->sig_key, h->sig_cnt, h->sig_slot, h->parent,
                    h->csize,  h->cmin,    h->out_key,  h->out_cnt, h->out_cid, h->stage_xy[0], h->stage_xy[1],
                    h->stage_lab[0], h->stage_lab[1], h->stage_keys, h->cursor, h->item_start, h->ovf_key,
                    h->ovf_cnt, h->d_work, h->out_slot, h->point_rr, h->row_count, h->scan_sums,
                    h->stage2,  h->bcursor, h->d_nbr, h->res_xy, h->lidx, h->lbitmap, h->d_lidx, h->d_sum};
    for (void* p : bufs)
        if (p) cudaFree(p);
    if (h->h_ctr) cudaFreeHost(h->h_ctr);
    for (int b = 0; b < 2; ++b) {
        if (h->ev_copied[b]) cudaEventDestroy(h->ev_copied[b]);
        if (h->ev_done[b]) cudaEventDestroy(h->ev_done[b]);
    }
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    delete h;
    return RASTER_OK;
}

}  // extern "C"
