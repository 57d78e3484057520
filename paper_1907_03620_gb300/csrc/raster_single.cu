// Single-instance RASTER on one GB300: the contraction, agglomeration and
// labelling kernels, and the C ABI declared in include/raster.h.
//
// Pipeline (Alg. 1):
//   k_contract  -- 16-byte coalesced loads of (x, y), exact integer
//                  projection, warp pre-aggregation of equal tiles with
//                  __match_any_sync, insertion into the resident tile table
//                  (Alg. 1 first loop; chunked, Sect. 3.6).
//   k_select    -- block-scan compaction of tiles with count >= tau
//                  (Alg. 1 second loop); records each significant tile's
//                  index in its slot.
//   k_hook      -- each significant tile probes its 4 forward neighbours
//                  (adjacency at Chebyshev distance 1 is symmetric, so every
//                  one of the 8 neighbour pairs is seen once) and unites
//                  components (Alg. 1 while loop, as union-find).
//   k_flatten   -- every tile points at its root.
//   k_stats     -- component size and smallest (ix, iy) per root.
//   k_emit      -- keep components of >= mu tiles (Alg. 1 mu test), write
//                  (key, count, cluster id) rows and each kept tile's label
//                  code.
//   k_labels    -- second projection pass giving per-point labels (RASTER*,
//                  Sect. 4.1).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
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
constexpr int kContractUnroll = 4;
// Table load: lookups (neighbour probes, labels) touch fewer sectors in a
// sparse table, which outweighs the larger clear and scan; measured best
// around 0.25-0.35 on the 500M-point workload.
constexpr double kMaxLoad = 0.5;      // grow after a round that leaves the table fuller than this
constexpr double kGrowLoad = 0.3;     // target load after growing
constexpr int kUnionLimit = 1 << 30;

// ---------------------------------------------------------------------------
// Block helpers

// ---------------------------------------------------------------------------
// Kernels

__global__ void k_fill_table(Slot* tab, unsigned long long cap) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    ulonglong2 v;
    v.x = kEmptyKey;
    v.y = (unsigned long long)kAuxNone << 32;  // count 0, aux none
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += stride)
        reinterpret_cast<ulonglong2*>(tab)[i] = v;
}

// Pass 1 of contraction: project a tile of kPartTile points (keys stay in
// registers), counting-sort the keys by table region in shared memory (with
// each key's region beside it, as a 16-bit index), reserve space in each region's
// staging segment with one atomic per (tile, region), and append the keys in
// coalesced runs.  Keys beyond a segment's capacity (a region far above its
// share) go to the overflow list.
constexpr int kPartTile = 2048;
constexpr int kPartPer = kPartTile / kBlock;
constexpr long long kInsertItem = 2048;

template <int BLOCK = kBlock>
__device__ __forceinline__ unsigned int block_excl_scan_bins(unsigned int* bins, int nbins, unsigned int* start,
                                                             unsigned int* scratch) {
    // each thread owns a contiguous run of bins
    const int per = (nbins + BLOCK - 1) / BLOCK;
    const int b0 = threadIdx.x * per;
    unsigned int sum = 0;
    for (int b = b0; b < min(b0 + per, nbins); ++b) sum += bins[b];
    unsigned int total;
    unsigned int off = block_excl_scan<BLOCK>(sum, scratch, &total);
    for (int b = b0; b < min(b0 + per, nbins); ++b) {
        start[b] = off;
        off += bins[b];
    }
    __syncthreads();
    return total;
}

// Append (key, c) to the overflow list (warp-aggregated); the list has room
// for every key of a round, so it cannot overflow itself.
__device__ __forceinline__ void overflow_append(bool want, unsigned long long key, unsigned int c,
                                                unsigned long long* ovf_key, unsigned int* ovf_cnt,
                                                unsigned long long* ovf_n) {
    const unsigned int m = __ballot_sync(__activemask(), want);
    if (!want) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(ovf_n, (unsigned long long)__popc(m));
    base = __shfl_sync(m, base, leader);
    const unsigned long long pos = base + __popc(m & ((1u << lane) - 1u));
    ovf_key[pos] = key;
    ovf_cnt[pos] = c;
}

// Point i of an array of DIMS coordinates per point (two: one 16-byte load),
// and its tile key, or kInvalidKey.
template <int DIMS>
struct PointIn {
    double c[DIMS];
};
template <int DIMS>
__device__ __forceinline__ PointIn<DIMS> load_point(const double* __restrict__ xy, long long i) {
    PointIn<DIMS> p;
    if (DIMS == 2) {
        const double2 v = __ldcs(reinterpret_cast<const double2*>(xy) + i);
        p.c[0] = v.x;
        p.c[1] = v.y;
    } else {
#pragma unroll
        for (int a = 0; a < DIMS; ++a) p.c[a] = __ldcs(xy + DIMS * i + a);
    }
    return p;
}
template <bool WIDE, int DIMS>
__device__ __forceinline__ unsigned long long project_in(const PointIn<DIMS>& p, const ProjParams& pp) {
    if (DIMS == 2) return project_point<WIDE>(p.c[0], p.c[1], pp);
    return project_point3<WIDE>(p.c[0], p.c[1], p.c[DIMS - 1], pp);
}

template <bool WIDE, int DIMS>
__global__ void __launch_bounds__(kBlock, 4) k_part(const double* __restrict__ xy, long long n, ProjParams pp,
                                                RegionTable t, unsigned long long* __restrict__ stage,
                                                unsigned long long seg_cap, unsigned int* __restrict__ cursor,
                                                unsigned long long* ovf_key, unsigned int* ovf_cnt,
                                                unsigned long long* ovf_n, unsigned int* d_status) {
    extern __shared__ unsigned char smem[];
    unsigned long long* s_sorted = reinterpret_cast<unsigned long long*>(smem);         // kPartTile keys
    unsigned int* s_fill = reinterpret_cast<unsigned int*>(s_sorted + kPartTile);       // regions
    unsigned int* s_start = s_fill + t.regions;                                         // regions
    unsigned int* s_gbase = s_start + t.regions;                                        // regions
    unsigned short* s_reg = reinterpret_cast<unsigned short*>(s_gbase + t.regions);     // kPartTile regions
    __shared__ unsigned int scratch[33];
    const int R = (int)t.regions;
    unsigned int st = 0;
    for (long long t0 = (long long)blockIdx.x * kPartTile; t0 < n; t0 += (long long)gridDim.x * kPartTile) {
        for (int r = threadIdx.x; r < R; r += kBlock) s_fill[r] = 0u;
        __syncthreads();
        // two coordinates: all of the thread's loads in flight before projecting;
        // three: loaded where projected (registers)
        PointIn<DIMS> p[DIMS == 2 ? kPartPer : 1];
        if (DIMS == 2) {
#pragma unroll
            for (int k = 0; k < kPartPer; ++k) {
                const long long idx = t0 + k * kBlock + threadIdx.x;
                if (idx < n) p[DIMS == 2 ? k : 0] = load_point<DIMS>(xy, idx);
            }
        }
        unsigned long long key[kPartPer];
        unsigned int meta[kPartPer];
#pragma unroll
        for (int k = 0; k < kPartPer; ++k) {
            const long long idx = t0 + k * kBlock + threadIdx.x;
            meta[k] = 0xFFFFFFFFu;
            key[k] = 0ull;
            if (idx < n) {
                key[k] = project_in<WIDE, DIMS>(DIMS == 2 ? p[DIMS == 2 ? k : 0] : load_point<DIMS>(xy, idx), pp);
                if (key[k] == kInvalidKey) {
                    st |= kStRange;
                } else {
                    const unsigned int r = region_of(key[k], t);
                    meta[k] = (r << 12) | atomicAdd(&s_fill[r], 1u);
                }
            }
        }
        __syncthreads();
        const unsigned int total = block_excl_scan_bins(s_fill, R, s_start, scratch);
        for (int r = threadIdx.x; r < R; r += kBlock)
            if (s_fill[r]) s_gbase[r] = atomicAdd(&cursor[r], s_fill[r]);
#pragma unroll
        for (int k = 0; k < kPartPer; ++k) {
            if (meta[k] != 0xFFFFFFFFu) {
                const unsigned int r = meta[k] >> 12;
                const unsigned int pos = s_start[r] + (meta[k] & 0xFFFu);
                s_sorted[pos] = key[k];
                s_reg[pos] = (unsigned short)r;
            }
        }
        __syncthreads();
        for (unsigned int j0 = 0; j0 < total; j0 += kBlock) {  // block-uniform loop (warp ballots inside)
            const unsigned int j = j0 + threadIdx.x;
            unsigned long long key = 0;
            bool spill = false;
            if (j < total) {
                key = s_sorted[j];
                const unsigned int r = s_reg[j];
                const unsigned long long pos = (unsigned long long)s_gbase[r] + (j - s_start[r]);
                if (pos < seg_cap)
                    stage[(unsigned long long)r * seg_cap + pos] = key;
                else
                    spill = true;  // region far above its share: to the overflow list
            }
            overflow_append(spill, key, 1u, ovf_key, ovf_cnt, ovf_n);
        }
        __syncthreads();
    }
    if (st) atomicOr(d_status, st);
}

// Work items of pass 2: kInsertItem staged keys of one region; items are
// numbered region after region.
__global__ void __launch_bounds__(kBlock) k_region_items(const unsigned int* __restrict__ cursor, int regions,
                                                        unsigned long long seg_cap, long long* item_start) {
    __shared__ unsigned int scratch[33];
    long long carry = 0;
    for (int r0 = 0; r0 < regions; r0 += kBlock) {
        const int r = r0 + threadIdx.x;
        unsigned int items = 0;
        if (r < regions) {
            const unsigned long long c = min((unsigned long long)cursor[r], seg_cap);
            items = (unsigned int)((c + kInsertItem - 1) / kInsertItem);
        }
        unsigned int tot;
        const unsigned int off = block_excl_scan(items, scratch, &tot);
        if (r < regions) item_start[r] = carry + off;
        carry += tot;
    }
    if (threadIdx.x == 0) item_start[regions] = carry;
}

__device__ __forceinline__ int find_region(const long long* __restrict__ start, int count, long long c) {
    int lo = 0, hi = count;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (start[mid] <= c)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Pass 1b of contraction: counting-sort each region's staged keys by bucket
// (the 2^kBucketBits-slot unit of pass 2) into per-bucket segments of a second
// staging buffer.  Work items are kInsertItem keys of one region; keys beyond
// a bucket segment's capacity go to the overflow list.  A block claims its
// next item and starts copying that item's keys to shared memory (cp.async)
// before sorting the current one, so the claim, the region lookup and the
// loads of one item overlap the work on the previous.
constexpr size_t kBucketSmem = (size_t)kInsertItem * (2 * 8 + 2);  // two key buffers + bucket per key
__global__ void __launch_bounds__(kBlock, 4) k_bucket(RegionTable t, const unsigned long long* __restrict__ stage,
                                                  unsigned long long seg_cap, const unsigned int* __restrict__ cursor,
                                                  const long long* __restrict__ item_start, int regions,
                                                  unsigned long long* __restrict__ stage2, unsigned long long seg2,
                                                  unsigned int* __restrict__ bcursor, unsigned long long* ovf_key,
                                                  unsigned int* ovf_cnt, unsigned long long* ovf_n,
                                                  unsigned long long* work) {
    extern __shared__ __align__(16) unsigned char smem_b[];
    unsigned long long* s_in = reinterpret_cast<unsigned long long*>(smem_b);        // 2 x kInsertItem keys
    unsigned short* s_b = reinterpret_cast<unsigned short*>(s_in + 2 * kInsertItem); // kInsertItem
    __shared__ unsigned int s_fill[kBlock], s_start[kBlock], s_gbase[kBlock];
    __shared__ unsigned int scratch[33];
    __shared__ long long s_it[2];
    __shared__ int s_r[2];
    __shared__ unsigned long long s_k0[2], s_k1[2];
    const int bb = (int)t.region_bits - kBucketBits;  // buckets per region: 2^bb <= kBlock
    const int NB = 1 << bb;
    const unsigned int local_mask = (1u << t.region_bits) - 1u;
    const long long total = item_start[regions];
    // claim an item for buffer q and start copying its keys there (one group)
    auto claim = [&](int q) {
        if (threadIdx.x == 0) {
            const long long it = (long long)atomicAdd(work, 1ull);
            s_it[q] = it;
            if (it < total) {
                const int r = find_region(item_start, regions, it);
                const unsigned long long cnt = min((unsigned long long)cursor[r], seg_cap);
                const unsigned long long k0 = (unsigned long long)(it - item_start[r]) * kInsertItem;
                s_r[q] = r;
                s_k0[q] = k0;
                s_k1[q] = min(k0 + kInsertItem, cnt);
            }
        }
        __syncthreads();
        if (s_it[q] < total) {
            const unsigned long long k0 = s_k0[q], k1 = s_k1[q];
            const unsigned long long* seg = stage + (unsigned long long)s_r[q] * seg_cap;
#pragma unroll
            for (int k = 0; k < (int)(kInsertItem / kBlock); ++k) {
                const unsigned long long j = k0 + (unsigned long long)(k * kBlock + threadIdx.x);
                if (j < k1) {
                    const unsigned int dst = (unsigned int)__cvta_generic_to_shared(
                        s_in + (size_t)q * kInsertItem + k * kBlock + threadIdx.x);
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(seg + j) : "memory");
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    int q = 0;
    claim(0);
    for (;;) {
        claim(q ^ 1);  // the next item's keys copy while this one is sorted
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        if (threadIdx.x < NB) s_fill[threadIdx.x] = 0u;
        __syncthreads();
        const long long it = s_it[q];
        if (it >= total) break;
        const int r = s_r[q];
        const unsigned long long k0 = s_k0[q], k1 = s_k1[q];
        unsigned long long* s_cur = s_in + (size_t)q * kInsertItem;  // this item's keys, then its sorted keys
        unsigned long long key[kInsertItem / kBlock];
        unsigned int meta[kInsertItem / kBlock];
#pragma unroll
        for (int k = 0; k < (int)(kInsertItem / kBlock); ++k) {
            const unsigned long long j = k0 + (unsigned long long)(k * kBlock + threadIdx.x);
            meta[k] = 0xFFFFFFFFu;
            key[k] = 0ull;
            if (j < k1) {
                key[k] = s_cur[k * kBlock + threadIdx.x];
                const unsigned int b = (tile_hash(key[k]) & local_mask) >> kBucketBits;
                meta[k] = (b << 12) | atomicAdd(&s_fill[b], 1u);
            }
        }
        __syncthreads();  // also: every key of s_cur is in registers
        const unsigned int n_items = block_excl_scan_bins(s_fill, NB, s_start, scratch);
        const unsigned long long g0 = (unsigned long long)r << bb;  // first bucket of region r
        if (threadIdx.x < NB && s_fill[threadIdx.x])
            s_gbase[threadIdx.x] = atomicAdd(&bcursor[g0 + threadIdx.x], s_fill[threadIdx.x]);
#pragma unroll
        for (int k = 0; k < (int)(kInsertItem / kBlock); ++k) {
            if (meta[k] != 0xFFFFFFFFu) {
                const unsigned int b = meta[k] >> 12;
                const unsigned int pos = s_start[b] + (meta[k] & 0xFFFu);
                s_cur[pos] = key[k];
                s_b[pos] = (unsigned short)b;
            }
        }
        __syncthreads();
        for (unsigned int j0 = 0; j0 < n_items; j0 += kBlock) {  // block-uniform loop (warp ballots inside)
            const unsigned int j = j0 + threadIdx.x;
            unsigned long long k = 0;
            bool spill = false;
            if (j < n_items) {
                k = s_cur[j];
                const unsigned int b = s_b[j];
                const unsigned long long pos = (unsigned long long)s_gbase[b] + (j - s_start[b]);
                if (pos < seg2)
                    stage2[(g0 + b) * seg2 + pos] = k;
                else
                    spill = true;  // bucket far above its share: to the overflow list
            }
            overflow_append(spill, k, 1u, ovf_key, ovf_cnt, ovf_n);
        }
        __syncthreads();
        q ^= 1;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Add one point to `key` in a bucket held in shared memory (linear probing
// from the tile's slot within the bucket, as in the global table).  Returns
// false when the key finds neither itself nor an empty slot within
// kBucketProbe slots (the bucket is nearly full).
constexpr unsigned int kBucketProbe = 128;
__device__ __forceinline__ bool bucket_add(Slot* s_tab, unsigned long long key) {
    unsigned int i = tile_hash(key) & (kBucketSlots - 1u);
    for (unsigned int p = 0; p < kBucketProbe; ++p) {
        unsigned long long k = *reinterpret_cast<volatile unsigned long long*>(&s_tab[i].key);
        if (k == kEmptyKey) k = atomicCAS(&s_tab[i].key, kEmptyKey, key);
        if (k == kEmptyKey || k == key) {
            atomicAdd(&s_tab[i].count, 1u);
            return true;
        }
        i = (i + 1u) & (kBucketSlots - 1u);
    }
    return false;
}

// Pass 2 of contraction: one bucket at a time per block.  The bucket's slots
// are copied to shared memory (or cleared, for the first round after a reset,
// when the table's contents are void), its staged keys are inserted there with
// shared-memory atomics, and the bucket is written back whole.  New tiles are
// counted once per bucket, as the growth of its occupied slots.  A key that
// finds no room within kBucketProbe slots goes to the overflow list and
// switches the bucket to passing its remaining keys there unprobed; such keys,
// and a bucket left holding more than `limit` tiles, are counted in *d_full so
// that the host grows the table.
constexpr int kInsBlock = 512;
constexpr int kInsertUnroll = 4;
__global__ void __launch_bounds__(kInsBlock) k_insert_bucket(Slot* __restrict__ tab, unsigned long long n_buckets,
                                                            const unsigned long long* __restrict__ stage2,
                                                            unsigned long long seg2,
                                                            const unsigned int* __restrict__ bcursor, int fresh,
                                                            unsigned int limit, unsigned long long* d_newkeys,
                                                            unsigned long long* d_full, unsigned long long* ovf_key,
                                                            unsigned int* ovf_cnt, unsigned long long* ovf_n,
                                                            unsigned long long* work) {
    extern __shared__ __align__(16) unsigned char smem[];
    Slot* s_tab = reinterpret_cast<Slot*>(smem);  // kBucketSlots slots
    __shared__ unsigned int s_occ0, s_occ1, s_nfull;
    __shared__ int s_full;
    __shared__ unsigned long long s_b;
    const int lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) {
            s_b = atomicAdd(work, 1ull);
            s_occ0 = 0u;
            s_occ1 = 0u;
            s_nfull = 0u;
            s_full = 0;
        }
        __syncthreads();
        const unsigned long long b = s_b;
        if (b >= n_buckets) break;
        const unsigned long long n = min((unsigned long long)bcursor[b], seg2);
        if (n == 0 && !fresh) {  // untouched bucket of a live table: nothing to do
            __syncthreads();
            continue;
        }
        ulonglong2* g = reinterpret_cast<ulonglong2*>(tab + (b << kBucketBits));
        ulonglong2* sv = reinterpret_cast<ulonglong2*>(s_tab);
        if (fresh) {
            ulonglong2 e;
            e.x = kEmptyKey;
            e.y = (unsigned long long)kAuxNone << 32;  // count 0, aux none
            for (unsigned int i = threadIdx.x; i < kBucketSlots; i += kInsBlock) sv[i] = e;
        } else {
            // all 4096 16-byte slot copies in flight at once, straight to shared memory
            for (unsigned int i = threadIdx.x; i < kBucketSlots; i += kInsBlock) {
                const unsigned int dst = (unsigned int)__cvta_generic_to_shared(sv + i);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(g + i) : "memory");
            }
            asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        unsigned int occ = 0;
        if (!fresh)
            for (unsigned int i = threadIdx.x; i < kBucketSlots; i += kInsBlock) occ += sv[i].x != kEmptyKey;
        occ = __reduce_add_sync(0xFFFFFFFFu, occ);
        if (lane == 0 && occ) atomicAdd(&s_occ0, occ);
        __syncthreads();  // every slot counted before any insertion
        const unsigned long long* keys = stage2 + b * seg2;
        unsigned int full = 0;
        for (unsigned long long j0 = 0; j0 < n; j0 += (unsigned long long)kInsBlock * kInsertUnroll) {
            unsigned long long kk[kInsertUnroll];
#pragma unroll
            for (int u = 0; u < kInsertUnroll; ++u) {
                const unsigned long long j = j0 + (unsigned long long)(u * kInsBlock + threadIdx.x);
                kk[u] = j < n ? __ldcs(keys + j) : kInvalidKey;
            }
#pragma unroll
            for (int u = 0; u < kInsertUnroll; ++u) {
                bool spill = false;
                if (kk[u] != kInvalidKey) {
                    if (*reinterpret_cast<volatile int*>(&s_full) || !bucket_add(s_tab, kk[u])) {
                        spill = true;
                        s_full = 1;
                        ++full;
                    }
                }
                overflow_append(spill, kk[u], 1u, ovf_key, ovf_cnt, ovf_n);
            }
        }
        full = __reduce_add_sync(0xFFFFFFFFu, full);
        if (lane == 0 && full) atomicAdd(&s_nfull, full);
        __syncthreads();
        occ = 0;
        for (unsigned int i = threadIdx.x; i < kBucketSlots; i += kInsBlock) {
            const ulonglong2 v = sv[i];
            occ += v.x != kEmptyKey;
            g[i] = v;
        }
        occ = __reduce_add_sync(0xFFFFFFFFu, occ);
        if (lane == 0 && occ) atomicAdd(&s_occ1, occ);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_occ1 > s_occ0) atomicAdd(d_newkeys, (unsigned long long)(s_occ1 - s_occ0));
            const unsigned int over = s_nfull + (s_occ1 > limit ? 1u : 0u);
            if (over) atomicAdd(d_full, (unsigned long long)over);
        }
    }
}

// Pass 2 of contraction for a round much smaller than the table (a later chunk
// of a stream): insert the staged keys straight into the table with global
// atomics, region after region, so the table lines being updated stay in L2,
// instead of rewriting every bucket.  Equal keys within a warp are merged.
// New tiles are only created while the table holds fewer than `new_limit`
// tiles; past it, and for probe sequences longer than the bound, keys go to
// the overflow list with their counts.  Table plus list always hold the exact
// counts; the host grows the table and re-inserts the list.
__global__ void __launch_bounds__(kBlock) k_insert(RegionTable t, const unsigned long long* __restrict__ stage,
                                                  unsigned long long seg_cap, const unsigned int* __restrict__ cursor,
                                                  const long long* __restrict__ item_start, int regions,
                                                  unsigned long long new_limit, unsigned long long* d_newkeys,
                                                  unsigned long long* ovf_key, unsigned int* ovf_cnt,
                                                  unsigned long long* ovf_n, unsigned long long* work) {
    __shared__ int s_allow;
    __shared__ unsigned int s_new;
    __shared__ long long s_it;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long total = item_start[regions];
    for (;;) {
        // items are taken in order from a shared counter, so all blocks work on
        // one narrow window of regions (a static stride lets blocks drift apart)
        if (threadIdx.x == 0) {
            s_it = (long long)atomicAdd(work, 1ull);
            s_allow = *reinterpret_cast<volatile unsigned long long*>(d_newkeys) < new_limit;
            s_new = 0u;
        }
        __syncthreads();
        const long long it = s_it;
        if (it >= total) break;
        const bool allow = s_allow != 0;
        const int r = find_region(item_start, regions, it);
        const unsigned long long cnt = min((unsigned long long)cursor[r], seg_cap);
        const unsigned long long k0 = (unsigned long long)(it - item_start[r]) * kInsertItem;
        const unsigned long long k1 = min(k0 + kInsertItem, cnt);
        const unsigned long long* seg = stage + (unsigned long long)r * seg_cap;
        unsigned int newk = 0;
        for (unsigned long long base = k0 + warp * 32; base < k0 + kInsertItem; base += kBlock) {
            const unsigned long long k = base + lane;
            const unsigned long long key = k < k1 ? __ldcs(seg + k) : kInvalidKey;
            const unsigned int grp = __match_any_sync(0xFFFFFFFFu, key);
            const unsigned int c = (unsigned int)__popc(grp);
            bool spill = false;
            if (lane == __ffs(grp) - 1 && key != kInvalidKey) {
                // past the new-tile limit the table is due to grow: spill at once
                const int rc = allow ? rt_add(t, key, c) : -1;
                if (rc > 0)
                    ++newk;
                else if (rc < 0)
                    spill = true;
            }
            overflow_append(spill, key, c, ovf_key, ovf_cnt, ovf_n);
        }
        newk = __reduce_add_sync(0xFFFFFFFFu, newk);
        if (lane == 0 && newk) atomicAdd(&s_new, newk);
        __syncthreads();
        if (threadIdx.x == 0 && s_new) atomicAdd(d_newkeys, (unsigned long long)s_new);
        __syncthreads();
    }
}

// Re-insert the overflow list (after the table has grown); must succeed.
__global__ void k_reinsert(RegionTable t, const unsigned long long* __restrict__ ovf_key,
                           const unsigned int* __restrict__ ovf_cnt, unsigned long long n,
                           unsigned long long* d_newkeys, unsigned int* d_status) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned int newk = 0, st = 0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int rc = rt_add(t, ovf_key[i], ovf_cnt[i]);
        if (rc > 0)
            ++newk;
        else if (rc < 0)
            st |= kStFull;
    }
    if (newk) atomicAdd(d_newkeys, (unsigned long long)newk);
    if (st) atomicOr(d_status, st);
}

__global__ void k_rehash(const Slot* __restrict__ old_tab, unsigned long long old_cap, RegionTable t,
                         unsigned int* d_status) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned int st = 0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < old_cap; i += stride) {
        const Slot s = old_tab[i];
        if (s.key != kEmptyKey && rt_add(t, s.key, s.count) < 0) st |= kStFull;
    }
    if (st) atomicOr(d_status, st);
}

// Compaction of occupied slots with count >= min_count into (key, count, slot)
// rows.  With min_count = tau this is the significant-tile selection; each
// selected slot's aux receives its row index.
constexpr int kSelItems = 8;
__global__ void __launch_bounds__(kBlock) k_select(Slot* tab, unsigned long long cap, unsigned int min_count,
                                                  unsigned long long* out_key, unsigned int* out_cnt,
                                                  unsigned int* out_slot, unsigned long long* d_rows,
                                                  unsigned long long row_cap, int write_aux, int marked) {
    __shared__ unsigned int scratch[33];
    __shared__ unsigned long long s_base;
    const unsigned long long tile = (unsigned long long)kBlock * kSelItems;
    for (unsigned long long t0 = (unsigned long long)blockIdx.x * tile; t0 < cap;
         t0 += (unsigned long long)gridDim.x * tile) {
        unsigned long long k[kSelItems];
        unsigned int c[kSelItems];
        unsigned int flags = 0;
#pragma unroll
        for (int it = 0; it < kSelItems; ++it) {
            const unsigned long long idx = t0 + (unsigned long long)it * kBlock + threadIdx.x;
            k[it] = kEmptyKey;
            c[it] = 0;
            bool mark = false;
            if (idx < cap) {
                const ulonglong2 v = __ldcs(reinterpret_cast<const ulonglong2*>(tab) + idx);
                k[it] = v.x;
                c[it] = (unsigned int)v.y;
                mark = marked && (unsigned int)(v.y >> 32) == kAuxGroup;
            }
            if (k[it] != kEmptyKey && (c[it] >= min_count || mark)) flags |= 1u << it;
        }
        unsigned int total;
        unsigned int off = block_excl_scan((unsigned int)__popc(flags), scratch, &total);
        if (threadIdx.x == 0) s_base = total ? atomicAdd(d_rows, (unsigned long long)total) : 0ull;
        __syncthreads();
        const unsigned long long base = s_base;
#pragma unroll
        for (int it = 0; it < kSelItems; ++it) {
            if (flags & (1u << it)) {
                const unsigned long long idx = t0 + (unsigned long long)it * kBlock + threadIdx.x;
                const unsigned long long row = base + off++;
                if (row >= row_cap) continue;  // more rows than the tile count allows: reported by the host
                out_key[row] = k[it];
                out_cnt[row] = c[it];
                if (out_slot) out_slot[row] = (unsigned int)idx;
                if (write_aux) tab[idx].aux = (unsigned int)row;
            }
        }
        __syncthreads();
    }
}

// Probe lengths of the occupied slots: a lookup of a tile reads 1 + its
// distance from its home slot, along the bucket.
__global__ void __launch_bounds__(kBlock) k_probe_stats(const Slot* __restrict__ tab, RegionTable t,
                                                       unsigned long long* out) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned long long occ = 0, sum = 0;
    unsigned int mx = 0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < t.cap; i += stride) {
        const unsigned long long key = tab[i].key;
        if (key == kEmptyKey) continue;
        const unsigned int p = (unsigned int)((i - home_slot(key, t)) & (kBucketSlots - 1u)) + 1u;
        ++occ;
        sum += p;
        mx = max(mx, p);
    }
    occ = __reduce_add_sync(0xFFFFFFFFu, (unsigned int)occ);
    sum = __reduce_add_sync(0xFFFFFFFFu, (unsigned int)sum);
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    if ((threadIdx.x & 31) == 0 && occ) {
        atomicAdd(&out[0], occ);
        atomicAdd(&out[1], sum);
        atomicMax(&out[2], (unsigned long long)mx);
    }
}

// The selection never writes more rows than its buffers hold; if it counted
// more (the tile count was wrong), clamp the count for the kernels after it
// and report an internal error.
__global__ void k_clamp_rows(unsigned long long* d_rows, unsigned long long row_cap, unsigned int* d_status) {
    if (*d_rows > row_cap) {
        *d_rows = row_cap;
        atomicOr(d_status, kStInternal);
    }
}

__global__ void k_uf_init(const unsigned long long* d_nsig, int* parent, unsigned int* csize,
                          unsigned long long* cmin) {
    const long long S = (long long)*d_nsig;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += stride) {
        parent[i] = (int)i;
        csize[i] = 0u;
        cmin[i] = ~0ull;
    }
}

// Next chunk of kBlock rows for this block, taken in order from a shared
// counter: rows in flight stay in one window (and so do the table regions and
// union-find roots they touch).  Returns a value >= limit when done.
__device__ __forceinline__ long long next_chunk(unsigned long long* work, long long* s_chunk) {
    if (threadIdx.x == 0) *s_chunk = (long long)atomicAdd(work, 1ull) * kBlock;
    __syncthreads();
    const long long c = *s_chunk;
    __syncthreads();
    return c;
}

// The forward half of neighbors(u, delta) (Alg. 1): offsets (dx, dy) with
// dx > 0, or dx = 0 and dy > 0, inside the Chebyshev or Manhattan ball of
// radius delta (Sect. 3.2).  Adjacency is symmetric, so these visit every
// neighbour pair once.
constexpr int kMaxFwd = ((2 * RASTER_MAX_DELTA + 1) * (2 * RASTER_MAX_DELTA + 1) - 1) / 2;
struct NbrSet {
    int n;
    int dims;
    signed char dx[kMaxFwd];
    signed char dy[kMaxFwd];
    signed char dz[kMaxFwd];
};

// One thread per (significant tile, forward neighbour); a tile's lookups and
// unions run in parallel threads.  The default neighbourhood (Chebyshev
// distance 1: (x+1, y-1), (x+1, y), (x+1, y+1), (x, y+1)) is specialised.
// Significance is read from the slot: the selection wrote each significant
// tile's row into aux, every other slot holds kAuxNone.
template <bool GENERAL>
__global__ void __launch_bounds__(kBlock) k_hook(const unsigned long long* d_nsig,
                                                const unsigned long long* __restrict__ sig_key, RegionTable t,
                                                const NbrSet* __restrict__ nbr, int nfwd, int dims, int* parent,
                                                unsigned long long* work, unsigned int* d_status) {
    __shared__ long long s_chunk;
    const int F = GENERAL ? nfwd : 4;
    const long long SF = (long long)F * (long long)*d_nsig;
    unsigned int st = 0;
    for (long long w0 = next_chunk(work, &s_chunk); w0 < SF; w0 = next_chunk(work, &s_chunk)) {
        const long long w = w0 + threadIdx.x;
        if (w >= SF) continue;
        long long i;
        int dx, dy, dz = 0;
        if (GENERAL) {
            i = w / F;
            const int q = (int)(w - i * F);
            dx = __ldg(&nbr->dx[q]);
            dy = __ldg(&nbr->dy[q]);
            dz = __ldg(&nbr->dz[q]);
        } else {
            i = w >> 2;
            const int q = (int)(w & 3);
            dx = q < 3 ? 1 : 0;
            dy = q < 3 ? q - 1 : 1;
        }
        const unsigned long long key = sig_key[i];
        unsigned long long nk;
        if (GENERAL && dims == 3) {
            const int nx = key3(key, 0) + dx, ny = key3(key, 1) + dy, nz = key3(key, 2) + dz;
            if (nx < kMin3 || nx > kMax3 || ny < kMin3 || ny > kMax3 || nz < kMin3 || nz > kMax3) continue;
            nk = pack_key3(nx, ny, nz);
        } else {
            const long long nx = (long long)key_x(key) + dx;
            const long long ny = (long long)key_y(key) + dy;
            if (nx > 2147483646ll || ny > 2147483646ll || ny < -2147483647ll) continue;
            nk = pack_key((int)nx, (int)ny);
        }
        const Slot nb = rt_get(t, nk);
        if (nb.key != nk || nb.aux == kAuxNone) continue;
        if (!uf_unite(parent, (int)i, (int)nb.aux, kUnionLimit)) st |= kStInternal;
    }
    if (st) atomicOr(d_status, st);
}

// The post-processing of Sect. 3.6 ("disadvantageous grid layouts"): an
// occupied tile with fewer than tau points is marked (aux = kAuxGroup) when
// one of the four 2 x 2 tile groups it belongs to holds at least tau points;
// the selection then takes it as significant.  One thread per slot reads the
// counts of the tile's eight neighbours; slots are taken in order, chunk by
// chunk, so the lookups stay within the few regions in flight.
__global__ void __launch_bounds__(kBlock) k_groups(Slot* tab, RegionTable t, unsigned int tau,
                                                  unsigned long long* work) {
    __shared__ long long s_chunk;
    for (long long c0 = next_chunk(work, &s_chunk); c0 < (long long)t.cap; c0 = next_chunk(work, &s_chunk)) {
        const unsigned long long i = (unsigned long long)c0 + threadIdx.x;
        if (i >= t.cap) continue;
        const Slot sl = load_slot(&tab[i]);
        if (sl.key == kEmptyKey || sl.count >= tau) continue;
        const long long x = key_x(sl.key), y = key_y(sl.key);
        unsigned long long c[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                c[a][b] = 0ull;
                const long long nx = x + a - 1, ny = y + b - 1;
                if (a == 1 && b == 1) {
                    c[a][b] = sl.count;
                } else if (nx >= -2147483647ll && nx <= 2147483646ll && ny >= -2147483647ll && ny <= 2147483646ll) {
                    const unsigned long long nk = pack_key((int)nx, (int)ny);
                    const Slot nb = rt_get(t, nk);
                    if (nb.key == nk) c[a][b] = nb.count;
                }
            }
        bool keep = false;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
                keep |= c[a][b] + c[a + 1][b] + c[a][b + 1] + c[a + 1][b + 1] >= tau;
        if (keep) tab[i].aux = kAuxGroup;
    }
}

__global__ void __launch_bounds__(kBlock) k_flatten(const unsigned long long* d_nsig, int* parent,
                                                   unsigned long long* work) {
    __shared__ long long s_chunk;
    const long long S = (long long)*d_nsig;
    for (long long c = next_chunk(work, &s_chunk); c < S; c = next_chunk(work, &s_chunk)) {
        const long long i = c + threadIdx.x;
        if (i < S) parent[i] = uf_root(parent, (int)i);
    }
}

// Order of keys as unsigned integers: (x, y) order after flipping both sign
// bits of a two-coordinate key; a three-coordinate key is in (x, y, z) order
// as it stands.
constexpr unsigned long long kOrderXor2 = 0x8000000080000000ull, kOrderXor3 = 0ull;

// A kept tile's label code: offsets to its cluster-id tile for two
// coordinates, the escape to its result row for three.
__device__ __forceinline__ unsigned int label_code_d(unsigned long long key, unsigned long long cid, unsigned int row,
                                                     int dims) {
    return dims == 3 ? (0x80000000u | row) : label_code(key, cid, row);
}

__global__ void __launch_bounds__(kBlock) k_stats(const unsigned long long* d_nsig,
                                                 const unsigned long long* __restrict__ sig_key,
                                                 const int* __restrict__ parent, unsigned int* csize,
                                                 unsigned long long* cmin, unsigned long long* work,
                                                 unsigned long long order_xor) {
    __shared__ long long s_chunk;
    const long long S = (long long)*d_nsig;
    for (long long c = next_chunk(work, &s_chunk); c < S; c = next_chunk(work, &s_chunk)) {
        const long long i = c + threadIdx.x;
        if (i < S) {
            const int r = parent[i];
            atomicAdd(&csize[r], 1u);
            atomicMin(&cmin[r], sig_key[i] ^ order_xor);
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_emit(const unsigned long long* d_nsig,
                                                const unsigned long long* __restrict__ sig_key,
                                                const unsigned int* __restrict__ sig_cnt,
                                                const unsigned int* __restrict__ sig_slot,
                                                const int* __restrict__ parent, const unsigned int* __restrict__ csize,
                                                const unsigned long long* __restrict__ cmin, unsigned int mu,
                                                Slot* tab, unsigned long long* out_key, unsigned int* out_cnt,
                                                unsigned long long* out_cid, unsigned int* out_slot,
                                                unsigned long long* d_nkept, unsigned long long* d_nclusters,
                                                unsigned long long* work, unsigned long long order_xor, int dims) {
    __shared__ unsigned int scratch[33];
    __shared__ unsigned long long s_base;
    __shared__ long long s_chunk;
    const long long S = (long long)*d_nsig;
    unsigned int clusters = 0;
    for (long long t0 = next_chunk(work, &s_chunk); t0 < S; t0 = next_chunk(work, &s_chunk)) {
        const long long i = t0 + threadIdx.x;
        bool keep = false;
        unsigned long long key = 0, cid = 0;
        int r = 0;
        if (i < S) {
            r = parent[i];
            keep = csize[r] >= mu;
            key = sig_key[i];
            cid = cmin[r] ^ order_xor;
            if (keep && r == (int)i) ++clusters;
        }
        unsigned int total;
        const unsigned int off = block_excl_scan(keep ? 1u : 0u, scratch, &total);
        if (threadIdx.x == 0) s_base = total ? atomicAdd(d_nkept, (unsigned long long)total) : 0ull;
        __syncthreads();
        if (i < S) {
            unsigned int code = kAuxNone;
            if (keep) {
                const unsigned long long row = s_base + off;
                out_key[row] = key;
                out_cnt[row] = sig_cnt[i];
                out_cid[row] = cid;
                out_slot[row] = sig_slot[i];
                code = label_code_d(key, cid, (unsigned int)row, dims);
            }
            tab[sig_slot[i]].aux = code;
        }
        __syncthreads();
    }
    clusters = __reduce_add_sync(0xFFFFFFFFu, clusters);
    if ((threadIdx.x & 31) == 0 && clusters) atomicAdd(d_nclusters, (unsigned long long)clusters);
}

template <bool WIDE, int DIMS>
__global__ void k_labels(const double* __restrict__ xy, long long n, ProjParams pp, RegionTable t, unsigned int tau,
                         const long long* __restrict__ cid_rows, long long* __restrict__ labels,
                         unsigned int* d_status) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned int st = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned long long key = project_in<WIDE, DIMS>(load_point<DIMS>(xy, i), pp);
        long long lab = (long long)kEmptyKey;
        if (key == kInvalidKey) {
            st |= kStRange;
        } else {
            const Slot sl = rt_get(t, key);
            if (sl.key == key) lab = label_decode(key, sl.aux, cid_rows);  // kAuxNone decodes to noise
        }
        __stcs(labels + i, lab);
    }
    if (st) atomicOr(d_status, st);
}

// RASTER' (Sect. 3.4): the points of every kept tile, as a CSR over result
// rows.  The slots of kept tiles temporarily hold their result row in aux.
__global__ void k_aux_rows(const unsigned long long* d_nkept, const unsigned int* __restrict__ out_slot, Slot* tab) {
    const long long K = (long long)*d_nkept;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < K; r += stride)
        tab[out_slot[r]].aux = (unsigned int)r;
}

__global__ void k_aux_codes(const unsigned long long* d_nkept, const unsigned int* __restrict__ out_slot,
                            const unsigned long long* __restrict__ out_key,
                            const unsigned long long* __restrict__ out_cid, Slot* tab, int dims) {
    const long long K = (long long)*d_nkept;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < K; r += stride)
        tab[out_slot[r]].aux = label_code_d(out_key[r], out_cid[r], (unsigned int)r, dims);
}

template <bool WIDE, int DIMS>
__global__ void k_group_count(const double* __restrict__ xy, long long n, ProjParams pp, RegionTable t,
                              unsigned int tau, unsigned int* row_count, int* point_row, unsigned int* d_status) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned int st = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned long long key = project_in<WIDE, DIMS>(load_point<DIMS>(xy, i), pp);
        int row = -1;
        if (key == kInvalidKey) {
            st |= kStRange;
        } else {
            const Slot sl = rt_get(t, key);
            if (sl.key == key && sl.aux != kAuxNone) {
                row = (int)sl.aux;
                atomicAdd(&row_count[row], 1u);
            }
        }
        point_row[i] = row;
    }
    if (st) atomicOr(d_status, st);
}

// Exclusive scan of row_count[0..K) into row_start[0..K]; three launches.
constexpr int kScanTile = kBlock * 8;
__global__ void __launch_bounds__(kBlock) k_scan_tiles(const unsigned long long* d_nkept,
                                                      const unsigned int* __restrict__ in, long long* out,
                                                      long long* tile_sums) {
    __shared__ unsigned int scratch[33];
    const long long K = (long long)*d_nkept;
    for (long long t0 = (long long)blockIdx.x * kScanTile; t0 < K; t0 += (long long)gridDim.x * kScanTile) {
        unsigned int v[8];
        unsigned int sum = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const long long i = t0 + threadIdx.x * 8 + k;
            v[k] = i < K ? in[i] : 0u;
            sum += v[k];
        }
        unsigned int total;
        unsigned int off = block_excl_scan(sum, scratch, &total);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const long long i = t0 + threadIdx.x * 8 + k;
            if (i < K) out[i] = off;
            off += v[k];
        }
        if (threadIdx.x == 0) tile_sums[t0 / kScanTile] = total;
    }
}

__global__ void __launch_bounds__(kBlock) k_scan_sums(const unsigned long long* d_nkept, long long* tile_sums,
                                                     long long* out) {
    __shared__ long long s_part[kBlock];
    const long long K = (long long)*d_nkept;
    const long long T = (K + kScanTile - 1) / kScanTile;
    // each thread owns a contiguous run of tile sums
    const long long per = (T + kBlock - 1) / kBlock;
    const long long a = threadIdx.x * per, b = min(a + per, T);
    long long sum = 0;
    for (long long j = a; j < b; ++j) sum += tile_sums[j];
    s_part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int j = 0; j < kBlock; ++j) {
            const long long x = s_part[j];
            s_part[j] = acc;
            acc += x;
        }
        out[K] = acc;  // total points in kept tiles
    }
    __syncthreads();
    long long acc = s_part[threadIdx.x];
    for (long long j = a; j < b; ++j) {
        const long long x = tile_sums[j];
        tile_sums[j] = acc;
        acc += x;
    }
}

__global__ void k_scan_add(const unsigned long long* d_nkept, const long long* __restrict__ tile_sums, long long* out) {
    const long long K = (long long)*d_nkept;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += stride)
        out[i] += tile_sums[i / kScanTile];
}

__global__ void k_group_scatter(long long n, const int* __restrict__ point_row, const long long* __restrict__ row_start,
                                unsigned int* cursor, long long* point_index) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int r = point_row[i];
        if (r >= 0) point_index[row_start[r] + atomicAdd(&cursor[r], 1u)] = i;
    }
}

// ---------------------------------------------------------------------------
// Host side

std::atomic<unsigned long long> g_launches{0};

}  // namespace

namespace raster {
void note_launch(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
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
    unsigned long long* h_ctr = nullptr;  // pinned mirror: 7 counters, then the status word

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
    int* point_row = nullptr;
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

    unsigned long long* d_work = nullptr;  // work counters of the ordered kernels (8)

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
    RCHECK(h, cudaMemcpyAsync(h->h_ctr, h->d_ctr, 7 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
    h->h_ctr[7] = 0;
    RCHECK(h, cudaMemcpyAsync(h->h_ctr + 7, h->d_status, sizeof(unsigned int), cudaMemcpyDeviceToHost, h->stream));
    RCHECK(h, cudaStreamSynchronize(h->stream));
    merge_status(h, status_from_bits((unsigned int)h->h_ctr[7]));
    return RASTER_OK;
}

// Replace the table by one of `regions` x 2^bits slots, re-inserting every tile.
int grow_table(raster_handle* h, unsigned int regions, unsigned int bits) {
    // capacity is at most 2^32 slots, so at most 4096 regions: k_part keeps
    // region indices in 16 bits
    if (regions > 0xFFFFu) return RASTER_E_OOM;
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
    t.max_probe = max_probe_for(new_cap);
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
int round_part(raster_handle* h, const double* xy, long long m) {
    if (m <= 0) return RASTER_OK;
    const unsigned long long seg = h->stage_cap / h->regions;
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
                                                         h->ovf_cnt, h->d_ctr + 5, h->d_status);
    else
        k_part<WIDE, 2><<<g1, kBlock, smem, h->stream>>>(xy, m, h->pp, t, h->stage_keys, seg, h->cursor, h->ovf_key,
                                                         h->ovf_cnt, h->d_ctr + 5, h->d_status);
    note_launch();
    RCHECK(h, cudaGetLastError());
    return RASTER_OK;
}

int round_finish(raster_handle* h, long long n) {
    int rc;
    const bool grew_before = h->round_grew;
    const unsigned long long seg = h->stage_cap / h->regions;
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
        ti.max_probe = std::min<unsigned int>(t.max_probe, kInsertProbe);
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
        k_bucket<<<gb, kBlock, kBucketSmem, h->stream>>>(t, h->stage_keys, seg, h->cursor, h->item_start, (int)h->regions,
                                              h->stage2, seg2, h->bcursor, h->ovf_key, h->ovf_cnt, h->d_ctr + 5,
                                              h->d_work);
        // pass 2: bucket by bucket in shared memory
        const size_t bsmem = sizeof(Slot) * kBucketSlots;
        static bool battr = false;
        if (!battr) {
            RCHECK(h, cudaFuncSetAttribute(k_insert_bucket, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsmem));
            battr = true;
        }
        static int gi = grid_for((const void*)k_insert_bucket, kInsBlock, bsmem);
        k_insert_bucket<<<(int)std::min<unsigned long long>((unsigned long long)gi, n_buckets), kInsBlock, bsmem,
                          h->stream>>>(h->tab, n_buckets, h->stage2, seg2, h->bcursor, h->fresh ? 1 : 0,
                                       (unsigned int)(kNewLimit * kBucketSlots), h->d_ctr, h->d_ctr + 6, h->ovf_key,
                                       h->ovf_cnt, h->d_ctr + 5, h->d_work + 1);
        h->fresh = false;  // every bucket has been written
        note_launch(3);
        RCHECK(h, cudaGetLastError());
    }
    rc = read_counters(h);
    if (rc) return rc;
    const unsigned long long D = h->h_ctr[0], ovf = h->h_ctr[5], full = h->h_ctr[6];
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
        k_reinsert<<<g3, kBlock, 0, h->stream>>>(table_of(h), h->ovf_key, h->ovf_cnt, ovf, h->d_ctr, h->d_status);
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
    return RASTER_OK;
}

template <bool WIDE>
int contract_round(raster_handle* h, const double* xy, long long n) {
    int rc = round_begin(h, n);
    if (rc) return rc;
    rc = round_part<WIDE>(h, xy, n);
    if (rc) return rc;
    return round_finish(h, n);
}

int contract_device(raster_handle* h, const double* xy, long long n) {
    for (long long off = 0; off < n; off += kRoundPoints) {
        const long long m = std::min(n - off, kRoundPoints);
        const double* p = xy + (long long)h->dims * off;
        const int rc = h->wide ? contract_round<true>(h, p, m) : contract_round<false>(h, p, m);
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

template <bool WIDE, int DIMS>
void launch_labels(raster_handle* h, const double* xy, long long n, int64_t* labels) {
    static int grid = grid_for((const void*)k_labels<WIDE, DIMS>, kBlock);
    k_labels<WIDE, DIMS><<<(int)std::min<long long>(grid, (n + kBlock - 1) / kBlock), kBlock, 0, h->stream>>>(
        xy, n, h->pp, table_of(h), h->tau, reinterpret_cast<const long long*>(h->out_cid),
        reinterpret_cast<long long*>(labels), h->d_status);
}

template <bool WIDE, int DIMS>
void launch_group_count(raster_handle* h, const double* xy, long long n) {
    static int grid = grid_for((const void*)k_group_count<WIDE, DIMS>, kBlock);
    k_group_count<WIDE, DIMS><<<(int)std::min<long long>(grid, (n + kBlock - 1) / kBlock), kBlock, 0, h->stream>>>(
        xy, n, h->pp, table_of(h), h->tau, h->row_count, h->point_row, h->d_status);
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
    if (e == cudaSuccess) e = cudaMallocHost(&h->h_ctr, 8 * sizeof(unsigned long long));
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
    k_select<<<g_sel, kBlock, 0, s>>>(h->tab, h->cap, h->tau, h->sig_key, h->sig_cnt, h->sig_slot, d_nsig,
                                      (unsigned long long)h->agg_cap, 1, h->groups ? 1 : 0);
    k_clamp_rows<<<1, 1, 0, s>>>(d_nsig, (unsigned long long)h->agg_cap, h->d_status);
    note_launch(2);
    RCHECK(h, cudaGetLastError());
    static int g_init = grid_for((const void*)k_uf_init, kBlock);
    static int g_hook = grid_for((const void*)k_hook<false>, kBlock);
    static int g_flat = grid_for((const void*)k_flatten, kBlock);
    static int g_stat = grid_for((const void*)k_stats, kBlock);
    static int g_emit = grid_for((const void*)k_emit, kBlock);
    const int lim = (int)std::max<long long>(1, (D + kBlock - 1) / kBlock);
    k_uf_init<<<std::min(g_init, lim), kBlock, 0, s>>>(d_nsig, h->parent, h->csize, h->cmin);
    RCHECK(h, cudaMemsetAsync(h->d_work, 0, 8 * sizeof(unsigned long long), s));
    const long long F = h->general ? h->nbr.n : 4;  // forward neighbours per significant tile
    if (h->general)
        k_hook<true><<<std::min<long long>(g_hook, F * lim), kBlock, 0, s>>>(d_nsig, h->sig_key, table_of(h), h->d_nbr,
                                                                           h->nbr.n, h->dims, h->parent,
                                                                           h->d_work + 1, h->d_status);
    else
        k_hook<false><<<std::min<long long>(g_hook, F * lim), kBlock, 0, s>>>(d_nsig, h->sig_key, table_of(h), h->d_nbr,
                                                                            4, 2, h->parent, h->d_work + 1,
                                                                            h->d_status);
    k_flatten<<<std::min(g_flat, lim), kBlock, 0, s>>>(d_nsig, h->parent, h->d_work + 2);
    const unsigned long long order_xor = h->dims == 3 ? kOrderXor3 : kOrderXor2;
    k_stats<<<std::min(g_stat, lim), kBlock, 0, s>>>(d_nsig, h->sig_key, h->parent, h->csize, h->cmin,
                                                     h->d_work + 3, order_xor);
    k_emit<<<std::min(g_emit, lim), kBlock, 0, s>>>(d_nsig, h->sig_key, h->sig_cnt, h->sig_slot, h->parent, h->csize,
                                                    h->cmin, h->mu, h->tab, h->out_key, h->out_cnt, h->out_cid,
                                                    h->out_slot, h->d_ctr + 2, h->d_ctr + 3, h->d_work + 4, order_xor,
                                                    h->dims);
    note_launch(5);
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
    return h->status;
}

int raster_point_labels(raster_handle* h, const double* xy, int64_t n, int64_t* labels, void* stream) {
    if (!h || n < 0 || (n > 0 && (!xy || !labels || misaligned(xy, h->dims)))) return RASTER_E_ARG;
    if (hard_error(h->status)) return h->status;
    if (h->state != raster_handle::kAgglomerated) return RASTER_E_STATE;
    h->stream = (cudaStream_t)stream;
    if (n == 0) return RASTER_OK;
    if (h->dims == 3)
        h->wide ? launch_labels<true, 3>(h, xy, n, labels) : launch_labels<false, 3>(h, xy, n, labels);
    else
        h->wide ? launch_labels<true, 2>(h, xy, n, labels) : launch_labels<false, 2>(h, xy, n, labels);
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
    // scratch: a row per point, a counter and a cursor per result row
    if (n > h->point_row_cap) {
        RCHECK(h, cudaStreamSynchronize(s));
        if (h->point_row) cudaFree(h->point_row);
        h->point_row = nullptr;
        h->point_row_cap = 0;
        RCHECK(h, cudaMalloc(&h->point_row, sizeof(int) * (size_t)std::max<long long>(n, 1)));
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
        RCHECK(h, cudaMemsetAsync(h->row_count, 0, sizeof(unsigned int) * (size_t)K, s));  // reuse as cursors
        static int g2 = grid_for((const void*)k_group_scatter, kBlock);
        k_group_scatter<<<(int)std::min<long long>(g2, (n + kBlock - 1) / kBlock), kBlock, 0, s>>>(
            n, h->point_row, rs, h->row_count, reinterpret_cast<long long*>(point_index));
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

int raster_destroy(raster_handle* h) {
    if (!h) return RASTER_E_ARG;
    if (h->stream) cudaStreamSynchronize(h->stream);
    void* bufs[] = {h->tab,    h->d_ctr,   h->d_status, h->sig_key, h->sig_cnt, h->sig_slot, h->parent,
                    h->csize,  h->cmin,    h->out_key,  h->out_cnt, h->out_cid, h->stage_xy[0], h->stage_xy[1],
                    h->stage_lab[0], h->stage_lab[1], h->stage_keys, h->cursor, h->item_start, h->ovf_key,
                    h->ovf_cnt, h->d_work, h->out_slot, h->point_row, h->row_count, h->scan_sums,
                    h->stage2,  h->bcursor, h->d_nbr, h->res_xy};
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
