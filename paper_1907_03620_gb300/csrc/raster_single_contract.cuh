// Contraction kernels (Alg. 1 first loop; chunked processing, Sect. 3.6): table clear, pass 1
// (project and sort by region), item prefix, pass 1b (sort by bucket), pass 2
// (insert bucket by bucket in shared memory, or with global atomics for small
// rounds), and the re-insertion and rehash of table growth.
// Part of the single-instance library: included once, inside the anonymous
// namespace of raster_single.cu, after its constants (kBlock, the load and
// union limits) and the device, region and block helpers.
#pragma once

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
// share) go to the overflow list.  With keys_out, every point's key (or
// kInvalidKey) is also stored there in point order, for the labels.
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
                                                unsigned long long* ovf_n, unsigned int* d_status,
                                                unsigned long long* __restrict__ keys_out) {
    extern __shared__ unsigned char smem[];
    unsigned long long* s_sorted = reinterpret_cast<unsigned long long*>(smem);         // kPartTile keys
    unsigned int* s_fill = reinterpret_cast<unsigned int*>(s_sorted + kPartTile);       // regions
    unsigned int* s_start = s_fill + t.regions;                                         // regions
    unsigned int* s_gbase = s_start + t.regions;  // regions: segment position minus tile position (mod 2^32)
    unsigned short* s_reg = reinterpret_cast<unsigned short*>(s_gbase + t.regions);     // kPartTile regions
    __shared__ unsigned int scratch[33];
    const int R = (int)t.regions;
    unsigned int st = 0;
    for (long long t0 = (long long)blockIdx.x * kPartTile; t0 < n; t0 += (long long)gridDim.x * kPartTile) {
        for (int r = threadIdx.x; r < R; r += kBlock) s_fill[r] = 0u;
        __syncthreads();
        // two coordinates: half of the thread's loads in flight before projecting
        // that half (all of them at once spill registers); three: loaded where
        // projected
        unsigned long long key[kPartPer];
        unsigned int meta[kPartPer];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            PointIn<DIMS> p[DIMS == 2 ? kPartPer / 2 : 1];
            if (DIMS == 2) {
#pragma unroll
                for (int k = 0; k < kPartPer / 2; ++k) {
                    const long long idx = t0 + (h * (kPartPer / 2) + k) * kBlock + threadIdx.x;
                    if (idx < n) p[DIMS == 2 ? k : 0] = load_point<DIMS>(xy, idx);
                }
            }
#pragma unroll
            for (int k = 0; k < kPartPer / 2; ++k) {
                const int kk = h * (kPartPer / 2) + k;
                const long long idx = t0 + kk * kBlock + threadIdx.x;
                meta[kk] = 0xFFFFFFFFu;
                key[kk] = 0ull;
                if (idx < n) {
                    key[kk] = project_in<WIDE, DIMS>(DIMS == 2 ? p[DIMS == 2 ? k : 0] : load_point<DIMS>(xy, idx), pp);
                    if (keys_out) __stcs(keys_out + idx, key[kk]);  // each point's key, in point order
                    if (key[kk] == kInvalidKey) {
                        st |= kStRange;
                    } else {
                        const unsigned int r = region_of(key[kk], t);
                        meta[kk] = (r << 12) | atomicAdd(&s_fill[r], 1u);
                    }
                }
            }
        }
        __syncthreads();
        const unsigned int total = block_excl_scan_bins(s_fill, R, s_start, scratch);
        for (int r = threadIdx.x; r < R; r += kBlock)
            if (s_fill[r]) s_gbase[r] = atomicAdd(&cursor[r], s_fill[r]) - s_start[r];
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
                const unsigned long long pos = s_gbase[r] + j;  // below 2^32: within the segment or just past it
                if (pos < seg_cap)
                    stage[(unsigned long long)r * seg_cap + pos] = key;
                else
                    spill = true;  // region far above its share: to the overflow list
            }
            if (__any_sync(0xFFFFFFFFu, spill)) overflow_append(spill, key, 1u, ovf_key, ovf_cnt, ovf_n);
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
            // two keys per 16-byte copy: k0 and seg_cap are even, so a pair that
            // starts below k1 ends inside the segment (its second key may lie past
            // k1, and is not read)
            const unsigned long long k0 = s_k0[q], k1 = s_k1[q];
            const unsigned long long* seg = stage + (unsigned long long)s_r[q] * seg_cap;
#pragma unroll
            for (int k = 0; k < (int)(kInsertItem / kBlock / 2); ++k) {
                const unsigned int pj = 2u * (unsigned int)(k * kBlock + threadIdx.x);
                const unsigned long long j = k0 + pj;
                if (j < k1) {
                    const unsigned int dst =
                        (unsigned int)__cvta_generic_to_shared(s_in + (size_t)q * kInsertItem + pj);
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(seg + j) : "memory");
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
        if (threadIdx.x < NB && s_fill[threadIdx.x])  // segment position minus item position (mod 2^32)
            s_gbase[threadIdx.x] = atomicAdd(&bcursor[g0 + threadIdx.x], s_fill[threadIdx.x]) - s_start[threadIdx.x];
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
                const unsigned long long pos = s_gbase[b] + j;  // below 2^32: within the segment or just past it
                if (pos < seg2)
                    stage2[(g0 + b) * seg2 + pos] = k;
                else
                    spill = true;  // bucket far above its share: to the overflow list
            }
            if (__any_sync(0xFFFFFFFFu, spill)) overflow_append(spill, k, 1u, ovf_key, ovf_cnt, ovf_n);
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
template <bool LIMITED>
__device__ __forceinline__ bool bucket_add(Slot* s_tab, unsigned long long key, unsigned int max_probe) {
    unsigned int i = tile_hash(key) & (kBucketSlots - 1u);
    for (unsigned int p = 0; p < (LIMITED ? max_probe : kBucketProbe); ++p) {
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

// bucket_add on a bucket held as separate key and count arrays.
template <bool LIMITED>
__device__ __forceinline__ bool bucket_add_split(unsigned long long* s_key, unsigned int* s_cnt,
                                                 unsigned long long key, unsigned int max_probe) {
    unsigned int i = tile_hash(key) & (kBucketSlots - 1u);
    for (unsigned int p = 0; p < (LIMITED ? max_probe : kBucketProbe); ++p) {
        unsigned long long k = *reinterpret_cast<volatile unsigned long long*>(&s_key[i]);
        if (k == kEmptyKey) k = atomicCAS(&s_key[i], kEmptyKey, key);
        if (k == kEmptyKey || k == key) {
            atomicAdd(&s_cnt[i], 1u);
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
// switches the bucket to passing its remaining keys there unprobed (LIMITED:
// a test's lower probe bound, max_probe, in place of kBucketProbe); such keys,
// and a bucket left holding more than `limit` tiles, are counted in *d_full so
// that the host grows the table.
constexpr int kInsBlock = 512;
constexpr int kInsertUnroll = 4;
template <bool LIMITED>
__global__ void __launch_bounds__(kInsBlock) k_insert_bucket(Slot* __restrict__ tab, unsigned long long n_buckets,
                                                            const unsigned long long* __restrict__ stage2,
                                                            unsigned long long seg2,
                                                            const unsigned int* __restrict__ bcursor, int fresh,
                                                            unsigned int limit, unsigned int max_probe,
                                                            unsigned long long* d_newkeys,
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
                    if (*reinterpret_cast<volatile int*>(&s_full) || !bucket_add<LIMITED>(s_tab, kk[u], max_probe)) {
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

// Pass 2 for the first round into a void table (after a reset): as
// k_insert_bucket, but the bucket is cleared rather than loaded, and held as
// separate key and count arrays (48 KiB instead of 64 KiB: four blocks of
// kInsBlock threads per SM instead of three); it is written back as whole
// slots.  Every bucket is written, so the table needs no fill.
// With sel.tau > 0 it also selects the significant tiles (count >= tau) of
// each bucket as it writes it back, as the agglomeration's selection would
// (Alg. 1 second loop): their (key, count, slot) rows go to sel, and each
// such slot's aux gets its row (every other slot: aux none).  The counts are
// final for the round when the bucket is written; whether no later insertion
// changed them (overflow, growth, another round) is the host's to check.
struct PreSelect {
    unsigned int tau;  // 0: no selection
    unsigned long long* key;
    unsigned int* cnt;
    unsigned int* slot;
    unsigned long long* n;  // rows selected (may exceed cap: rows beyond it are not written)
    unsigned long long cap;
};
template <bool LIMITED>
__global__ void __launch_bounds__(kInsBlock, 4)
    k_insert_fresh(Slot* __restrict__ tab, unsigned long long n_buckets, const unsigned long long* __restrict__ stage2,
                   unsigned long long seg2, const unsigned int* __restrict__ bcursor, unsigned int limit,
                   unsigned int max_probe, unsigned long long* d_newkeys, unsigned long long* d_full,
                   unsigned long long* ovf_key, unsigned int* ovf_cnt, unsigned long long* ovf_n,
                   unsigned long long* work, PreSelect sel) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* s_key = reinterpret_cast<unsigned long long*>(smem);     // kBucketSlots keys
    unsigned int* s_cnt = reinterpret_cast<unsigned int*>(s_key + kBucketSlots);  // kBucketSlots counts
    __shared__ unsigned int s_occ, s_nfull;
    __shared__ int s_full;
    __shared__ unsigned long long s_b, s_row;
    __shared__ unsigned int scratch[33];
    const int lane = threadIdx.x & 31;
    constexpr int kPairs = (int)(kBucketSlots / 2 / kInsBlock);  // slot pairs per thread in the write-back
    for (;;) {
        // the previous bucket's write-back ended at a barrier
        if (threadIdx.x == 0) {
            s_b = atomicAdd(work, 1ull);
            s_occ = 0u;
            s_nfull = 0u;
            s_full = 0;
        }
        {
            ulonglong2 e;
            e.x = kEmptyKey;
            e.y = kEmptyKey;
            for (unsigned int i = threadIdx.x; i < kBucketSlots / 2; i += kInsBlock)
                reinterpret_cast<ulonglong2*>(s_key)[i] = e;
            for (unsigned int i = threadIdx.x; i < kBucketSlots / 4; i += kInsBlock)
                reinterpret_cast<uint4*>(s_cnt)[i] = make_uint4(0u, 0u, 0u, 0u);
        }
        __syncthreads();
        const unsigned long long b = s_b;
        if (b >= n_buckets) break;
        const unsigned long long n = min((unsigned long long)bcursor[b], seg2);
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
                    if (*reinterpret_cast<volatile int*>(&s_full) ||
                        !bucket_add_split<LIMITED>(s_key, s_cnt, kk[u], max_probe)) {
                        spill = true;
                        s_full = 1;
                        ++full;
                    }
                }
                if (__any_sync(0xFFFFFFFFu, spill)) overflow_append(spill, kk[u], 1u, ovf_key, ovf_cnt, ovf_n);
            }
        }
        full = __reduce_add_sync(0xFFFFFFFFu, full);
        if (lane == 0 && full) atomicAdd(&s_nfull, full);
        __syncthreads();
        // significant slots of the bucket: bit 2k (2k+1) for the first (second)
        // slot of the thread's k-th pair; their rows, in the thread's order
        unsigned int sig = 0;
        unsigned long long row = 0;
        if (sel.tau) {  // block-uniform
#pragma unroll
            for (int k = 0; k < kPairs; ++k) {
                const unsigned int i = threadIdx.x + (unsigned int)k * kInsBlock;
                const ulonglong2 k2 = reinterpret_cast<const ulonglong2*>(s_key)[i];
                const uint2 c2 = reinterpret_cast<const uint2*>(s_cnt)[i];
                sig |= (unsigned int)(k2.x != kEmptyKey && c2.x >= sel.tau) << (2 * k);
                sig |= (unsigned int)(k2.y != kEmptyKey && c2.y >= sel.tau) << (2 * k + 1);
            }
            unsigned int total;
            const unsigned int off = block_excl_scan<kInsBlock>((unsigned int)__popc(sig), scratch, &total);
            if (threadIdx.x == 0) s_row = total ? atomicAdd(sel.n, (unsigned long long)total) : 0ull;
            __syncthreads();
            row = s_row + off;
        }
        // two slots per thread and step: one 16-byte and one 8-byte shared load, two 16-byte stores
        ulonglong2* g = reinterpret_cast<ulonglong2*>(tab + (b << kBucketBits));
        unsigned int occ = 0;
#pragma unroll
        for (int k = 0; k < kPairs; ++k) {
            const unsigned int i = threadIdx.x + (unsigned int)k * kInsBlock;
            const ulonglong2 k2 = reinterpret_cast<const ulonglong2*>(s_key)[i];
            const uint2 c2 = reinterpret_cast<const uint2*>(s_cnt)[i];
            unsigned int aux0 = kAuxNone, aux1 = kAuxNone;
            if (sig & (1u << (2 * k))) {
                if (row < sel.cap) {
                    aux0 = (unsigned int)row;
                    sel.key[row] = k2.x;
                    sel.cnt[row] = c2.x;
                    sel.slot[row] = (unsigned int)((b << kBucketBits) + 2 * i);
                }
                ++row;
            }
            if (sig & (2u << (2 * k))) {
                if (row < sel.cap) {
                    aux1 = (unsigned int)row;
                    sel.key[row] = k2.y;
                    sel.cnt[row] = c2.y;
                    sel.slot[row] = (unsigned int)((b << kBucketBits) + 2 * i + 1);
                }
                ++row;
            }
            ulonglong2 v0, v1;
            v0.x = k2.x;
            v0.y = ((unsigned long long)aux0 << 32) | c2.x;
            v1.x = k2.y;
            v1.y = ((unsigned long long)aux1 << 32) | c2.y;
            occ += (k2.x != kEmptyKey) + (k2.y != kEmptyKey);
            g[2 * i] = v0;
            g[2 * i + 1] = v1;
        }
        occ = __reduce_add_sync(0xFFFFFFFFu, occ);
        if (lane == 0 && occ) atomicAdd(&s_occ, occ);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_occ) atomicAdd(d_newkeys, (unsigned long long)s_occ);
            const unsigned int over = s_nfull + (s_occ > limit ? 1u : 0u);
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

// Tiles counted elsewhere, added to the table: count[i] points of tile key[i]
// (the join of partial count maps, as when P-RASTER joins its per-thread maps,
// Sect. 3.5).  Keys outside the valid index range are skipped and reported.
__global__ void k_sum_counts(const unsigned int* __restrict__ count, long long n, unsigned long long* sum) {
    unsigned long long s = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += count[i];
    __syncwarp();
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(sum, s);
}

__device__ __forceinline__ bool valid_tile_key(unsigned long long k, int dims) {
    if (dims == 3) {
        if (k >> 63) return false;
        for (int a = 0; a < 3; ++a) {
            const int v = key3(k, a);
            if (v < kMin3 || v > kMax3) return false;
        }
        return true;
    }
    const int x = key_x(k), y = key_y(k);
    return x != INT_MIN && x != INT_MAX && y != INT_MIN && y != INT_MAX;
}

__global__ void k_add_tiles(RegionTable t, const unsigned long long* __restrict__ key,
                            const unsigned int* __restrict__ count, long long n, unsigned long long* d_newkeys,
                            unsigned int* d_status) {
    unsigned int newk = 0, st = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long k = key[i];
        const unsigned int c = count[i];
        if (c == 0) continue;
        if (!valid_tile_key(k, t.dims)) {
            st |= kStRange;
            continue;
        }
        const int rc = rt_add(t, k, c);
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
