// Per-point kernels after agglomeration: labels (RASTER*, Sect. 4.1) and the
// points of every kept tile (RASTER', Sect. 3.4).
// Part of the single-instance library: included once, inside the anonymous
// namespace of raster_single.cu, after its constants (kBlock, the load and
// union limits) and the device, region and block helpers.
#pragma once

// Block index of the kept tiles (two coordinates).  A point's label needs one
// random lookup; in the tile table that lookup lands anywhere in a table of
// 16-byte slots sized for every occupied tile, so nearly every one goes to
// DRAM.  Kept tiles are few and bunched in clusters, so the labels look them
// up in a much smaller index instead: one 16-byte entry per 8 x 8-tile block
// that holds a kept tile, two entries to a 32-byte bucket (one L2 sector,
// read with one load), with
//   word 0: the block (x >> 3, y >> 3), each plus 2^23 in 24 bits, above a
//           16-bit code: the offset from the block's corner tile to the
//           cluster id of its kept tiles, one signed byte per axis, or
//           kLidxMixed when the block's kept tiles name different cluster ids
//           or the offset does not fit; 0 marks an empty entry;
//   word 1: one bit per tile of the block, set for the kept ones.
// The buckets are split into one share per tile-table region, and a block's
// home bucket lies in the share of its region (a hash of the block within
// the share): the build, which takes the kept tiles in table order, then
// works on a few shares at a time in L2, while the labels' lookups still
// spread evenly.  A block's entry is in the first bucket, from its home
// bucket on, that had room when it was inserted; a bucket whose second entry
// is empty ends a search.  The index is sized from a linear-counting estimate
// of the block count (Whang, Vander-Zanden and Taylor, 1990), so that it
// fills to about kLidxLoad.  The tile table stays the reference: a point
// whose block is out of the index's range or mixed, or that meets an index
// whose build ran out of probes, takes the table lookup instead.  (Where a
// cluster breaks into pieces at its rim, a block often holds two cluster
// ids; a per-block record of two codes answered those points from the index
// but cost more to build and read than the table lookups it saved.)
constexpr int kLidxShift = 3;                     // blocks of 8 x 8 tiles
constexpr long long kLidxBias = 1ll << 23;        // block index bias (24-bit fields)
constexpr unsigned int kLidxMixed = 0x8000u;      // an x offset of -128 is never stored
constexpr unsigned int kLidxProbe = 512;          // buckets searched at most (build and lookup)
constexpr double kLidxLoad = 0.45;

struct LabelIndex {
    const unsigned long long* ent;  // 4 words per bucket; nullptr: no index
    unsigned long long buckets;     // regions x share
    unsigned long long share;       // buckets per table region
    const unsigned int* bad;        // nonzero: the build failed, use the table
};

// One 32-byte bucket (32-byte aligned) in one load, through L2.
__device__ __forceinline__ ulonglong4 lidx_load(const unsigned long long* p) {
    ulonglong4 v;
    asm volatile("ld.global.cg.v4.u64 {%0, %1, %2, %3}, [%4];"
                 : "=l"(v.x), "=l"(v.y), "=l"(v.z), "=l"(v.w)
                 : "l"(p));
    return v;
}

// The index word of the block holding `key`, without its code; false when
// the block lies outside the 24-bit fields.
__device__ __forceinline__ bool lidx_block(unsigned long long key, unsigned long long* bk) {
    const long long bx = (long long)(key_x(key) >> kLidxShift) + kLidxBias;  // floor division
    const long long by = (long long)(key_y(key) >> kLidxShift) + kLidxBias;
    if (bx < 1 || bx > (1ll << 24) - 2 || by < 1 || by > (1ll << 24) - 2) return false;
    *bk = ((unsigned long long)bx << 24) | (unsigned long long)by;
    return true;
}

// The splitmix64 finaliser (Steele, Lea and Flood, 2014) as the block hash.
__device__ __forceinline__ unsigned long long lidx_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Home bucket of a block: its region's share, at a 32-bit hash of the block
// (multiplicative combine of the two 24-bit fields, then xor-shift-multiply
// rounds) scaled to the share (shares hold fewer than 2^32 buckets).
__device__ __forceinline__ unsigned long long lidx_home(unsigned long long key, unsigned long long bk,
                                                        const RegionTable& t, unsigned long long share) {
    unsigned int h = ((unsigned int)(bk >> 24) * 0x9E3779B1u) ^ ((unsigned int)(bk & 0xFFFFFFull) * 0x85EBCA77u);
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    return (unsigned long long)region_of(key, t) * share + __umulhi(h, (unsigned int)share);
}

// A kept tile's code: the offset from its block's corner to its cluster id,
// or kLidxMixed when that does not fit a signed byte per axis.
__device__ __forceinline__ unsigned int lidx_code(unsigned long long key, unsigned long long cid) {
    const long long ox = (long long)key_x(cid) - (long long)(key_x(key) & ~7);
    const long long oy = (long long)key_y(cid) - (long long)(key_y(key) & ~7);
    return (ox >= -127 && ox <= 127 && oy >= -127 && oy <= 127)
               ? (((unsigned int)ox & 0xFFu) << 8) | ((unsigned int)oy & 0xFFu)
               : kLidxMixed;
}

__device__ __forceinline__ unsigned int lidx_bit(unsigned long long key) {
    return ((unsigned int)key_x(key) & 7u) * 8u + ((unsigned int)key_y(key) & 7u);
}

// Linear counting: one bit per hash value of each kept tile's block.
__global__ void k_lidx_count(const unsigned long long* d_nkept, const unsigned long long* __restrict__ out_key,
                             unsigned int* bitmap, int log2_bits) {
    const long long K = (long long)*d_nkept;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < K; r += stride) {
        unsigned long long bk;
        if (!lidx_block(out_key[r], &bk)) continue;
        const unsigned long long hv = lidx_mix(bk) >> (64 - log2_bits);
        atomicOr(&bitmap[hv >> 5], 1u << (hv & 31u));
    }
}

__global__ void __launch_bounds__(kBlock) k_lidx_zeros(const unsigned int* __restrict__ bitmap,
                                                      unsigned long long words, unsigned long long* zeros) {
    __shared__ unsigned int scratch[33];
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned int z = 0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride)
        z += 32u - (unsigned int)__popc(bitmap[i]);
    unsigned int total;
    block_excl_scan(z, scratch, &total);
    if (threadIdx.x == 0 && total) atomicAdd(zeros, (unsigned long long)total);
}

// Insert every kept tile: its block's entry (first come), the code (merged
// to kLidxMixed on disagreement) and its mask bit.
__global__ void k_lidx_build(const unsigned long long* d_nkept, const unsigned long long* __restrict__ out_key,
                             const unsigned long long* __restrict__ out_cid, RegionTable t, unsigned long long* ent,
                             unsigned long long buckets, unsigned long long share, unsigned int* bad) {
    const long long K = (long long)*d_nkept;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < K; r += stride) {
        const unsigned long long key = out_key[r];
        unsigned long long bk;
        if (!lidx_block(key, &bk)) continue;
        const unsigned int code = lidx_code(key, out_cid[r]);
        unsigned long long b = lidx_home(key, bk, t, share);
        unsigned long long* slot = nullptr;  // word 0 of the block's entry
        for (unsigned int p = 0; p < kLidxProbe && !slot; ++p) {
            for (int j = 0; j < 2; ++j) {  // entry 1 is taken only after entry 0
                unsigned long long* w0 = ent + 4 * b + 2 * j;
                unsigned long long w = *reinterpret_cast<volatile unsigned long long*>(w0);
                if (w == 0ull) {
                    const unsigned long long old = atomicCAS(w0, 0ull, (bk << 16) | code);
                    if (old == 0ull) {
                        slot = w0;
                        break;
                    }
                    w = old;
                }
                if ((w >> 16) == bk) {
                    // the code only ever moves to kLidxMixed, so this settles in two rounds
                    for (int it = 0; it < 4; ++it) {
                        const unsigned int cur = (unsigned int)(w & 0xFFFFull);
                        if (cur == code || cur == kLidxMixed) break;
                        const unsigned long long old = atomicCAS(w0, w, (w & ~0xFFFFull) | kLidxMixed);
                        if (old == w) break;
                        w = old;
                    }
                    slot = w0;
                    break;
                }
            }
            b = b + 1 == buckets ? 0 : b + 1;
        }
        if (!slot) {
            atomicOr(bad, 1u);
            continue;
        }
        atomicOr(slot + 1, 1ull << lidx_bit(key));
    }
}

// Label of a valid two-coordinate key of block bk from the block index,
// searching from bucket b on (at most `probes` buckets): true with *lab set
// (a cluster id or noise), false when the tile table has to answer.
__device__ __forceinline__ bool lidx_label_from(const LabelIndex& li, unsigned long long key, unsigned long long bk,
                                                unsigned long long b, unsigned int probes, long long* lab) {
    for (unsigned int p = 0; p < probes; ++p) {
        const ulonglong4 v = lidx_load(li.ent + 4 * b);
        unsigned long long w, w1;  // the entry: code word, kept mask
        if ((v.x >> 16) == bk) {
            w = v.x;
            w1 = v.y;
        } else if ((v.z >> 16) == bk) {
            w = v.z;
            w1 = v.w;
        } else {
            if (v.z == 0ull) {  // no kept tile in the block
                *lab = (long long)kEmptyKey;
                return true;
            }
            b = b + 1 == li.buckets ? 0 : b + 1;
            continue;
        }
        if (!((w1 >> lidx_bit(key)) & 1ull)) {  // not a kept tile
            *lab = (long long)kEmptyKey;
            return true;
        }
        const unsigned int code = (unsigned int)(w & 0xFFFFull);
        if (code == kLidxMixed) return false;
        *lab = (long long)pack_key((key_x(key) & ~7) + (int)(signed char)(code >> 8),
                                   (key_y(key) & ~7) + (int)(signed char)(code & 0xFFu));
        return true;
    }
    return false;
}

// The same from the block's home bucket.
__device__ __forceinline__ bool lidx_label(const LabelIndex& li, const RegionTable& t, unsigned long long key,
                                           long long* lab) {
    unsigned long long bk;
    if (!lidx_block(key, &bk)) return false;
    return lidx_label_from(li, key, bk, lidx_home(key, bk, t, li.share), kLidxProbe, lab);
}

// The tile key of point i: projected from its coordinates, or (KEYS) read
// from the keys that contraction stored for the same points.
template <bool WIDE, int DIMS, bool KEYS>
__device__ __forceinline__ unsigned long long point_key(const double* __restrict__ xy,
                                                        const unsigned long long* __restrict__ keys, long long i,
                                                        const ProjParams& pp) {
    if (KEYS) return __ldcs(keys + i);
    return project_in<WIDE, DIMS>(load_point<DIMS>(xy, i), pp);
}

template <bool WIDE, int DIMS, bool KEYS = false>
__global__ void k_labels(const double* __restrict__ xy, const unsigned long long* __restrict__ keys, long long n,
                         ProjParams pp, RegionTable t, unsigned int tau, const long long* __restrict__ cid_rows,
                         long long* __restrict__ labels, unsigned int* d_status, LabelIndex li) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const bool use_index = DIMS == 2 && li.ent != nullptr && *li.bad == 0u;
    unsigned int st = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned long long key = point_key<WIDE, DIMS, KEYS>(xy, keys, i, pp);
        long long lab = (long long)kEmptyKey;
        if (key == kInvalidKey) {
            st |= kStRange;
        } else if (!(use_index && lidx_label(li, t, key, &lab))) {
            const Slot sl = rt_get(t, key);
            if (sl.key == key) lab = label_decode(key, sl.aux, cid_rows);  // kAuxNone decodes to noise
        }
        __stcs(labels + i, lab);
    }
    if (st) atomicOr(d_status, st);
}

// Labels of two-coordinate points with the block index, without idle lanes.
// Most points are answered by the first bucket of their block's probe (the
// block's entry, or an empty second entry: no kept tile there).  The others
// -- a block that sits in a later bucket, a block whose kept tiles name
// several cluster ids, a block out of the index's range -- are queued per
// warp in shared memory and answered 32 at a time, the full index lookup
// and the table behind it, with every lane busy.  Answering them where they
// arise left most lanes of a warp idle while a few probed on.
constexpr int kLabQueue = 64;  // per warp: up to 31 waiting plus 32 new
constexpr long long kQueueTable = 1ll << 62;  // queued point that only the tile table can answer

// What the home bucket says about a key: kLidxAnswered with *lab set;
// kLidxLater when the block may sit in a later bucket (*next: the bucket
// after the home bucket); kLidxTable when only the tile table can answer (a
// mixed block, or a block out of the index's range).
constexpr int kLidxLater = 0, kLidxAnswered = 1, kLidxTable = 2;
__device__ __forceinline__ int lidx_first(const LabelIndex& li, const RegionTable& t, unsigned long long key,
                                          long long* lab, unsigned long long* next) {
    unsigned long long bk;
    if (!lidx_block(key, &bk)) return kLidxTable;
    const unsigned long long b = lidx_home(key, bk, t, li.share);
    const ulonglong4 v = lidx_load(li.ent + 4 * b);
    unsigned long long w, w1;
    if ((v.x >> 16) == bk) {
        w = v.x;
        w1 = v.y;
    } else if ((v.z >> 16) == bk) {
        w = v.z;
        w1 = v.w;
    } else {
        if (v.z != 0ull) {  // the block may sit in a later bucket
            *next = b + 1 == li.buckets ? 0 : b + 1;
            return kLidxLater;
        }
        *lab = (long long)kEmptyKey;
        return kLidxAnswered;
    }
    if (!((w1 >> lidx_bit(key)) & 1ull)) {
        *lab = (long long)kEmptyKey;
        return kLidxAnswered;
    }
    const unsigned int code = (unsigned int)(w & 0xFFFFull);
    if (code == kLidxMixed) return kLidxTable;
    *lab = (long long)pack_key((key_x(key) & ~7) + (int)(signed char)(code >> 8),
                               (key_y(key) & ~7) + (int)(signed char)(code & 0xFFu));
    return kLidxAnswered;
}

template <bool WIDE, bool KEYS = false>
__global__ void __launch_bounds__(kBlock) k_labels_idx(const double* __restrict__ xy,
                                                      const unsigned long long* __restrict__ keys, long long n,
                                                      ProjParams pp, RegionTable t,
                                                      const long long* __restrict__ cid_rows,
                                                      long long* __restrict__ labels, unsigned int* d_status,
                                                      LabelIndex li) {
    __shared__ unsigned long long s_key[kBlock / 32][kLabQueue];
    __shared__ long long s_idx[kBlock / 32][kLabQueue];            // point, with kQueueTable for the table
    __shared__ unsigned long long s_next[kBlock / 32][kLabQueue];  // the bucket to search from
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool index_ok = *li.bad == 0u;
    const long long warps_total = (long long)gridDim.x * (kBlock / 32);
    unsigned int st = 0;
    int qn = 0;  // warp-uniform
    // the last `count` queued points, one per lane
    auto drain = [&](int count) {
        if (lane < count) {
            const unsigned long long key = s_key[warp][qn - count + lane];
            const long long qi = s_idx[warp][qn - count + lane];
            const long long i = qi & ~kQueueTable;
            long long lab = (long long)kEmptyKey;
            unsigned long long bk;
            // a later bucket: the rest of the search (the home bucket was read)
            if (!(index_ok && !(qi & kQueueTable) && lidx_block(key, &bk) &&
                  lidx_label_from(li, key, bk, s_next[warp][qn - count + lane], kLidxProbe - 1, &lab))) {
                const Slot sl = rt_get(t, key);
                if (sl.key == key) lab = label_decode(key, sl.aux, cid_rows);  // kAuxNone decodes to noise
            }
            __stcs(labels + i, lab);
        }
        qn -= count;
        __syncwarp();
    };
    for (long long base = ((long long)blockIdx.x * (kBlock / 32) + warp) * 32; base < n; base += warps_total * 32) {
        const long long i = base + lane;
        unsigned long long key = kInvalidKey, next = 0;
        long long lab = (long long)kEmptyKey;
        bool defer = false, have = false;
        int mode = kLidxTable;
        if (i < n) {
            key = point_key<WIDE, 2, KEYS>(xy, keys, i, pp);
            if (key == kInvalidKey) {
                st |= kStRange;
                have = true;
            } else {
                if (index_ok) mode = lidx_first(li, t, key, &lab, &next);
                have = mode == kLidxAnswered;
                defer = !have;
            }
        }
        const unsigned int m = __ballot_sync(0xFFFFFFFFu, defer);
        if (defer) {
            const int pos = qn + __popc(m & ((1u << lane) - 1u));
            s_key[warp][pos] = key;
            s_idx[warp][pos] = mode == kLidxTable ? (i | kQueueTable) : i;
            s_next[warp][pos] = next;
        }
        qn += __popc(m);
        __syncwarp();
        if (have) __stcs(labels + i, lab);
        if (qn >= 32) drain(32);
    }
    if (qn > 0) drain(qn);
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

// After the table grew under live results (rehashing keeps keys and counts
// only): each result row finds its tile's new slot, and the slot gets back
// the row's label code.
__global__ void k_restore_rows(const unsigned long long* d_nkept, const unsigned long long* __restrict__ out_key,
                               const unsigned long long* __restrict__ out_cid, RegionTable t, unsigned int* out_slot,
                               unsigned int* d_status) {
    const long long K = (long long)*d_nkept;
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned int st = 0;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < K; r += stride) {
        const long long i = rt_find(t, out_key[r]);
        if (i < 0) {  // every kept tile was re-inserted
            st |= kStInternal;
            continue;
        }
        out_slot[r] = (unsigned int)i;
        t.tab[i].aux = label_code_d(out_key[r], out_cid[r], (unsigned int)r, t.dims);
    }
    if (st) atomicOr(d_status, st);
}

constexpr unsigned long long kNoRow = ~0ull;  // a point outside every kept tile

template <bool WIDE, int DIMS>
__global__ void k_group_count(const double* __restrict__ xy, long long n, ProjParams pp, RegionTable t,
                              unsigned int tau, unsigned int* row_count, unsigned long long* point_rr,
                              unsigned int* d_status) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned int st = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned long long key = project_in<WIDE, DIMS>(load_point<DIMS>(xy, i), pp);
        unsigned long long rr = kNoRow;  // (row << 32 | rank of the point within its row)
        if (key == kInvalidKey) {
            st |= kStRange;
        } else {
            const Slot sl = rt_get(t, key);
            if (sl.key == key && sl.aux != kAuxNone)
                rr = ((unsigned long long)sl.aux << 32) | atomicAdd(&row_count[sl.aux], 1u);
        }
        point_rr[i] = rr;
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

// Each grouped point goes to its row's start plus the rank it drew while
// counting, so the scatter takes no atomics.
__global__ void k_group_scatter(long long n, const unsigned long long* __restrict__ point_rr,
                                const long long* __restrict__ row_start, long long* point_index) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned long long rr = point_rr[i];
        if (rr != kNoRow) point_index[row_start[rr >> 32] + (unsigned int)rr] = i;
    }
}
