// Agglomeration kernels (Alg. 1 second loop, while loop and mu test):
// selection of significant tiles, table diagnostics, union-find hooking over
// neighbors(u, delta), the 2 x 2 group rule of Sect. 3.6, root walk, component
// statistics and result rows.
// Part of the single-instance library: included once, inside the anonymous
// namespace of raster_single.cu, after its constants (kBlock, the load and
// union limits) and the device, region and block helpers.
#pragma once

// Compaction of occupied slots with count >= min_count into (key, count, slot)
// rows.  With min_count = tau this is the significant-tile selection; each
// selected slot's aux receives its row index.  With `work`, blocks claim
// their tiles of slots in order from that counter, so the rows follow slot
// order (and table regions); without it they take a static grid stride.
constexpr int kSelItems = 8;
__global__ void __launch_bounds__(kBlock) k_select(Slot* tab, unsigned long long cap, unsigned int min_count,
                                                  unsigned long long* out_key, unsigned int* out_cnt,
                                                  unsigned int* out_slot, unsigned long long* d_rows,
                                                  unsigned long long row_cap, int write_aux, int marked,
                                                  unsigned long long* work = nullptr) {
    __shared__ unsigned int scratch[33];
    __shared__ unsigned long long s_base, s_t0;
    const unsigned long long tile = (unsigned long long)kBlock * kSelItems;
    auto next = [&](unsigned long long prev) {  // the block's next tile of slots (prev = ~0: its first)
        if (!work) return prev == ~0ull ? (unsigned long long)blockIdx.x * tile : prev + (unsigned long long)gridDim.x * tile;
        if (threadIdx.x == 0) s_t0 = atomicAdd(work, 1ull) * tile;
        __syncthreads();
        const unsigned long long v = s_t0;
        __syncthreads();
        return v;
    };
    for (unsigned long long t0 = next(~0ull); t0 < cap; t0 = next(t0)) {
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
                // kept in L2: a significant slot's aux is written right after
                const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(tab) + idx);
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

// The default neighbourhood (Chebyshev distance 1: (x+1, y-1), (x+1, y),
// (x+1, y+1), (x, y+1)) takes one thread per significant tile, which walks
// the four in turn: fewer threads of one cluster then hook into the same
// roots at once than with a thread per neighbour.  Other neighbourhoods (up
// to 40 forward offsets) take one thread per (significant tile, forward
// neighbour).  Significance is read from the slot: the selection wrote each
// significant tile's row into aux, every other slot holds kAuxNone.
constexpr long long kHookStreams = 8;    // chunk streams of the default hook
constexpr long long kHookSpacing = 1024;  // chunks between two streams

template <bool GENERAL>
__global__ void __launch_bounds__(kBlock) k_hook(const unsigned long long* d_nsig,
                                                const unsigned long long* __restrict__ sig_key, RegionTable t,
                                                const NbrSet* __restrict__ nbr, int nfwd, int dims, int* parent,
                                                int union_limit, unsigned long long* work, unsigned int* d_status) {
    __shared__ long long s_chunk;
    const long long S = (long long)*d_nsig;
    unsigned int st = 0;
    if (!GENERAL) {
        // Rows come in slot order (the selection claims its slots in order), so
        // consecutive chunks hold the tiles of the same clusters.  Claims
        // are spread over kHookStreams streams kHookSpacing chunks apart, so
        // that the blocks in flight hook into different clusters' roots while
        // each stream still walks the table in order.
        // (fewer rows than kHookStreams * kHookSpacing chunks: the streams close up,
        // so that a small table makes no more claims than it has chunks, about)
        const long long nch = (S + kBlock - 1) / kBlock;
        const long long P = max(1ll, min(kHookSpacing, (nch + kHookStreams - 1) / kHookStreams));
        const long long G = kHookStreams * P, nclaims = (nch + G - 1) / G * G;
        for (long long q = next_chunk(work, &s_chunk) / kBlock; q < nclaims; q = next_chunk(work, &s_chunk) / kBlock) {
            const long long w = q % G;
            const long long c = ((q - w) + (w % kHookStreams) * P + w / kHookStreams) * kBlock;
            if (c >= S) continue;  // the last group's claims beyond the rows
            const long long i = c + threadIdx.x;
            if (i >= S) continue;
            const unsigned long long key = sig_key[i];
            const long long x = key_x(key), y = key_y(key);
            for (int q = 0; q < 4; ++q) {
                const long long nx = x + (q < 3 ? 1 : 0), ny = y + (q < 3 ? q - 1 : 1);
                if (nx > 2147483646ll || ny > 2147483646ll || ny < -2147483647ll) continue;
                const unsigned long long nk = pack_key((int)nx, (int)ny);
                const Slot nb = rt_get(t, nk);
                if (nb.key != nk || nb.aux == kAuxNone) continue;
                if (!uf_unite(parent, (int)i, (int)nb.aux, union_limit)) st |= kStInternal;
            }
        }
        if (st) atomicOr(d_status, st);
        return;
    }
    const int F = nfwd;
    const long long SF = (long long)F * S;
    for (long long w0 = next_chunk(work, &s_chunk); w0 < SF; w0 = next_chunk(work, &s_chunk)) {
        const long long w = w0 + threadIdx.x;
        if (w >= SF) continue;
        const long long i = w / F;
        const int q = (int)(w - i * F);
        const int dx = __ldg(&nbr->dx[q]), dy = __ldg(&nbr->dy[q]), dz = __ldg(&nbr->dz[q]);
        const unsigned long long key = sig_key[i];
        unsigned long long nk;
        if (dims == 3) {
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
        if (!uf_unite(parent, (int)i, (int)nb.aux, union_limit)) st |= kStInternal;
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

// Root walk and component statistics in one pass: each significant tile's
// parent becomes its root, and the root's size and smallest tile (in key
// order) take the tile in.  Roots are final once hooking is done, and a
// parent read while another thread rewrites it is either the old parent or
// the root, both on the path to the same root.
__global__ void __launch_bounds__(kBlock) k_flatten_stats(const unsigned long long* d_nsig, int* parent,
                                                         const unsigned long long* __restrict__ sig_key,
                                                         unsigned int* csize, unsigned long long* cmin,
                                                         unsigned long long* work, unsigned long long order_xor) {
    __shared__ long long s_chunk;
    const long long S = (long long)*d_nsig;
    for (long long c = next_chunk(work, &s_chunk); c < S; c = next_chunk(work, &s_chunk)) {
        const long long i = c + threadIdx.x;
        if (i < S) {
            const int r = uf_root(parent, (int)i);
            parent[i] = r;
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
