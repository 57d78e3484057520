// Per-point kernels after agglomeration: labels (RASTER*, Sect. 4.1) and the
// points of every kept tile (RASTER', Sect. 3.4).
// Part of the single-instance library: included once, inside the anonymous
// namespace of raster_single.cu, after its constants (kBlock, the load and
// union limits) and the device, region and block helpers.
#pragma once

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
