// Segmented RASTER kernels: one launch serves many independent instances.
//
// An instance is a BatchInst: its points (for contraction), its projection
// parameters, its own tile table and the first row of its segment in shared
// row arrays (significant tiles, union-find, results).  Work items are found
// by binary search over prefix arrays, so instances of any sizes share one
// grid.  Used by the batched form (one fixed set of instances, replayed from a
// CUDA graph) and by the serving engine (a different mix every step).
#pragma once

#include <cuda_runtime.h>

#include "raster_block.cuh"
#include "raster_device.cuh"

namespace raster {
namespace {

constexpr long long kChunkPoints = 512;  // points per contraction work item
constexpr long long kSlotChunk = 2048;    // table slots per select work item
constexpr unsigned long long kMinTable = 4096;
constexpr int kAggBlock = 256;

struct BatchInst {
    const double2* xy;
    long long n;
    ProjParams pp;
    Slot* tab;
    unsigned int mask;
    unsigned int wide;
    unsigned int tau, mu;
    long long row_off;  // first row of this instance in the sig/result arenas
    unsigned int max_probe;  // most slots one insertion probes (the table size, unless a test lowers it)
    int union_limit;         // most steps of one union-find join
};

struct InstCounters {
    unsigned long long tiles;     // D
    unsigned long long sig;       // S
    unsigned long long kept;      // rows
    unsigned long long clusters;
    unsigned long long status;
};

// Index of the segment holding item c: start[i] <= c < start[i+1].
__device__ __forceinline__ int find_segment(const long long* __restrict__ start, int count, long long c) {
    int lo = 0, hi = count;  // invariant: start[lo] <= c < start[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (start[mid] <= c)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__global__ void k_batch_fill(Slot* tab, unsigned long long slots, InstCounters* ctr, int count) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    ulonglong2 v;
    v.x = kEmptyKey;
    v.y = 0ull;
    for (unsigned long long i = t; i < slots; i += stride) reinterpret_cast<ulonglong2*>(tab)[i] = v;
    for (unsigned long long i = t; i < (unsigned long long)count; i += stride) ctr[i] = InstCounters{0, 0, 0, 0, 0};
}

template <int W, bool PREAGG>
__global__ void __launch_bounds__(512) k_batch_contract(const BatchInst* __restrict__ inst,
                                                       const long long* __restrict__ chunk_start, int count,
                                                       InstCounters* ctr) {
    const int lane = threadIdx.x & 31;
    const long long warps_total = (long long)gridDim.x * (blockDim.x >> 5);
    const long long total = chunk_start[count];
    for (long long c = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < total; c += warps_total) {
        const int i = find_segment(chunk_start, count, c);
        const BatchInst I = inst[i];
        const long long p0 = (c - chunk_start[i]) * kChunkPoints;
        const long long p1 = min(p0 + kChunkPoints, I.n);
        unsigned int newk = 0, st = 0;
        for (long long base = p0; base < p1; base += 32 * W) {
            double2 p[W];
#pragma unroll
            for (int u = 0; u < W; ++u) {
                const long long k = base + u * 32 + lane;
                if (k < p1) p[u] = __ldcs(I.xy + k);
            }
#pragma unroll
            for (int u = 0; u < W; ++u) {
                const long long k = base + u * 32 + lane;
                unsigned long long key = kInvalidKey;
                if (k < p1) {
                    key = I.wide ? project_point<true>(p[u].x, p[u].y, I.pp) : project_point<false>(p[u].x, p[u].y, I.pp);
                    if (key == kInvalidKey) st |= kStRange;
                }
                unsigned int c_add = key != kInvalidKey ? 1u : 0u;
                if (PREAGG) {
                    const unsigned int grp = __match_any_sync(0xFFFFFFFFu, key);
                    c_add = (lane == __ffs(grp) - 1 && key != kInvalidKey) ? (unsigned int)__popc(grp) : 0u;
                }
                if (c_add) {
                    const int r = table_add(I.tab, I.mask, key, c_add, I.max_probe);
                    if (r > 0)
                        ++newk;
                    else if (r < 0)
                        st |= kStFull;
                }
            }
        }
        newk = __reduce_add_sync(0xFFFFFFFFu, newk);
        st = __reduce_or_sync(0xFFFFFFFFu, st);
        if (lane == 0) {
            if (newk) atomicAdd(&ctr[i].tiles, (unsigned long long)newk);
            if (st) atomicOr(&ctr[i].status, (unsigned long long)st);
        }
    }
}

// One block per table chunk of kSlotChunk slots (tables are multiples of it).
__global__ void __launch_bounds__(kScanBlock) k_batch_select(const BatchInst* __restrict__ inst,
                                                            const long long* __restrict__ slot_chunk_start,
                                                            int count, InstCounters* ctr,
                                                            unsigned long long* sig_key, unsigned int* sig_cnt,
                                                            unsigned int* sig_slot) {
    __shared__ unsigned int scratch[33];
    __shared__ unsigned long long s_base;
    constexpr int kItems = (int)(kSlotChunk / kScanBlock);
    const long long total = slot_chunk_start[count];
    for (long long c = blockIdx.x; c < total; c += gridDim.x) {
        const int i = find_segment(slot_chunk_start, count, c);
        const BatchInst I = inst[i];
        const unsigned long long s0 = (unsigned long long)(c - slot_chunk_start[i]) * kSlotChunk;
        unsigned long long k[kItems];
        unsigned int cn[kItems];
        unsigned int flags = 0;
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const ulonglong2 v = __ldcs(reinterpret_cast<const ulonglong2*>(I.tab) + s0 + it * kScanBlock + threadIdx.x);
            k[it] = v.x;
            cn[it] = (unsigned int)v.y;
            if (k[it] != kEmptyKey && cn[it] >= I.tau) flags |= 1u << it;
        }
        unsigned int tot;
        unsigned int off = block_excl_scan((unsigned int)__popc(flags), scratch, &tot);
        if (threadIdx.x == 0) s_base = tot ? atomicAdd(&ctr[i].sig, (unsigned long long)tot) : 0ull;
        __syncthreads();
        const unsigned long long base = (unsigned long long)I.row_off + s_base;
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            if (flags & (1u << it)) {
                const unsigned long long slot = s0 + it * kScanBlock + threadIdx.x;
                const unsigned long long row = base + off++;
                sig_key[row] = k[it];
                sig_cnt[row] = cn[it];
                sig_slot[row] = (unsigned int)slot;
                I.tab[slot].aux = (unsigned int)row;
            }
        }
        __syncthreads();
    }
}

// Exclusive prefix of the per-instance significant counts: sprefix[count] = total.
__global__ void __launch_bounds__(kScanBlock) k_batch_scan(const InstCounters* ctr, int count, long long* sprefix) {
    __shared__ unsigned int scratch[33];
    long long carry = 0;
    for (int t0 = 0; t0 < count; t0 += kScanBlock) {
        const int i = t0 + threadIdx.x;
        const unsigned long long v = i < count ? ctr[i].sig : 0ull;
        // counts fit in 32 bits per instance (n_i < 2^32); partial sums are widened below
        unsigned int tot;
        const unsigned int off = block_excl_scan((unsigned int)v, scratch, &tot);
        if (i < count) sprefix[i] = carry + off;
        carry += tot;
    }
    if (threadIdx.x == 0) sprefix[count] = carry;
}

struct RowRef {
    int inst;
    long long row;
};

__device__ __forceinline__ RowRef row_of(const BatchInst* __restrict__ inst, const long long* __restrict__ sprefix,
                                        int count, long long g) {
    const int i = find_segment(sprefix, count, g);
    return RowRef{i, inst[i].row_off + (g - sprefix[i])};
}

__global__ void k_batch_uf_init(const BatchInst* __restrict__ inst, const long long* __restrict__ sprefix, int count,
                                int* parent, unsigned int* csize, unsigned long long* cmin) {
    const long long total = sprefix[count];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        const long long row = row_of(inst, sprefix, count, g).row;
        parent[row] = (int)row;
        csize[row] = 0u;
        cmin[row] = ~0ull;
    }
}

__global__ void k_batch_hook(const BatchInst* __restrict__ inst, const long long* __restrict__ sprefix, int count,
                             const unsigned long long* __restrict__ sig_key, int* parent, InstCounters* ctr) {
    const long long total = sprefix[count];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        const RowRef rr = row_of(inst, sprefix, count, g);
        const BatchInst& I = inst[rr.inst];
        const Slot* tab = I.tab;
        const unsigned int mask = I.mask;
        const unsigned int tau = I.tau;
        const unsigned long long key = sig_key[rr.row];
        const long long x = key_x(key), y = key_y(key);
        unsigned long long nk[4];
        unsigned int ns[4];
        Slot sl[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long nx = x + (q < 3 ? 1 : 0);
            const long long ny = y + (q < 3 ? q - 1 : 1);
            const bool valid = !(nx > 2147483646ll || ny > 2147483646ll || ny < -2147483647ll);
            nk[q] = valid ? pack_key((int)nx, (int)ny) : kInvalidKey;
            ns[q] = tile_hash(nk[q]) & mask;
            if (valid)
                sl[q] = load_slot(&tab[ns[q]]);
            else
                sl[q].key = kEmptyKey;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (nk[q] == kInvalidKey) continue;
            const Slot nb = table_find_from(tab, mask, nk[q], ns[q], sl[q], mask + 1u);
            if (nb.key != nk[q] || nb.count < tau) continue;
            if (!uf_unite(parent, (int)rr.row, (int)nb.aux, I.union_limit))
                atomicOr(&ctr[rr.inst].status, (unsigned long long)kStInternal);
        }
    }
}

__global__ void k_batch_flatten(const BatchInst* __restrict__ inst, const long long* __restrict__ sprefix, int count,
                                int* parent) {
    const long long total = sprefix[count];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        const long long row = row_of(inst, sprefix, count, g).row;
        parent[row] = uf_root(parent, (int)row);
    }
}

__global__ void k_batch_stats(const BatchInst* __restrict__ inst, const long long* __restrict__ sprefix, int count,
                              const unsigned long long* __restrict__ sig_key, const int* __restrict__ parent,
                              unsigned int* csize, unsigned long long* cmin) {
    const long long total = sprefix[count];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        const long long row = row_of(inst, sprefix, count, g).row;
        const int r = parent[row];
        atomicAdd(&csize[r], 1u);
        atomicMin(&cmin[r], order_of(sig_key[row]));
    }
}

// Warp-uniform loop; kept rows are appended per instance with one atomic per
// (warp, instance) group.
__global__ void k_batch_emit(const BatchInst* __restrict__ inst, const long long* __restrict__ sprefix, int count,
                             const unsigned long long* __restrict__ sig_key, const unsigned int* __restrict__ sig_cnt,
                             const int* __restrict__ parent, const unsigned int* __restrict__ csize,
                             const unsigned long long* __restrict__ cmin, InstCounters* ctr,
                             unsigned long long* out_key, unsigned int* out_cnt, unsigned long long* out_cid) {
    const long long total = sprefix[count];
    const int lane = threadIdx.x & 31;
    const long long warps_total = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long w0 = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; w0 < total;
         w0 += warps_total * 32) {
        const long long g = w0 + lane;
        int inst_id = -1;
        long long row = 0;
        bool keep = false, root = false;
        int r = 0;
        if (g < total) {
            const RowRef rr = row_of(inst, sprefix, count, g);
            inst_id = rr.inst;
            row = rr.row;
            r = parent[row];
            keep = csize[r] >= inst[inst_id].mu;
            root = keep && r == (int)row;
        }
        const unsigned int lt = (1u << lane) - 1u;
        const unsigned int grp = __match_any_sync(0xFFFFFFFFu, keep ? inst_id : -1);
        const int leader = __ffs(grp) - 1;
        unsigned long long base = 0;
        if (keep && lane == leader) base = atomicAdd(&ctr[inst_id].kept, (unsigned long long)__popc(grp));
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
        if (keep) {
            const long long orow = inst[inst_id].row_off + (long long)base + __popc(grp & lt);
            out_key[orow] = sig_key[row];
            out_cnt[orow] = sig_cnt[row];
            out_cid[orow] = key_of_order(cmin[r]);
        }
        const unsigned int rg = __match_any_sync(0xFFFFFFFFu, root ? inst_id : -1);
        if (root && lane == __ffs(rg) - 1) atomicAdd(&ctr[inst_id].clusters, (unsigned long long)__popc(rg));
    }
}

}  // namespace
}  // namespace raster
