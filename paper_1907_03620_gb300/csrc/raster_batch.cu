// Batched RASTER: thousands of independent instances in one graph launch.
//
// Every instance i has its own points, scale, tau, mu, tile table (a power of
// two of at least n_i / load slots, so it can never overflow: an instance has
// at most n_i tiles) and its own segment of the significant-tile and result
// arenas (at most n_i / tau_i rows: each significant tile holds tau_i points).
//
//   k_batch_fill      clear every table and counter
//   k_batch_contract  persistent: warps stride over uniform chunks of points;
//                     a chunk belongs to one instance (binary search over the
//                     chunk prefix), so projection parameters are warp-uniform
//   k_batch_select    per table chunk: compaction of tiles with count >= tau_i
//   k_batch_scan      prefix over the per-instance significant counts, which
//                     gives one compact index space for the kernels below
//   k_batch_uf_init / k_batch_hook / k_batch_flatten / k_batch_stats /
//   k_batch_emit      the agglomeration of raster_single.cu over that index
//                     space, each index mapped back to its instance
//
// The sequence is captured once into a CUDA graph and replayed per run.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/raster.h"
#include "raster_block.cuh"
#include "raster_device.cuh"
#include "raster_host.h"

using namespace raster;

namespace {

constexpr long long kChunkPoints = 2048;  // points per contraction work item
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
                    const int r = table_add(I.tab, I.mask, key, c_add, I.mask + 1u);
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
            if (!uf_unite(parent, (int)rr.row, (int)nb.aux, 1 << 30))
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

int grid_of(const void* kernel, int block) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0);
    return std::max(1, sms * std::max(1, per_sm));
}

using ContractFn = void (*)(const BatchInst*, const long long*, int, InstCounters*);

template <int W, bool P>
ContractFn contract_fn() {
    return k_batch_contract<W, P>;
}

ContractFn pick_contract(int width, bool preagg) {
    switch (width) {
        case 1: return preagg ? contract_fn<1, true>() : contract_fn<1, false>();
        case 2: return preagg ? contract_fn<2, true>() : contract_fn<2, false>();
        case 4: return preagg ? contract_fn<4, true>() : contract_fn<4, false>();
        default: return preagg ? contract_fn<8, true>() : contract_fn<8, false>();
    }
}

}  // namespace

struct raster_batch {
    int count = 0;
    raster_batch_config cfg{};
    std::vector<BatchInst> host_inst;
    std::vector<long long> row_cap;
    cudaStream_t capture_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t last_stream = nullptr;
    bool ran = false;
    // device
    BatchInst* d_inst = nullptr;
    long long* d_chunk = nullptr;
    long long* d_slot_chunk = nullptr;
    long long* d_sprefix = nullptr;
    InstCounters* d_ctr = nullptr;
    InstCounters* h_ctr = nullptr;  // pinned
    Slot* tab = nullptr;
    unsigned long long slots = 0;
    long long rows = 0;
    unsigned long long* sig_key = nullptr;
    unsigned int* sig_cnt = nullptr;
    unsigned int* sig_slot = nullptr;
    int* parent = nullptr;
    unsigned int* csize = nullptr;
    unsigned long long* cmin = nullptr;
    unsigned long long* out_key = nullptr;
    unsigned int* out_cnt = nullptr;
    unsigned long long* out_cid = nullptr;
    long long bytes = 0;
    int g_fill = 1, g_con = 1, g_sel = 1, g_agg = 1;  // grids, computed before capture
};

namespace {

int status_of_bits(unsigned long long bits) {
    if (bits & kStInternal) return RASTER_E_INTERNAL;
    if (bits & kStFull) return RASTER_E_TABLE_FULL;
    if (bits & kStRange) return RASTER_E_RANGE;
    return RASTER_OK;
}

template <typename T>
int dalloc(raster_batch* b, T** p, size_t n) {
    const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? RASTER_E_OOM : RASTER_E_CUDA;
    }
    b->bytes += (long long)bytes;
    return RASTER_OK;
}

int record(raster_batch* b, cudaStream_t s) {
    const int count = b->count;
    const int g_fill = b->g_fill, g_con = b->g_con, g_sel = b->g_sel, g_agg = b->g_agg;
    k_batch_fill<<<g_fill, 256, 0, s>>>(b->tab, b->slots, b->d_ctr, count);
    const int block = b->cfg.block;
    ContractFn fn = pick_contract(b->cfg.width, b->cfg.preagg != 0);
    fn<<<g_con, block, 0, s>>>(b->d_inst, b->d_chunk, count, b->d_ctr);
    k_batch_select<<<g_sel, kScanBlock, 0, s>>>(b->d_inst, b->d_slot_chunk, count, b->d_ctr, b->sig_key, b->sig_cnt,
                                               b->sig_slot);
    k_batch_scan<<<1, kScanBlock, 0, s>>>(b->d_ctr, count, b->d_sprefix);
    k_batch_uf_init<<<g_agg, kAggBlock, 0, s>>>(b->d_inst, b->d_sprefix, count, b->parent, b->csize, b->cmin);
    k_batch_hook<<<g_agg, kAggBlock, 0, s>>>(b->d_inst, b->d_sprefix, count, b->sig_key, b->parent, b->d_ctr);
    k_batch_flatten<<<g_agg, kAggBlock, 0, s>>>(b->d_inst, b->d_sprefix, count, b->parent);
    k_batch_stats<<<g_agg, kAggBlock, 0, s>>>(b->d_inst, b->d_sprefix, count, b->sig_key, b->parent, b->csize,
                                             b->cmin);
    k_batch_emit<<<g_agg, kAggBlock, 0, s>>>(b->d_inst, b->d_sprefix, count, b->sig_key, b->sig_cnt, b->parent,
                                            b->csize, b->cmin, b->d_ctr, b->out_key, b->out_cnt, b->out_cid);
    if (cudaMemcpyAsync(b->h_ctr, b->d_ctr, sizeof(InstCounters) * (size_t)std::max(count, 1), cudaMemcpyDeviceToHost,
                        s) != cudaSuccess)
        return RASTER_E_CUDA;
    return cudaGetLastError() == cudaSuccess ? RASTER_OK : RASTER_E_CUDA;
}

}  // namespace

extern "C" {

int raster_batch_destroy(raster_batch* b) {
    if (!b) return RASTER_E_ARG;
    if (b->last_stream) cudaStreamSynchronize(b->last_stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    void* bufs[] = {b->d_inst, b->d_chunk, b->d_slot_chunk, b->d_sprefix, b->d_ctr, b->tab,     b->sig_key,
                    b->sig_cnt, b->sig_slot, b->parent,     b->csize,     b->cmin,  b->out_key, b->out_cnt,
                    b->out_cid};
    for (void* p : bufs)
        if (p) cudaFree(p);
    if (b->h_ctr) cudaFreeHost(b->h_ctr);
    delete b;
    return RASTER_OK;
}

int raster_batch_create(const raster_instance* inst, int32_t count, const raster_batch_config* cfg,
                        raster_batch** out) {
    if (!out || count < 0 || (count > 0 && !inst)) return RASTER_E_ARG;
    *out = nullptr;
    raster_batch_config c{0.75, 256, 4, 1};
    if (cfg) {
        if (cfg->load > 0.0) c.load = cfg->load;
        if (cfg->block > 0) c.block = cfg->block;
        if (cfg->width > 0) c.width = cfg->width;
        if (cfg->preagg >= 0) c.preagg = cfg->preagg;
    }
    if (!(c.load > 0.0 && c.load <= 0.75) || (c.block != 128 && c.block != 256 && c.block != 512) ||
        (c.width != 1 && c.width != 2 && c.width != 4 && c.width != 8) || (c.preagg != 0 && c.preagg != 1))
        return RASTER_E_ARG;
    raster_batch* b = new (std::nothrow) raster_batch();
    if (!b) return RASTER_E_OOM;
    b->count = count;
    b->cfg = c;
    b->host_inst.resize(count);
    b->row_cap.resize(count);
    std::vector<long long> chunk(count + 1, 0), slot_chunk(count + 1, 0);
    std::vector<unsigned long long> tab_off(count, 0);
    long long rows = 0;
    unsigned long long slots = 0;
    for (int i = 0; i < count; ++i) {
        const raster_instance& r = inst[i];
        if (r.n < 0 || r.n > 0xFFFFFFFFll || r.tau == 0 || r.mu == 0 || !std::isfinite(r.precision) ||
            (r.n > 0 && (!r.xy || ((uintptr_t)r.xy & 15u)))) {
            delete b;
            return RASTER_E_ARG;
        }
        BatchInst& I = b->host_inst[i];
        bool wide = false;
        if (make_proj_params(scale_of_precision(r.precision), &I.pp, &wide) != RASTER_OK) {
            delete b;
            return RASTER_E_ARG;
        }
        I.wide = wide ? 1u : 0u;
        I.xy = reinterpret_cast<const double2*>(r.xy);
        I.n = r.n;
        I.tau = r.tau;
        I.mu = r.mu;
        unsigned long long cap = kMinTable;
        while ((double)cap * c.load < (double)r.n) cap <<= 1;
        if (cap > (1ull << 31)) {
            delete b;
            return RASTER_E_ARG;
        }
        I.mask = (unsigned int)(cap - 1);
        tab_off[i] = slots;
        slots += cap;
        const long long rc = std::max<long long>(1, r.n / (long long)r.tau);
        b->row_cap[i] = rc;
        I.row_off = rows;
        rows += rc;
        chunk[i + 1] = chunk[i] + (r.n + kChunkPoints - 1) / kChunkPoints;
        slot_chunk[i + 1] = slot_chunk[i] + (long long)(cap / kSlotChunk);
    }
    if (rows >= 0x7FFFFFFFll) {
        delete b;
        return RASTER_E_ARG;
    }
    b->slots = slots;
    b->rows = rows;
    int rc = RASTER_OK;
    const size_t nI = (size_t)std::max(count, 1);
    if (!rc) rc = dalloc(b, &b->tab, slots);
    if (!rc) rc = dalloc(b, &b->d_inst, nI);
    if (!rc) rc = dalloc(b, &b->d_chunk, (size_t)count + 1);
    if (!rc) rc = dalloc(b, &b->d_slot_chunk, (size_t)count + 1);
    if (!rc) rc = dalloc(b, &b->d_sprefix, (size_t)count + 1);
    if (!rc) rc = dalloc(b, &b->d_ctr, nI);
    if (!rc) rc = dalloc(b, &b->sig_key, (size_t)rows);
    if (!rc) rc = dalloc(b, &b->sig_cnt, (size_t)rows);
    if (!rc) rc = dalloc(b, &b->sig_slot, (size_t)rows);
    if (!rc) rc = dalloc(b, &b->parent, (size_t)rows);
    if (!rc) rc = dalloc(b, &b->csize, (size_t)rows);
    if (!rc) rc = dalloc(b, &b->cmin, (size_t)rows);
    if (!rc) rc = dalloc(b, &b->out_key, (size_t)rows);
    if (!rc) rc = dalloc(b, &b->out_cnt, (size_t)rows);
    if (!rc) rc = dalloc(b, &b->out_cid, (size_t)rows);
    if (!rc && cudaMallocHost(&b->h_ctr, sizeof(InstCounters) * nI) != cudaSuccess) rc = RASTER_E_OOM;
    if (rc) {
        raster_batch_destroy(b);
        return rc;
    }
    for (int i = 0; i < count; ++i) b->host_inst[i].tab = b->tab + tab_off[i];
    std::memset(b->h_ctr, 0, sizeof(InstCounters) * nI);
    if (cudaMemcpy(b->d_inst, b->host_inst.data(), sizeof(BatchInst) * (size_t)count, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(b->d_chunk, chunk.data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_slot_chunk, slot_chunk.data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        raster_batch_destroy(b);
        return RASTER_E_CUDA;
    }
    b->g_fill = grid_of((const void*)k_batch_fill, 256);
    b->g_con = grid_of((const void*)pick_contract(c.width, c.preagg != 0), c.block);
    b->g_sel = grid_of((const void*)k_batch_select, kScanBlock);
    b->g_agg = grid_of((const void*)k_batch_hook, kAggBlock);
    // capture the whole run once
    if (cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        raster_batch_destroy(b);
        return RASTER_E_CUDA;
    }
    rc = record(b, b->capture_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->capture_stream, &g);
    b->graph = g;
    if (rc || ec != cudaSuccess || cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
        cudaGetLastError();
        raster_batch_destroy(b);
        return rc ? rc : RASTER_E_CUDA;
    }
    *out = b;
    return RASTER_OK;
}

int raster_batch_run(raster_batch* b, void* stream) {
    if (!b) return RASTER_E_ARG;
    b->last_stream = (cudaStream_t)stream;
    if (cudaGraphLaunch(b->exec, b->last_stream) != cudaSuccess) return RASTER_E_CUDA;
    note_launch(9);
    b->ran = true;
    return RASTER_OK;
}

int raster_batch_wait(raster_batch* b) {
    if (!b) return RASTER_E_ARG;
    if (!b->ran) return RASTER_E_STATE;
    if (cudaStreamSynchronize(b->last_stream) != cudaSuccess) return RASTER_E_CUDA;
    int worst = RASTER_OK;
    for (int i = 0; i < b->count; ++i) {
        const int s = status_of_bits(b->h_ctr[i].status);
        if (s != RASTER_OK && (worst == RASTER_OK || worst == RASTER_E_RANGE)) worst = s;
    }
    return worst;
}

int raster_batch_result(raster_batch* b, int32_t i, raster_clusters* out) {
    if (!b || !out || i < 0 || i >= b->count) return RASTER_E_ARG;
    if (!b->ran) return RASTER_E_STATE;
    const InstCounters& c = b->h_ctr[i];
    const long long off = b->host_inst[i].row_off;
    out->key = reinterpret_cast<const int64_t*>(b->out_key + off);
    out->count = b->out_cnt + off;
    out->cid = reinterpret_cast<const int64_t*>(b->out_cid + off);
    out->n_tiles = (int64_t)c.kept;
    out->n_clusters = (int64_t)c.clusters;
    out->n_distinct = (int64_t)c.tiles;
    out->n_significant = (int64_t)c.sig;
    out->n_points = (int64_t)b->host_inst[i].n;
    return status_of_bits(c.status);
}

int64_t raster_batch_device_bytes(const raster_batch* b) { return b ? b->bytes : 0; }

}  // extern "C"
