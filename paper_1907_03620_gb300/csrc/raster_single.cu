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

using namespace raster;

namespace {

constexpr int kBlock = 256;
constexpr int kContractUnroll = 4;
constexpr double kMaxLoad = 0.75;     // a launch never pushes the table beyond this load
constexpr double kGrowLoad = 0.7;     // target load after growing (before the next chunk)
constexpr long long kMinStep = 1 << 20;
constexpr long long kGrowStep = 64ll << 20;
constexpr int kUnionLimit = 1 << 30;

// ---------------------------------------------------------------------------
// Block helpers

// ---------------------------------------------------------------------------
// Kernels

__global__ void k_fill_table(Slot* tab, unsigned long long cap) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    ulonglong2 v;
    v.x = kEmptyKey;
    v.y = 0ull;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += stride)
        reinterpret_cast<ulonglong2*>(tab)[i] = v;
}

template <bool WIDE, int U>
__global__ void __launch_bounds__(kBlock) k_contract(const double2* __restrict__ xy, long long n, ProjParams pp,
                                                    Slot* tab, unsigned int mask, unsigned int max_probe,
                                                    unsigned long long* d_newkeys, unsigned int* d_status) {
    const int lane = threadIdx.x & 31;
    const long long warps_total = (long long)gridDim.x * (kBlock >> 5);
    const long long per_warp = 32ll * U;
    unsigned int newk = 0, st = 0;
    for (long long base = ((long long)blockIdx.x * (kBlock >> 5) + (threadIdx.x >> 5)) * per_warp; base < n;
         base += warps_total * per_warp) {
        double2 p[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long i = base + u * 32 + lane;
            if (i < n) p[u] = __ldcs(xy + i);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long i = base + u * 32 + lane;
            unsigned long long key = kInvalidKey;
            if (i < n) {
                key = project_point<WIDE>(p[u].x, p[u].y, pp);
                if (key == kInvalidKey) st |= kStRange;
            }
            const unsigned int grp = __match_any_sync(0xFFFFFFFFu, key);
            if (lane == __ffs(grp) - 1 && key != kInvalidKey) {
                const int r = table_add(tab, mask, key, (unsigned int)__popc(grp), max_probe);
                if (r > 0)
                    ++newk;
                else if (r < 0)
                    st |= kStFull;
            }
        }
    }
    flush_counts(newk, st, d_newkeys, d_status);
}

__global__ void k_rehash(const Slot* __restrict__ old_tab, unsigned long long old_cap, Slot* tab, unsigned int mask,
                         unsigned int max_probe, unsigned int* d_status) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned int st = 0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < old_cap; i += stride) {
        const Slot s = old_tab[i];
        if (s.key != kEmptyKey && table_add(tab, mask, s.key, s.count, max_probe) < 0) st |= kStFull;
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
                                                  int write_aux) {
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
            if (idx < cap) {
                const ulonglong2 v = __ldcs(reinterpret_cast<const ulonglong2*>(tab) + idx);
                k[it] = v.x;
                c[it] = (unsigned int)v.y;
            }
            if (k[it] != kEmptyKey && c[it] >= min_count) flags |= 1u << it;
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
                out_key[row] = k[it];
                out_cnt[row] = c[it];
                if (out_slot) out_slot[row] = (unsigned int)idx;
                if (write_aux) tab[idx].aux = (unsigned int)row;
            }
        }
        __syncthreads();
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

__global__ void k_hook(const unsigned long long* d_nsig, const unsigned long long* __restrict__ sig_key,
                       const Slot* __restrict__ tab, unsigned int mask, unsigned int max_probe, unsigned int tau,
                       int* parent, unsigned int* d_status) {
    const long long S = (long long)*d_nsig;
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned int st = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += stride) {
        const unsigned long long key = __ldcs(sig_key + i);
        const long long x = key_x(key), y = key_y(key);
        // forward neighbours: (x+1, y-1), (x+1, y), (x+1, y+1), (x, y+1); their
        // first probes are issued together
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
            if (valid) sl[q] = load_slot(&tab[ns[q]]);
            else sl[q].key = kEmptyKey;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (nk[q] == kInvalidKey) continue;
            const Slot nb = table_find_from(tab, mask, nk[q], ns[q], sl[q], max_probe);
            if (nb.key != nk[q] || nb.count < tau) continue;
            if (!uf_unite(parent, (int)i, (int)nb.aux, kUnionLimit)) st |= kStInternal;
        }
    }
    if (st) atomicOr(d_status, st);
}

__global__ void k_flatten(const unsigned long long* d_nsig, int* parent) {
    const long long S = (long long)*d_nsig;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += stride)
        parent[i] = uf_root(parent, (int)i);
}

__global__ void k_stats(const unsigned long long* d_nsig, const unsigned long long* __restrict__ sig_key,
                        const int* __restrict__ parent, unsigned int* csize, unsigned long long* cmin) {
    const long long S = (long long)*d_nsig;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += stride) {
        const int r = parent[i];
        atomicAdd(&csize[r], 1u);
        atomicMin(&cmin[r], order_of(sig_key[i]));
    }
}

__global__ void __launch_bounds__(kBlock) k_emit(const unsigned long long* d_nsig,
                                                const unsigned long long* __restrict__ sig_key,
                                                const unsigned int* __restrict__ sig_cnt,
                                                const unsigned int* __restrict__ sig_slot,
                                                const int* __restrict__ parent, const unsigned int* __restrict__ csize,
                                                const unsigned long long* __restrict__ cmin, unsigned int mu,
                                                Slot* tab, unsigned long long* out_key, unsigned int* out_cnt,
                                                unsigned long long* out_cid, unsigned long long* d_nkept,
                                                unsigned long long* d_nclusters) {
    __shared__ unsigned int scratch[33];
    __shared__ unsigned long long s_base;
    const long long S = (long long)*d_nsig;
    unsigned int clusters = 0;
    for (long long t0 = (long long)blockIdx.x * kBlock; t0 < S; t0 += (long long)gridDim.x * kBlock) {
        const long long i = t0 + threadIdx.x;
        bool keep = false;
        unsigned long long key = 0, cid = 0;
        int r = 0;
        if (i < S) {
            r = parent[i];
            keep = csize[r] >= mu;
            key = sig_key[i];
            cid = key_of_order(cmin[r]);
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
                code = label_code(key, cid, (unsigned int)row);
            }
            tab[sig_slot[i]].aux = code;
        }
        __syncthreads();
    }
    clusters = __reduce_add_sync(0xFFFFFFFFu, clusters);
    if ((threadIdx.x & 31) == 0 && clusters) atomicAdd(d_nclusters, (unsigned long long)clusters);
}

template <bool WIDE>
__global__ void k_labels(const double2* __restrict__ xy, long long n, ProjParams pp, const Slot* __restrict__ tab,
                         unsigned int mask, unsigned int max_probe, unsigned int tau,
                         const long long* __restrict__ cid_rows, long long* __restrict__ labels,
                         unsigned int* d_status) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned int st = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double2 p = __ldcs(xy + i);
        const unsigned long long key = project_point<WIDE>(p.x, p.y, pp);
        long long lab = (long long)kEmptyKey;
        if (key == kInvalidKey) {
            st |= kStRange;
        } else {
            const long long s = table_find(tab, mask, key, max_probe);
            if (s >= 0) {
                const Slot sl = tab[s];
                if (sl.count >= tau) lab = label_decode(key, sl.aux, cid_rows);
            }
        }
        __stcs(labels + i, lab);
    }
    if (st) atomicOr(d_status, st);
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
    ProjParams pp{};
    bool wide = false;
    cudaStream_t stream = nullptr;
    int status = RASTER_OK;  // sticky
    enum { kContracting, kAgglomerated } state = kContracting;

    Slot* tab = nullptr;
    unsigned long long cap = 0;  // power of two
    long long d_bound = 0;       // upper bound on distinct tiles
    long long points = 0;        // points submitted (incl. invalid ones)

    // device counters: [0] new keys (D), [1] significant (S), [2] kept rows,
    // [3] clusters, [4] export rows
    unsigned long long* d_ctr = nullptr;
    unsigned int* d_status = nullptr;
    unsigned long long* h_ctr = nullptr;  // pinned mirror (5 counters + status)

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
    raster_clusters result{};

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
    return (unsigned int)std::min<unsigned long long>(cap, 1ull << 22);
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
    RCHECK(h, cudaMemcpyAsync(h->h_ctr, h->d_ctr, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
    RCHECK(h, cudaMemcpyAsync(h->h_ctr + 5, h->d_status, sizeof(unsigned int), cudaMemcpyDeviceToHost, h->stream));
    RCHECK(h, cudaStreamSynchronize(h->stream));
    merge_status(h, status_from_bits((unsigned int)h->h_ctr[5]));
    return RASTER_OK;
}

// Replace the table by one of capacity new_cap, re-inserting every tile.
int grow_table(raster_handle* h, unsigned long long new_cap) {
    Slot* nt = nullptr;
    RCHECK(h, cudaMalloc(&nt, new_cap * sizeof(Slot)));
    int rc = fill_table(h, nt, new_cap, h->stream);
    if (rc) {
        cudaFree(nt);
        return rc;
    }
    if (h->tab && h->cap) {
        static int grid = grid_for((const void*)k_rehash, kBlock);
        k_rehash<<<grid, kBlock, 0, h->stream>>>(h->tab, h->cap, nt, (unsigned int)(new_cap - 1),
                                                 max_probe_for(new_cap), h->d_status);
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
    return RASTER_OK;
}

unsigned long long pow2_at_least(double v) {
    unsigned long long c = 1ull << 12;
    while ((double)c < v) c <<= 1;
    return c;
}

int ensure_room(raster_handle* h, long long want, long long* room_out) {
    long long room = (long long)((double)h->cap * kMaxLoad) - h->d_bound;
    if (room >= std::min(want, kMinStep) && room > 0) {
        *room_out = room;
        return RASTER_OK;
    }
    int rc = read_counters(h);
    if (rc) return rc;
    h->d_bound = (long long)h->h_ctr[0];
    room = (long long)((double)h->cap * kMaxLoad) - h->d_bound;
    if (room < std::min(want, kMinStep) || room <= 0) {
        const double need = (double)(h->d_bound + std::min(want, kGrowStep)) / kGrowLoad;
        const unsigned long long nc = std::max(pow2_at_least(need), 2 * h->cap);
        if (nc > (1ull << 31)) return RASTER_E_OOM;  // 32-bit slot indices
        rc = grow_table(h, nc);
        if (rc) return rc;
        room = (long long)((double)h->cap * kMaxLoad) - h->d_bound;
    }
    *room_out = room;
    return RASTER_OK;
}

template <bool WIDE>
void launch_contract(raster_handle* h, const double* xy, long long n) {
    static int grid = grid_for((const void*)k_contract<WIDE, kContractUnroll>, kBlock);
    const long long per_block = (long long)kBlock * kContractUnroll;
    const long long need = (n + per_block - 1) / per_block;
    const int g = (int)std::max<long long>(1, std::min<long long>(grid, need));
    k_contract<WIDE, kContractUnroll><<<g, kBlock, 0, h->stream>>>(
        reinterpret_cast<const double2*>(xy), n, h->pp, h->tab, (unsigned int)(h->cap - 1), max_probe_for(h->cap),
        h->d_ctr, h->d_status);
    note_launch();
}

int contract_device(raster_handle* h, const double* xy, long long n) {
    long long off = 0;
    while (off < n) {
        long long room = 0;
        int rc = ensure_room(h, n - off, &room);
        if (rc) return rc;
        const long long m = std::min(n - off, room);
        if (h->wide)
            launch_contract<true>(h, xy + 2 * off, m);
        else
            launch_contract<false>(h, xy + 2 * off, m);
        RCHECK(h, cudaGetLastError());
        h->d_bound += m;
        off += m;
    }
    return RASTER_OK;
}

int ensure_agg_capacity(raster_handle* h, long long rows) {
    if (rows <= h->agg_cap) return RASTER_OK;
    const long long cap = std::max<long long>(rows + rows / 4, 1 << 16);
    void** bufs[] = {(void**)&h->sig_key, (void**)&h->sig_cnt, (void**)&h->sig_slot, (void**)&h->parent,
                     (void**)&h->csize,   (void**)&h->cmin,    (void**)&h->out_key,  (void**)&h->out_cnt,
                     (void**)&h->out_cid};
    const size_t sizes[] = {8, 4, 4, 4, 4, 8, 8, 4, 8};
    RCHECK(h, cudaStreamSynchronize(h->stream));
    for (int i = 0; i < 9; ++i) {
        if (*bufs[i]) cudaFree(*bufs[i]);
        *bufs[i] = nullptr;
    }
    h->agg_cap = 0;
    for (int i = 0; i < 9; ++i) RCHECK(h, cudaMalloc(bufs[i], (size_t)cap * sizes[i]));
    h->agg_cap = cap;
    return RASTER_OK;
}

int ensure_stage(raster_handle* h) {
    if (h->stage_points) return RASTER_OK;
    const long long pts = 16ll << 20;  // 16M points = 256 MiB of xy per buffer
    RCHECK(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
        RCHECK(h, cudaMalloc(&h->stage_xy[b], (size_t)pts * 16));
        RCHECK(h, cudaMalloc(&h->stage_lab[b], (size_t)pts * 8));
        RCHECK(h, cudaEventCreateWithFlags(&h->ev_copied[b], cudaEventDisableTiming));
        RCHECK(h, cudaEventCreateWithFlags(&h->ev_done[b], cudaEventDisableTiming));
    }
    h->stage_points = pts;
    return RASTER_OK;
}

bool misaligned(const void* p) { return ((uintptr_t)p & 15u) != 0; }

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
    if (!out || tau == 0 || mu == 0 || !std::isfinite(precision)) return RASTER_E_ARG;
    *out = nullptr;
    raster_handle* h = new (std::nothrow) raster_handle();
    if (!h) return RASTER_E_OOM;
    h->precision = precision;
    h->scale = scale_of_precision(precision);
    h->tau = tau;
    h->mu = mu;
    if (make_proj_params(h->scale, &h->pp, &h->wide) != RASTER_OK) {
        delete h;
        return RASTER_E_ARG;
    }
    cudaError_t e = cudaMalloc(&h->d_ctr, 5 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_status, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMallocHost(&h->h_ctr, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(h->d_ctr, 0, 5 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(unsigned int));
    if (e != cudaSuccess) {
        raster_destroy(h);
        return e == cudaErrorMemoryAllocation ? RASTER_E_OOM : RASTER_E_CUDA;
    }
    int rc = grow_table(h, 1ull << 16);
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
    const unsigned long long nc = pow2_at_least((double)std::max<long long>(n_tiles, h->d_bound) / kGrowLoad);
    if (nc > (1ull << 31)) return RASTER_E_OOM;
    if (nc <= h->cap) return RASTER_OK;
    return grow_table(h, nc);
}

int raster_contract(raster_handle* h, const double* xy, int64_t n, void* stream) {
    if (!h || n < 0 || (n > 0 && (!xy || misaligned(xy)))) return RASTER_E_ARG;
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
    long long off = 0;
    for (int c = 0; off < n; ++c) {
        const int b = c & 1;
        const long long m = std::min(n - off, h->stage_points);
        RCHECK(h, cudaStreamWaitEvent(h->copy_stream, h->ev_done[b], 0));
        RCHECK(h, cudaMemcpyAsync(h->stage_xy[b], xy_host + 2 * off, (size_t)m * 16, cudaMemcpyHostToDevice,
                                  h->copy_stream));
        RCHECK(h, cudaEventRecord(h->ev_copied[b], h->copy_stream));
        RCHECK(h, cudaStreamWaitEvent(h->stream, h->ev_copied[b], 0));
        rc = contract_device(h, h->stage_xy[b], m);
        if (rc) return rc;
        RCHECK(h, cudaEventRecord(h->ev_done[b], h->stream));
        off += m;
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
    rc = ensure_agg_capacity(h, std::max<long long>(D, 1));
    if (rc) return rc;
    cudaStream_t s = h->stream;
    RCHECK(h, cudaMemsetAsync(h->d_ctr + 1, 0, 4 * sizeof(unsigned long long), s));
    unsigned long long* d_nsig = h->d_ctr + 1;
    static int g_sel = grid_for((const void*)k_select, kBlock);
    k_select<<<g_sel, kBlock, 0, s>>>(h->tab, h->cap, h->tau, h->sig_key, h->sig_cnt, h->sig_slot, d_nsig, 1);
    note_launch();
    RCHECK(h, cudaGetLastError());
    static int g_init = grid_for((const void*)k_uf_init, kBlock);
    static int g_hook = grid_for((const void*)k_hook, kBlock);
    static int g_flat = grid_for((const void*)k_flatten, kBlock);
    static int g_stat = grid_for((const void*)k_stats, kBlock);
    static int g_emit = grid_for((const void*)k_emit, kBlock);
    const int lim = (int)std::max<long long>(1, (D + kBlock - 1) / kBlock);
    k_uf_init<<<std::min(g_init, lim), kBlock, 0, s>>>(d_nsig, h->parent, h->csize, h->cmin);
    k_hook<<<std::min(g_hook, lim), kBlock, 0, s>>>(d_nsig, h->sig_key, h->tab, (unsigned int)(h->cap - 1),
                                                    max_probe_for(h->cap), h->tau, h->parent, h->d_status);
    k_flatten<<<std::min(g_flat, lim), kBlock, 0, s>>>(d_nsig, h->parent);
    k_stats<<<std::min(g_stat, lim), kBlock, 0, s>>>(d_nsig, h->sig_key, h->parent, h->csize, h->cmin);
    k_emit<<<std::min(g_emit, lim), kBlock, 0, s>>>(d_nsig, h->sig_key, h->sig_cnt, h->sig_slot, h->parent, h->csize,
                                                    h->cmin, h->mu, h->tab, h->out_key, h->out_cnt, h->out_cid,
                                                    h->d_ctr + 2, h->d_ctr + 3);
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
    if (!h || n < 0 || (n > 0 && (!xy || !labels || misaligned(xy)))) return RASTER_E_ARG;
    if (hard_error(h->status)) return h->status;
    if (h->state != raster_handle::kAgglomerated) return RASTER_E_STATE;
    h->stream = (cudaStream_t)stream;
    if (n == 0) return RASTER_OK;
    if (h->wide) {
        static int grid = grid_for((const void*)k_labels<true>, kBlock);
        k_labels<true><<<(int)std::min<long long>(grid, (n + kBlock - 1) / kBlock), kBlock, 0, h->stream>>>(
            reinterpret_cast<const double2*>(xy), n, h->pp, h->tab, (unsigned int)(h->cap - 1),
            max_probe_for(h->cap), h->tau, reinterpret_cast<const long long*>(h->out_cid),
            reinterpret_cast<long long*>(labels), h->d_status);
    } else {
        static int grid = grid_for((const void*)k_labels<false>, kBlock);
        k_labels<false><<<(int)std::min<long long>(grid, (n + kBlock - 1) / kBlock), kBlock, 0, h->stream>>>(
            reinterpret_cast<const double2*>(xy), n, h->pp, h->tab, (unsigned int)(h->cap - 1),
            max_probe_for(h->cap), h->tau, reinterpret_cast<const long long*>(h->out_cid),
            reinterpret_cast<long long*>(labels), h->d_status);
    }
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
        RCHECK(h, cudaMemcpyAsync(h->stage_xy[b], xy_host + 2 * off, (size_t)m * 16, cudaMemcpyHostToDevice,
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

int raster_export_tiles(raster_handle* h, int64_t* key, uint32_t* count, int64_t capacity, int64_t* n_out) {
    if (!h || !n_out || capacity < 0) return RASTER_E_ARG;
    if (hard_error(h->status)) return h->status;
    int rc = read_counters(h);
    if (rc) return rc;
    const long long D = (long long)h->h_ctr[0];
    *n_out = D;
    if (capacity < D || (D > 0 && (!key || !count))) return RASTER_E_ARG;
    RCHECK(h, cudaMemsetAsync(h->d_ctr + 4, 0, sizeof(unsigned long long), h->stream));
    static int g_sel = grid_for((const void*)k_select, kBlock);
    k_select<<<g_sel, kBlock, 0, h->stream>>>(h->tab, h->cap, 1u, reinterpret_cast<unsigned long long*>(key), count,
                                              nullptr, h->d_ctr + 4, 0);
    note_launch();
    RCHECK(h, cudaGetLastError());
    return read_counters(h);
}

int raster_reset(raster_handle* h, void* stream) {
    if (!h) return RASTER_E_ARG;
    h->stream = (cudaStream_t)stream;
    if (h->status == RASTER_E_CUDA) {
        // a failed CUDA call may have left the context unusable; try anyway
        cudaGetLastError();
    }
    int rc = fill_table(h, h->tab, h->cap, h->stream);
    if (rc) return rc;
    RCHECK(h, cudaMemsetAsync(h->d_ctr, 0, 5 * sizeof(unsigned long long), h->stream));
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
                    h->stage_lab[0], h->stage_lab[1]};
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
