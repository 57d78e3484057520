// Tile counting without any allocation: raster_count_tiles_static.
//
// Some callers cannot allocate device memory at all: code running inside
// another runtime's memory pool or under a strict memory budget, plugins
// whose host application owns every allocation, or code paths that must not
// trigger the allocator's implicit device synchronisation.  For them this
// entry point counts the points per tile (the contraction of RASTER) with its
// hash table held in a fixed array of device memory that is part of the
// library image itself.  The caller passes the points and the output rows;
// the library calls no cudaMalloc, cudaFree or other allocating routine.
//
// Limits and sharing:
//   * the fixed array is 16 MiB (2^20 table slots of 16 bytes, plus counters),
//     so a call accepts at most RASTER_STATIC_MAX_POINTS = 2^19 points (the
//     table then stays at most half full); larger inputs are rejected with
//     RASTER_E_LIMIT;
//   * every GPU that loads the library holds this array until the process
//     exits;
//   * all calls share the one array: each call clears it first, and calls
//     whose GPU work overlaps (different streams, or several host threads)
//     race on it and must be serialised by the caller.
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/raster.h"
#include "raster_device.cuh"
#include "raster_host.h"

using namespace raster;

namespace {

constexpr unsigned long long kStaticSlots = 1ull << 20;
constexpr int kStaticBlock = 256;
constexpr int kMaxDevices = 64;

// Scratch: the slot array, then the counters (new keys, status, output rows).
struct StaticCounters {
    unsigned long long new_keys;
    unsigned int status;
    unsigned int pad;
    unsigned long long rows;
};
constexpr size_t kStaticBytes = kStaticSlots * sizeof(Slot) + 256;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

struct StaticScratch {
    Slot* slots;
    StaticCounters* ctr;
};

std::mutex g_setup_lock;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Address of the device array for the current device (set up once per device
// with that device current).  In host code g_static_scratch is only a
// stand-in symbol, so its address must come from the runtime.
int scratch_for_current_device(StaticScratch* out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RASTER_E_CUDA;
    std::lock_guard<std::mutex> g(g_setup_lock);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return RASTER_E_CUDA;
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    out->slots = reinterpret_cast<Slot*>(g_scratch_ptr[dev]);
    out->ctr = reinterpret_cast<StaticCounters*>(g_scratch_ptr[dev] + kStaticSlots * sizeof(Slot));
    return RASTER_OK;
}

__global__ void k_static_clear(StaticScratch sc) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    ulonglong2 v;
    v.x = kEmptyKey;
    v.y = 0ull;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < kStaticSlots;
         i += stride)
        reinterpret_cast<ulonglong2*>(sc.slots)[i] = v;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc.ctr->new_keys = 0ull;
        sc.ctr->status = 0u;
        sc.ctr->rows = 0ull;
    }
}

// The contraction kernel's variant on the fixed table: project, merge equal
// tiles within the warp, add to the table.
template <bool WIDE>
__global__ void __launch_bounds__(kStaticBlock) k_static_contract(const double2* __restrict__ xy, long long n,
                                                                ProjParams pp, StaticScratch sc) {
    const int lane = threadIdx.x & 31;
    const long long warps_total = (long long)gridDim.x * (kStaticBlock >> 5);
    unsigned int newk = 0, st = 0;
    for (long long base = ((long long)blockIdx.x * (kStaticBlock >> 5) + (threadIdx.x >> 5)) * 32; base < n;
         base += warps_total * 32) {
        const long long i = base + lane;
        unsigned long long key = kInvalidKey;
        if (i < n) {
            const double2 p = __ldcs(xy + i);
            key = project_point<WIDE>(p.x, p.y, pp);
            if (key == kInvalidKey) st |= kStRange;
        }
        const unsigned int grp = __match_any_sync(0xFFFFFFFFu, key);
        if (lane == __ffs(grp) - 1 && key != kInvalidKey) {
            const int r = table_add(sc.slots, (unsigned int)(kStaticSlots - 1), key, (unsigned int)__popc(grp),
                                    (unsigned int)kStaticSlots);
            if (r > 0)
                ++newk;
            else if (r < 0)
                st |= kStFull;
        }
    }
    newk = __reduce_add_sync(0xFFFFFFFFu, newk);
    st = __reduce_or_sync(0xFFFFFFFFu, st);
    if (lane == 0) {
        if (newk) atomicAdd(&sc.ctr->new_keys, (unsigned long long)newk);
        if (st) atomicOr(&sc.ctr->status, st);
    }
}

// Occupied slots -> caller rows (key, count); order unspecified.
__global__ void k_static_emit(StaticScratch sc, long long* key_out, unsigned int* count_out) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < kStaticSlots;
         i += stride) {
        const Slot s = sc.slots[i];
        const bool occ = s.key != kEmptyKey;
        const unsigned int m = __ballot_sync(__activemask(), occ);
        if (!m) continue;
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(&sc.ctr->rows, (unsigned long long)__popc(m));
        base = __shfl_sync(__activemask(), base, leader);
        if (occ) {
            const unsigned long long row = base + __popc(m & ((1u << lane) - 1u));
            key_out[row] = (long long)s.key;
            count_out[row] = s.count;
        }
    }
}

}  // namespace

extern "C" int raster_count_tiles_static(const double* xy, int64_t n, double precision, int64_t* key_out,
                                         uint32_t* count_out, int64_t* n_tiles_out, void* stream) {
    if (n < 0 || !n_tiles_out || !std::isfinite(precision)) return RASTER_E_ARG;
    if (n > RASTER_STATIC_MAX_POINTS) return RASTER_E_LIMIT;
    if (n > 0 && (!xy || !key_out || !count_out || ((uintptr_t)xy & 15u) != 0)) return RASTER_E_ARG;
    ProjParams pp;
    bool wide = false;
    if (make_proj_params(scale_of_precision(precision), &pp, &wide) != RASTER_OK) return RASTER_E_ARG;
    StaticScratch sc;
    int rc = scratch_for_current_device(&sc);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    k_static_clear<<<256, kStaticBlock, 0, s>>>(sc);
    if (n > 0) {
        const int grid = (int)std::min<long long>(1024, (n + kStaticBlock - 1) / kStaticBlock);
        if (wide)
            k_static_contract<true><<<grid, kStaticBlock, 0, s>>>(reinterpret_cast<const double2*>(xy), n, pp, sc);
        else
            k_static_contract<false><<<grid, kStaticBlock, 0, s>>>(reinterpret_cast<const double2*>(xy), n, pp, sc);
        k_static_emit<<<256, kStaticBlock, 0, s>>>(sc, reinterpret_cast<long long*>(key_out), count_out);
    }
    note_launch(n > 0 ? 3 : 1);
    if (cudaGetLastError() != cudaSuccess) return RASTER_E_CUDA;
    unsigned long long rows = 0;
    unsigned int status = 0;
    if (cudaMemcpyAsync(&rows, &sc.ctr->rows, sizeof(rows), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&status, &sc.ctr->status, sizeof(status), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return RASTER_E_CUDA;
    *n_tiles_out = (int64_t)rows;
    if (status & kStFull) return RASTER_E_TABLE_FULL;
    if (status & kStRange) return RASTER_E_RANGE;
    return RASTER_OK;
}
