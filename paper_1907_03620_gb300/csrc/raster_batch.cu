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
#include "raster_segmented.cuh"

using namespace raster;

namespace {

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
    const TestLimits lim = test_limits();
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
        I.max_probe = lim.probe >= 0 ? (unsigned int)std::min<unsigned long long>((unsigned long long)lim.probe, cap)
                                     : (unsigned int)cap;
        I.union_limit = lim.unions >= 0 ? lim.unions : (1 << 30);
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
