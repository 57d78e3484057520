// Serving engine: continuous batching of RASTER requests on one GPU.
//
// Clients submit requests (precision, tau, mu, total points, number of chunks)
// and push their chunks (device pointers) whenever they have them.  A worker
// thread runs steps.  Each step:
//   1. admits waiting requests in arrival order while free device memory
//      (cudaMemGetInfo, minus a reserve the caller sets) covers the pages the
//      request's tile table (>= n / 0.75 slots, so it cannot overflow) and its
//      result rows (n / tau) would add: admission by free HBM.  Tables and rows
//      live in address ranges reserved once and backed page by page, so the
//      engine holds only the memory of live requests;
//   2. launches ONE segmented contraction over every ready chunk of every
//      admitted request (each chunk adds into its own request's resident
//      table);
//   3. launches ONE segmented agglomeration (select, scan, union-find hooking,
//      flatten, stats, emit) for every request whose chunks are all in;
//   4. waits for the step and records completions; a finished request's
//      table pages are given back at once, its rows when the client releases
//      it.
// Requests that arrive while others run join the next step, so the work of
// many requests overlaps on the device; each request's result is exactly that
// of a separate handle (its table and rows are private to it).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/raster.h"
#include "raster_host.h"
#include "raster_segmented.cuh"
#include "raster_vmm.h"

using namespace raster;

namespace raster {
namespace {

__global__ void k_fill_ranges(Slot* arena, const unsigned long long* off, const unsigned long long* len, int count) {
    for (int r = blockIdx.y; r < count; r += gridDim.y) {
        Slot* t = arena + off[r];
        const unsigned long long n = len[r];
        ulonglong2 v;
        v.x = kEmptyKey;
        v.y = 0ull;
        for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (unsigned long long)gridDim.x * blockDim.x)
            reinterpret_cast<ulonglong2*>(t)[i] = v;
    }
}

}  // namespace
}  // namespace raster

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, capacity) with coalescing of freed ranges.
class RangeAllocator {
public:
    void init(unsigned long long capacity) {
        free_.clear();
        if (capacity) free_[0] = capacity;
        capacity_ = capacity;
    }
    bool alloc(unsigned long long n, unsigned long long align, unsigned long long* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            const unsigned long long start = (it->first + align - 1) / align * align;
            const unsigned long long end = it->first + it->second;
            if (start + n <= end) {
                const unsigned long long f0 = it->first;
                free_.erase(it);
                if (start > f0) free_[f0] = start - f0;
                if (start + n < end) free_[start + n] = end - (start + n);
                *off = start;
                used_ += n;
                return true;
            }
        }
        return false;
    }
    void release(unsigned long long off, unsigned long long n) {
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    unsigned long long capacity() const { return capacity_; }
    unsigned long long used() const { return used_; }

private:
    std::map<unsigned long long, unsigned long long> free_;
    unsigned long long capacity_ = 0, used_ = 0;
};

struct Chunk {
    const double* xy;
    long long n;
};

struct Request {
    long long id = 0;
    ProjParams pp{};
    bool wide = false;
    unsigned int tau = 1, mu = 1;
    long long n_total = 0;
    int n_chunks = 0;
    int pushed = 0, contracted = 0;
    long long pushed_points = 0;
    std::deque<Chunk> pending;
    enum State { kWaiting, kActive, kDone } state = kWaiting;
    unsigned long long tab_off = 0, cap = 0;
    unsigned long long row_off = 0, rows = 0;
    bool has_table = false, has_rows = false;  // ranges held in the arrays
    unsigned long long tiles = 0, status = 0;
    unsigned int max_probe = 0;  // probe bound of its table (its size unless a test lowered it)
    int union_limit = 1 << 30;
    InstCounters result{};
    Clock::time_point t_submit, t_done;
};

constexpr int kMaxStepItems = 8192;       // chunks (or finishing requests) per step
constexpr long long kMaxStepPoints = 256ll << 20;
constexpr double kServeLoad = 0.75;

struct DeviceStep {
    BatchInst* inst = nullptr;
    long long* prefix = nullptr;
    InstCounters* ctr = nullptr;
    long long* sprefix = nullptr;
    unsigned long long* fill_off = nullptr;
    unsigned long long* fill_len = nullptr;
};

struct HostStep {
    BatchInst* inst = nullptr;
    long long* prefix = nullptr;
    InstCounters* ctr = nullptr;
    unsigned long long* fill_off = nullptr;
    unsigned long long* fill_len = nullptr;
};

}  // namespace

struct raster_server {
    int device = 0;
    cudaStream_t stream = nullptr;
    VmDriver drv;
    // tile tables (16-byte slots) and the nine row arrays, each an address
    // range backed page by page
    VmArray tab_va;
    VmArray row_va[9];
    Slot* tab_arena = nullptr;
    long long row_capacity = 0;
    unsigned long long* sig_key = nullptr;
    unsigned int* sig_cnt = nullptr;
    unsigned int* sig_slot = nullptr;
    int* parent = nullptr;
    unsigned int* csize = nullptr;
    unsigned long long* cmin = nullptr;
    unsigned long long* out_key = nullptr;
    unsigned int* out_cnt = nullptr;
    unsigned long long* out_cid = nullptr;
    RangeAllocator tab_alloc, row_alloc;
    int max_active = 0;
    size_t reserve = 0;        // device memory admission leaves free
    size_t total_mem = 0;
    DeviceStep dc, da;  // contraction and agglomeration descriptors
    HostStep hc, ha;
    int g_fill = 1, g_con = 1, g_sel = 1, g_agg = 1;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::unordered_map<long long, Request*> reqs;
    std::deque<Request*> waiting;
    std::vector<Request*> active;  // admission order
    std::deque<Request*> completed;
    bool stop = false;
    int fatal = RASTER_OK;
    std::thread worker;

    long long steps = 0, points = 0, refused = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around each step's device work
    double gpu_ms = 0.0;
};

namespace {

int grid_for_kernel(const void* kernel, int block) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0);
    return std::max(1, sms * std::max(1, per_sm));
}

void table_rows_for(long long n, unsigned int tau, unsigned long long* cap, unsigned long long* rows) {
    unsigned long long c = kMinTable;
    while ((double)c * kServeLoad < (double)n) c <<= 1;
    *cap = c;
    *rows = (unsigned long long)std::max<long long>(1, n / (long long)tau);
}

// The nine row arrays, in the order of raster_server::row_va: sig_key,
// sig_cnt, sig_slot, parent, csize, cmin, out_key, out_cnt, out_cid.
constexpr size_t kRowElem[9] = {8, 4, 4, 4, 4, 8, 8, 4, 8};
constexpr size_t kRowBytes = 52;                 // their sum
constexpr size_t kTablePage = 32ull << 20;       // bytes per page of the table array
constexpr size_t kRowPageRows = 4ull << 20;      // rows per page of every row array
constexpr unsigned long long kMaxRows = 0x7FFFFFFEull;  // row indices are int32 in union-find
constexpr unsigned int kStOom = 8u;             // host-side status bit: refused for device memory
constexpr double kIdleTrimMs = 200.0;           // idle this long: give cached pages back

size_t free_device_memory() {
    size_t f = 0, t = 0;
    if (cudaMemGetInfo(&f, &t) != cudaSuccess) return 0;
    return f;
}

// Bytes of device memory that pinning a table range and a row range would add.
size_t new_bytes(const raster_server* s, unsigned long long toff, unsigned long long cap, unsigned long long roff,
                 unsigned long long rows) {
    size_t n = s->tab_va.need(toff * sizeof(Slot), (toff + cap) * sizeof(Slot));
    for (int a = 0; a < 9; ++a) n += s->row_va[a].need(roff * kRowElem[a], (roff + rows) * kRowElem[a]);
    return n;
}

void unpin_rows(raster_server* s, Request* r, int arrays = 9) {
    for (int a = 0; a < arrays; ++a) s->row_va[a].unpin(r->row_off * kRowElem[a], (r->row_off + r->rows) * kRowElem[a]);
}

// Map the pages of a request's table and rows; all or nothing.
bool pin_request(raster_server* s, Request* r) {
    if (s->tab_va.pin(r->tab_off * sizeof(Slot), (r->tab_off + r->cap) * sizeof(Slot)) != CUDA_SUCCESS) return false;
    for (int a = 0; a < 9; ++a) {
        if (s->row_va[a].pin(r->row_off * kRowElem[a], (r->row_off + r->rows) * kRowElem[a]) != CUDA_SUCCESS) {
            unpin_rows(s, r, a);
            s->tab_va.unpin(r->tab_off * sizeof(Slot), (r->tab_off + r->cap) * sizeof(Slot));
            return false;
        }
    }
    return true;
}

void free_table(raster_server* s, Request* r) {
    if (!r->has_table) return;
    s->tab_va.unpin(r->tab_off * sizeof(Slot), (r->tab_off + r->cap) * sizeof(Slot));
    s->tab_alloc.release(r->tab_off, r->cap);
    r->has_table = false;
}

void free_rows(raster_server* s, Request* r) {
    if (!r->has_rows) return;
    unpin_rows(s, r);
    s->row_alloc.release(r->row_off, r->rows);
    r->has_rows = false;
}

size_t trim_all(raster_server* s) {
    size_t n = s->tab_va.trim();
    for (auto& a : s->row_va) n += a.trim();
    return n;
}

size_t mapped_bytes(const raster_server* s) {
    size_t n = s->tab_va.mapped_bytes();
    for (const auto& a : s->row_va) n += a.mapped_bytes();
    return n;
}

// Admit the oldest waiting request if free device memory covers what it
// adds: 1 admitted, 0 it must wait, -1 it was refused (it could not fit even
// with no other request on the device).
int admit_front(raster_server* s) {
    Request* r = s->waiting.front();
    unsigned long long toff = 0, roff = 0;
    if (!s->tab_alloc.alloc(r->cap, kSlotChunk, &toff)) return 0;
    if (!s->row_alloc.alloc(r->rows, 1, &roff)) {
        s->tab_alloc.release(toff, r->cap);
        return 0;
    }
    r->tab_off = toff;
    r->row_off = roff;
    const size_t need = new_bytes(s, toff, r->cap, roff, r->rows);
    bool ok = need == 0 || free_device_memory() >= need + s->reserve;
    if (!ok && trim_all(s) > 0) ok = free_device_memory() >= need + s->reserve;
    if (ok) ok = pin_request(s, r);
    if (ok) {
        r->has_table = r->has_rows = true;
        return 1;
    }
    s->tab_alloc.release(toff, r->cap);
    s->row_alloc.release(roff, r->rows);
    if (!s->active.empty()) return 0;  // memory comes back as active requests finish
    // nothing on the device will give memory back: refuse the request
    s->waiting.pop_front();
    r->state = Request::kDone;
    r->result = InstCounters{};
    r->result.status = kStOom;
    r->t_done = Clock::now();
    s->completed.push_back(r);
    s->refused += 1;
    s->cv_done.notify_all();
    return -1;
}

BatchInst inst_of(const raster_server* s, const Request* r) {
    BatchInst I{};
    I.pp = r->pp;
    I.wide = r->wide ? 1u : 0u;
    I.tab = s->tab_arena + r->tab_off;
    I.mask = (unsigned int)(r->cap - 1);
    I.tau = r->tau;
    I.mu = r->mu;
    I.row_off = (long long)r->row_off;
    I.max_probe = r->max_probe;
    I.union_limit = r->union_limit;
    return I;
}

// One step; returns false when there was nothing to do.
bool run_step(raster_server* s) {
    std::vector<Request*> fills, finishing;
    std::vector<std::pair<Request*, Chunk>> work;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        // 1. admission in arrival order, by free device memory
        while (!s->waiting.empty() && (int)s->active.size() < s->max_active && (int)fills.size() < kMaxStepItems) {
            const int a = admit_front(s);
            if (a == 0) break;
            if (a < 0) continue;
            Request* r = s->waiting.front();
            r->state = Request::kActive;
            s->waiting.pop_front();
            s->active.push_back(r);
            fills.push_back(r);
        }
        // 2. ready chunks of admitted requests, oldest request first
        long long pts = 0;
        for (Request* r : s->active) {
            while (!r->pending.empty() && (int)work.size() < kMaxStepItems &&
                   (pts < kMaxStepPoints || work.empty())) {
                work.push_back({r, r->pending.front()});
                pts += r->pending.front().n;
                r->pending.pop_front();
            }
        }
        // 3. requests complete once every chunk is contracted (this step included)
        std::unordered_map<Request*, int> in_step;
        for (auto& w : work) in_step[w.first] += 1;
        for (Request* r : s->active) {
            const int done = r->contracted + (in_step.count(r) ? in_step[r] : 0);
            if (r->pushed == r->n_chunks && done == r->n_chunks && r->pending.empty() &&
                (int)finishing.size() < kMaxStepItems)
                finishing.push_back(r);
        }
    }
    if (fills.empty() && work.empty() && finishing.empty()) return false;
    cudaStream_t st = s->stream;
    cudaError_t e = cudaEventRecord(s->ev0, st);
    if (!fills.empty()) {
        const int nf = (int)fills.size();
        for (int i = 0; i < nf; ++i) {
            s->hc.fill_off[i] = fills[i]->tab_off;
            s->hc.fill_len[i] = fills[i]->cap;
        }
        e = cudaMemcpyAsync(s->dc.fill_off, s->hc.fill_off, sizeof(unsigned long long) * nf, cudaMemcpyHostToDevice, st);
        if (!e) e = cudaMemcpyAsync(s->dc.fill_len, s->hc.fill_len, sizeof(unsigned long long) * nf, cudaMemcpyHostToDevice, st);
        if (!e) {
            dim3 grid(64, (unsigned)std::min(nf, 1024));
            k_fill_ranges<<<grid, 256, 0, st>>>(s->tab_arena, s->dc.fill_off, s->dc.fill_len, nf);
            note_launch(1);
        }
    }
    const int nw = (int)work.size();
    if (!e && nw > 0) {
        s->hc.prefix[0] = 0;
        for (int i = 0; i < nw; ++i) {
            BatchInst I = inst_of(s, work[i].first);
            I.xy = reinterpret_cast<const double2*>(work[i].second.xy);
            I.n = work[i].second.n;
            s->hc.inst[i] = I;
            s->hc.prefix[i + 1] = s->hc.prefix[i] + (I.n + kChunkPoints - 1) / kChunkPoints;
        }
        e = cudaMemcpyAsync(s->dc.inst, s->hc.inst, sizeof(BatchInst) * nw, cudaMemcpyHostToDevice, st);
        if (!e) e = cudaMemcpyAsync(s->dc.prefix, s->hc.prefix, sizeof(long long) * (nw + 1), cudaMemcpyHostToDevice, st);
        if (!e) e = cudaMemsetAsync(s->dc.ctr, 0, sizeof(InstCounters) * nw, st);
        if (!e) {
            k_batch_contract<1, true><<<s->g_con, 256, 0, st>>>(s->dc.inst, s->dc.prefix, nw, s->dc.ctr);
            note_launch(1);
            e = cudaMemcpyAsync(s->hc.ctr, s->dc.ctr, sizeof(InstCounters) * nw, cudaMemcpyDeviceToHost, st);
        }
    }
    const int na = (int)finishing.size();
    if (!e && na > 0) {
        s->ha.prefix[0] = 0;
        for (int i = 0; i < na; ++i) {
            s->ha.inst[i] = inst_of(s, finishing[i]);
            s->ha.prefix[i + 1] = s->ha.prefix[i] + (long long)(finishing[i]->cap / kSlotChunk);
        }
        e = cudaMemcpyAsync(s->da.inst, s->ha.inst, sizeof(BatchInst) * na, cudaMemcpyHostToDevice, st);
        if (!e) e = cudaMemcpyAsync(s->da.prefix, s->ha.prefix, sizeof(long long) * (na + 1), cudaMemcpyHostToDevice, st);
        if (!e) e = cudaMemsetAsync(s->da.ctr, 0, sizeof(InstCounters) * na, st);
    }
    if (!e && na > 0) {
        k_batch_select<<<s->g_sel, kScanBlock, 0, st>>>(s->da.inst, s->da.prefix, na, s->da.ctr, s->sig_key,
                                                       s->sig_cnt, s->sig_slot);
        k_batch_scan<<<1, kScanBlock, 0, st>>>(s->da.ctr, na, s->da.sprefix);
        k_batch_uf_init<<<s->g_agg, kAggBlock, 0, st>>>(s->da.inst, s->da.sprefix, na, s->parent, s->csize, s->cmin);
        k_batch_hook<<<s->g_agg, kAggBlock, 0, st>>>(s->da.inst, s->da.sprefix, na, s->sig_key, s->parent, s->da.ctr);
        k_batch_flatten<<<s->g_agg, kAggBlock, 0, st>>>(s->da.inst, s->da.sprefix, na, s->parent);
        k_batch_stats<<<s->g_agg, kAggBlock, 0, st>>>(s->da.inst, s->da.sprefix, na, s->sig_key, s->parent, s->csize,
                                                     s->cmin);
        k_batch_emit<<<s->g_agg, kAggBlock, 0, st>>>(s->da.inst, s->da.sprefix, na, s->sig_key, s->sig_cnt, s->parent,
                                                    s->csize, s->cmin, s->da.ctr, s->out_key, s->out_cnt, s->out_cid);
        if (!e) e = cudaMemcpyAsync(s->ha.ctr, s->da.ctr, sizeof(InstCounters) * na, cudaMemcpyDeviceToHost, st);
        note_launch(7);
    }
    if (!e) e = cudaGetLastError();
    if (!e) e = cudaEventRecord(s->ev1, st);
    if (!e) e = cudaStreamSynchronize(st);
    float step_ms = 0.f;
    if (!e) e = cudaEventElapsedTime(&step_ms, s->ev0, s->ev1);
    const Clock::time_point now = Clock::now();
    std::unique_lock<std::mutex> lk(s->mu);
    if (e != cudaSuccess) {
        s->fatal = RASTER_E_CUDA;
        s->cv_done.notify_all();
        return true;
    }
    long long pts = 0;
    for (int i = 0; i < nw; ++i) {
        Request* r = work[i].first;
        r->tiles += s->hc.ctr[i].tiles;
        r->status |= s->hc.ctr[i].status;
        r->contracted += 1;
        pts += work[i].second.n;
    }
    for (int i = 0; i < na; ++i) {
        Request* r = finishing[i];
        r->result = s->ha.ctr[i];
        r->result.tiles = r->tiles;
        r->result.status |= r->status;
        r->state = Request::kDone;
        r->t_done = now;
        free_table(s, r);  // the rows hold the result; the table is no longer needed
        s->active.erase(std::find(s->active.begin(), s->active.end(), r));
        s->completed.push_back(r);
    }
    s->steps += 1;
    s->points += pts;
    s->gpu_ms += step_ms;
    if (na) s->cv_done.notify_all();
    return true;
}

void worker_main(raster_server* s) {
    cudaSetDevice(s->device);
    Clock::time_point busy = Clock::now();
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop || s->fatal) return;
        }
        if (run_step(s)) {
            busy = Clock::now();
        } else {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop || s->fatal) return;
            // idle for a while: give the pages no live request holds back to
            // the device (no kernel of the engine is running now)
            if (std::chrono::duration<double, std::milli>(Clock::now() - busy).count() > kIdleTrimMs) {
                trim_all(s);
                busy = Clock::now();
            }
            s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        }
    }
}

int status_bits_to_code(unsigned long long bits) {
    if (bits & kStOom) return RASTER_E_OOM;
    if (bits & kStInternal) return RASTER_E_INTERNAL;
    if (bits & kStFull) return RASTER_E_TABLE_FULL;
    if (bits & kStRange) return RASTER_E_RANGE;
    return RASTER_OK;
}

template <typename T>
cudaError_t dmal(T** p, size_t n) {
    return cudaMalloc(p, std::max<size_t>(n, 1) * sizeof(T));
}

}  // namespace

extern "C" {

int raster_server_destroy(raster_server* s) {
    if (!s) return RASTER_E_ARG;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    if (s->stream) cudaStreamSynchronize(s->stream);
    void* bufs[] = {s->dc.inst, s->dc.prefix, s->dc.ctr,      s->dc.sprefix, s->dc.fill_off, s->dc.fill_len,
                    s->da.inst, s->da.prefix, s->da.ctr,      s->da.sprefix, s->da.fill_off, s->da.fill_len};
    for (void* p : bufs)
        if (p) cudaFree(p);
    void* hbufs[] = {s->hc.inst, s->hc.prefix, s->hc.ctr, s->hc.fill_off, s->hc.fill_len,
                     s->ha.inst, s->ha.prefix, s->ha.ctr, s->ha.fill_off, s->ha.fill_len};
    for (void* p : hbufs)
        if (p) cudaFreeHost(p);
    s->tab_va.destroy();
    for (auto& a : s->row_va) a.destroy();
    if (s->ev0) cudaEventDestroy(s->ev0);
    if (s->ev1) cudaEventDestroy(s->ev1);
    if (s->stream) cudaStreamDestroy(s->stream);
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
    return RASTER_OK;
}

int raster_server_create(const raster_server_config* cfg, raster_server** out) {
    if (!cfg || !out || cfg->table_slots < 0 || cfg->result_rows < 0 || cfg->max_active <= 0 ||
        cfg->max_active > kMaxStepItems || cfg->reserve_bytes < 0 || cfg->table_slots > (1ll << 36) ||
        cfg->result_rows > (long long)kMaxRows)
        return RASTER_E_ARG;
    *out = nullptr;
    raster_server* s = new (std::nothrow) raster_server();
    if (!s) return RASTER_E_OOM;
    cudaGetDevice(&s->device);
    s->max_active = cfg->max_active;
    s->reserve = (size_t)cfg->reserve_bytes;
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreate(&s->ev0);
    if (!e) e = cudaEventCreate(&s->ev1);
    size_t free_b = 0;
    if (!e) e = cudaMemGetInfo(&free_b, &s->total_mem);
    if (!e && !s->drv.load()) e = cudaErrorNotSupported;
    // address ranges: as many slots and rows as the device could ever hold
    // (or the caller's bounds); no physical memory yet
    const unsigned long long slots =
        cfg->table_slots > 0 ? (unsigned long long)cfg->table_slots : s->total_mem / sizeof(Slot);
    const unsigned long long rows =
        cfg->result_rows > 0 ? (unsigned long long)cfg->result_rows : std::min<unsigned long long>(kMaxRows, s->total_mem / kRowBytes);
    if (!e && !s->tab_va.init(&s->drv, s->device, slots * sizeof(Slot), kTablePage)) e = cudaErrorMemoryAllocation;
    for (int a = 0; a < 9 && !e; ++a)
        if (!s->row_va[a].init(&s->drv, s->device, rows * kRowElem[a], kRowPageRows * kRowElem[a]))
            e = cudaErrorMemoryAllocation;
    for (DeviceStep* d : {&s->dc, &s->da}) {
        if (!e) e = dmal(&d->inst, kMaxStepItems);
        if (!e) e = dmal(&d->prefix, kMaxStepItems + 1);
        if (!e) e = dmal(&d->ctr, kMaxStepItems);
        if (!e) e = dmal(&d->sprefix, kMaxStepItems + 1);
        if (!e) e = dmal(&d->fill_off, kMaxStepItems);
        if (!e) e = dmal(&d->fill_len, kMaxStepItems);
    }
    for (HostStep* h : {&s->hc, &s->ha}) {
        if (!e) e = cudaMallocHost(&h->inst, sizeof(BatchInst) * kMaxStepItems);
        if (!e) e = cudaMallocHost(&h->prefix, sizeof(long long) * (kMaxStepItems + 1));
        if (!e) e = cudaMallocHost(&h->ctr, sizeof(InstCounters) * kMaxStepItems);
        if (!e) e = cudaMallocHost(&h->fill_off, sizeof(unsigned long long) * kMaxStepItems);
        if (!e) e = cudaMallocHost(&h->fill_len, sizeof(unsigned long long) * kMaxStepItems);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        raster_server_destroy(s);
        return e == cudaErrorMemoryAllocation ? RASTER_E_OOM : RASTER_E_CUDA;
    }
    s->tab_arena = reinterpret_cast<Slot*>(s->tab_va.base());
    s->sig_key = reinterpret_cast<unsigned long long*>(s->row_va[0].base());
    s->sig_cnt = reinterpret_cast<unsigned int*>(s->row_va[1].base());
    s->sig_slot = reinterpret_cast<unsigned int*>(s->row_va[2].base());
    s->parent = reinterpret_cast<int*>(s->row_va[3].base());
    s->csize = reinterpret_cast<unsigned int*>(s->row_va[4].base());
    s->cmin = reinterpret_cast<unsigned long long*>(s->row_va[5].base());
    s->out_key = reinterpret_cast<unsigned long long*>(s->row_va[6].base());
    s->out_cnt = reinterpret_cast<unsigned int*>(s->row_va[7].base());
    s->out_cid = reinterpret_cast<unsigned long long*>(s->row_va[8].base());
    unsigned long long row_cap = kMaxRows;
    for (int a = 0; a < 9; ++a) row_cap = std::min<unsigned long long>(row_cap, s->row_va[a].bytes() / kRowElem[a]);
    s->tab_alloc.init(s->tab_va.bytes() / sizeof(Slot));
    s->row_alloc.init(row_cap);
    s->row_capacity = (long long)row_cap;
    s->g_con = grid_for_kernel((const void*)k_batch_contract<1, true>, 256);
    s->g_sel = grid_for_kernel((const void*)k_batch_select, kScanBlock);
    s->g_agg = grid_for_kernel((const void*)k_batch_hook, kAggBlock);
    s->worker = std::thread(worker_main, s);
    *out = s;
    return RASTER_OK;
}

int raster_server_submit(raster_server* s, int64_t request_id, double precision, uint32_t tau, uint32_t mu,
                         int64_t n_total, int32_t n_chunks) {
    if (!s || tau == 0 || mu == 0 || n_total < 0 || n_total > 0xFFFFFFFFll || n_chunks < 1 ||
        !std::isfinite(precision))
        return RASTER_E_ARG;
    Request* r = new (std::nothrow) Request();
    if (!r) return RASTER_E_OOM;
    r->id = request_id;
    r->tau = tau;
    r->mu = mu;
    r->n_total = n_total;
    r->n_chunks = n_chunks;
    if (make_proj_params(scale_of_precision(precision), &r->pp, &r->wide) != RASTER_OK) {
        delete r;
        return RASTER_E_ARG;
    }
    table_rows_for(n_total, tau, &r->cap, &r->rows);
    {
        const TestLimits lim = test_limits();
        r->max_probe = lim.probe >= 0 ? (unsigned int)std::min<unsigned long long>((unsigned long long)lim.probe, r->cap)
                                      : (unsigned int)r->cap;
        if (lim.unions >= 0) r->union_limit = lim.unions;
    }
    r->t_submit = Clock::now();
    {
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->fatal) {
            delete r;
            return s->fatal;
        }
        if (r->cap > s->tab_alloc.capacity() || r->rows > s->row_alloc.capacity() ||
            r->cap * sizeof(Slot) + r->rows * kRowBytes + s->reserve > s->total_mem) {
            delete r;
            return RASTER_E_LIMIT;  // could never be admitted
        }
        if (s->reqs.count(request_id)) {
            delete r;
            return RASTER_E_ARG;
        }
        s->reqs[request_id] = r;
        s->waiting.push_back(r);
    }
    s->cv_work.notify_one();
    return RASTER_OK;
}

int raster_server_push(raster_server* s, int64_t request_id, const double* xy, int64_t n) {
    if (!s || n < 0 || (n > 0 && (!xy || ((uintptr_t)xy & 15u)))) return RASTER_E_ARG;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->reqs.find(request_id);
        if (it == s->reqs.end()) return RASTER_E_ARG;
        Request* r = it->second;
        if (r->pushed >= r->n_chunks || r->pushed_points + n > r->n_total) return RASTER_E_ARG;
        if (r->pushed + 1 == r->n_chunks && r->pushed_points + n != r->n_total) return RASTER_E_ARG;
        r->pending.push_back(Chunk{xy, n});
        r->pushed += 1;
        r->pushed_points += n;
    }
    s->cv_work.notify_one();
    return RASTER_OK;
}

int raster_server_poll(raster_server* s, int32_t wait_ms, int64_t* request_id, raster_clusters* out,
                       double* latency_ms) {
    if (!s || !request_id || !out) return RASTER_E_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->completed.empty() && !s->fatal && wait_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms),
                            [s] { return !s->completed.empty() || s->fatal; });
    if (s->completed.empty()) return s->fatal ? s->fatal : RASTER_E_STATE;
    Request* r = s->completed.front();
    s->completed.pop_front();
    *request_id = r->id;
    out->key = reinterpret_cast<const int64_t*>(s->out_key + r->row_off);
    out->count = s->out_cnt + r->row_off;
    out->cid = reinterpret_cast<const int64_t*>(s->out_cid + r->row_off);
    out->n_tiles = (int64_t)r->result.kept;
    out->n_clusters = (int64_t)r->result.clusters;
    out->n_distinct = (int64_t)r->result.tiles;
    out->n_significant = (int64_t)r->result.sig;
    out->n_points = r->n_total;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    return status_bits_to_code(r->result.status);
}

int raster_server_release(raster_server* s, int64_t request_id) {
    if (!s) return RASTER_E_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end() || it->second->state != Request::kDone) return RASTER_E_ARG;
    Request* r = it->second;
    free_table(s, r);
    free_rows(s, r);
    s->reqs.erase(it);
    delete r;
    lk.unlock();
    s->cv_work.notify_one();
    return RASTER_OK;
}

int raster_server_stats(raster_server* s, raster_server_stats_t* out) {
    if (!s || !out) return RASTER_E_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    out->steps = s->steps;
    out->points = s->points;
    out->waiting = (int64_t)s->waiting.size();
    out->active = (int64_t)s->active.size();
    out->completed_unpolled = (int64_t)s->completed.size();
    out->table_slots_used = (int64_t)s->tab_alloc.used();
    out->result_rows_used = (int64_t)s->row_alloc.used();
    out->device_bytes = (int64_t)mapped_bytes(s);
    out->refused = s->refused;
    out->gpu_us = (int64_t)(s->gpu_ms * 1000.0);
    return s->fatal;
}

}  // extern "C"
