// Device memory that grows and shrinks under a fixed address: the serving
// engine's tables and result rows.
//
// An array reserves a large range of device virtual addresses once and backs
// it with physical pages only where live data sits.  A request's range is
// mapped when it is admitted (after checking free device memory) and its
// pages are released when no live range touches them any more, so the engine
// never fixes its memory at creation, and the row offsets its kernels use stay
// valid.  Page handling uses the driver's virtual memory calls, looked up at
// run time through the runtime (the library links no driver library).
//
// Not thread-safe: the serving engine calls it under its lock, and maps or
// unmaps only from its worker thread while no kernel of the engine runs.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

namespace raster {

struct VmDriver {
    CUresult (*reserve)(CUdeviceptr*, size_t, size_t, CUdeviceptr, unsigned long long) = nullptr;
    CUresult (*free_va)(CUdeviceptr, size_t) = nullptr;
    CUresult (*create)(CUmemGenericAllocationHandle*, size_t, const CUmemAllocationProp*, unsigned long long) = nullptr;
    CUresult (*release)(CUmemGenericAllocationHandle) = nullptr;
    CUresult (*map)(CUdeviceptr, size_t, size_t, CUmemGenericAllocationHandle, unsigned long long) = nullptr;
    CUresult (*unmap)(CUdeviceptr, size_t) = nullptr;
    CUresult (*set_access)(CUdeviceptr, size_t, const CUmemAccessDesc*, size_t) = nullptr;
    CUresult (*granularity)(size_t*, const CUmemAllocationProp*, CUmemAllocationGranularity_flags) = nullptr;

    // Look the entry points up (once); false if any is missing.
    bool load() {
        if (map) return true;
        auto get = [](const char* name, void** fn) {
            cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
            return cudaGetDriverEntryPointByVersion(name, fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
                   q == cudaDriverEntryPointSuccess && *fn;
        };
        void* f[8] = {};
        const char* names[8] = {"cuMemAddressReserve", "cuMemAddressFree", "cuMemCreate", "cuMemRelease",
                                "cuMemMap",            "cuMemUnmap",       "cuMemSetAccess", "cuMemGetAllocationGranularity"};
        for (int i = 0; i < 8; ++i)
            if (!get(names[i], &f[i])) return false;
        reserve = reinterpret_cast<decltype(reserve)>(f[0]);
        free_va = reinterpret_cast<decltype(free_va)>(f[1]);
        create = reinterpret_cast<decltype(create)>(f[2]);
        release = reinterpret_cast<decltype(release)>(f[3]);
        set_access = reinterpret_cast<decltype(set_access)>(f[6]);
        granularity = reinterpret_cast<decltype(granularity)>(f[7]);
        unmap = reinterpret_cast<decltype(unmap)>(f[5]);
        map = reinterpret_cast<decltype(map)>(f[4]);
        return true;
    }
};

inline CUmemAllocationProp vm_prop(int device) {
    CUmemAllocationProp p = {};
    p.type = CU_MEM_ALLOCATION_TYPE_PINNED;
    p.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
    p.location.id = device;
    return p;
}

// One reserved address range backed page by page.
class VmArray {
public:
    // Reserve `bytes` of addresses (rounded up to whole pages of at least
    // `page_hint` bytes).  Returns false on failure.
    bool init(VmDriver* drv, int device, size_t bytes, size_t page_hint) {
        drv_ = drv;
        device_ = device;
        const CUmemAllocationProp prop = vm_prop(device);
        size_t g = 0;
        if (drv->granularity(&g, &prop, CU_MEM_ALLOC_GRANULARITY_RECOMMENDED) != CUDA_SUCCESS || g == 0) return false;
        page_ = (page_hint + g - 1) / g * g;
        const size_t pages = (bytes + page_ - 1) / page_;
        va_bytes_ = pages * page_;
        if (drv->reserve(&base_, va_bytes_, page_, 0, 0) != CUDA_SUCCESS) {
            base_ = 0;
            return false;
        }
        handle_.assign(pages, 0);
        refs_.assign(pages, 0);
        return true;
    }

    char* base() const { return reinterpret_cast<char*>(base_); }
    size_t bytes() const { return va_bytes_; }
    size_t page() const { return page_; }
    size_t mapped_bytes() const { return mapped_ * page_; }
    size_t cached_bytes() const { return cached_ * page_; }

    // Bytes of new physical memory that pinning [lo, hi) would map.
    size_t need(size_t lo, size_t hi) const {
        size_t n = 0;
        for (size_t p = lo / page_; hi > lo && p <= (hi - 1) / page_; ++p)
            if (!handle_[p]) n += page_;
        return n;
    }

    // Pin the pages of [lo, hi): map the missing ones.  On failure nothing
    // stays pinned and the driver's status is returned.
    CUresult pin(size_t lo, size_t hi) {
        if (hi <= lo) return CUDA_SUCCESS;
        const size_t p0 = lo / page_, p1 = (hi - 1) / page_;
        for (size_t p = p0; p <= p1; ++p) {
            if (!handle_[p]) {
                const CUresult r = map_page(p);
                if (r != CUDA_SUCCESS) {
                    for (size_t q = p0; q < p; ++q) unref(q);
                    return r;
                }
            } else if (refs_[p] == 0) {
                --cached_;
            }
            ++refs_[p];
        }
        return CUDA_SUCCESS;
    }

    // Unpin [lo, hi); pages no range holds stay mapped (cached) until trim().
    void unpin(size_t lo, size_t hi) {
        if (hi <= lo) return;
        for (size_t p = lo / page_; p <= (hi - 1) / page_; ++p) unref(p);
    }

    // Unmap every cached page; returns the bytes given back.
    size_t trim() {
        size_t freed = 0;
        for (size_t p = 0; p < handle_.size() && cached_ > 0; ++p)
            if (handle_[p] && refs_[p] == 0) {
                unmap_page(p);
                freed += page_;
            }
        return freed;
    }

    void destroy() {
        for (size_t p = 0; p < handle_.size(); ++p)
            if (handle_[p]) unmap_page(p);
        if (base_) drv_->free_va(base_, va_bytes_);
        base_ = 0;
        handle_.clear();
        refs_.clear();
    }

private:
    CUresult map_page(size_t p) {
        const CUmemAllocationProp prop = vm_prop(device_);
        CUmemGenericAllocationHandle h = 0;
        CUresult r = drv_->create(&h, page_, &prop, 0);
        if (r != CUDA_SUCCESS) return r;
        const CUdeviceptr at = base_ + p * page_;
        r = drv_->map(at, page_, 0, h, 0);
        if (r != CUDA_SUCCESS) {
            drv_->release(h);
            return r;
        }
        CUmemAccessDesc a = {};
        a.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
        a.location.id = device_;
        a.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
        r = drv_->set_access(at, page_, &a, 1);
        if (r != CUDA_SUCCESS) {
            drv_->unmap(at, page_);
            drv_->release(h);
            return r;
        }
        handle_[p] = h;
        ++mapped_;
        return CUDA_SUCCESS;
    }
    void unmap_page(size_t p) {
        drv_->unmap(base_ + p * page_, page_);
        drv_->release(handle_[p]);
        handle_[p] = 0;
        --mapped_;
        if (refs_[p] == 0) --cached_;
    }
    void unref(size_t p) {
        if (refs_[p] > 0 && --refs_[p] == 0) ++cached_;
    }

    VmDriver* drv_ = nullptr;
    int device_ = 0;
    CUdeviceptr base_ = 0;
    size_t va_bytes_ = 0, page_ = 0, mapped_ = 0, cached_ = 0;
    std::vector<CUmemGenericAllocationHandle> handle_;
    std::vector<uint32_t> refs_;
};

}  // namespace raster
