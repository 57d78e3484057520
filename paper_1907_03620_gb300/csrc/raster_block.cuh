// Warp and block helpers shared by the single-instance, batched and served kernels.
#pragma once

#include <cuda_runtime.h>

namespace raster {

constexpr int kScanBlock = 256;  // block size assumed by block_excl_scan

__device__ __forceinline__ unsigned int warp_incl_scan(unsigned int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned int t = __shfl_up_sync(0xFFFFFFFFu, v, d);
        if (lane >= d) v += t;
    }
    return v;
}

// Exclusive block scan of v (blockDim.x == BLOCK, at most 1024); returns the
// prefix and writes the block total to *total.  Uses `scratch` (>= 33 words).
template <int BLOCK = kScanBlock>
__device__ __forceinline__ unsigned int block_excl_scan(unsigned int v, unsigned int* scratch, unsigned int* total) {
    constexpr int kBlock = BLOCK;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned int incl = warp_incl_scan(v);
    if (lane == 31) scratch[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned int w = (lane < (kBlock >> 5)) ? scratch[lane] : 0u;
        const unsigned int wi = warp_incl_scan(w);
        if (lane < (kBlock >> 5)) scratch[lane] = wi - w;
        if (lane == (kBlock >> 5) - 1) scratch[32] = wi;
    }
    __syncthreads();
    const unsigned int r = scratch[warp] + incl - v;
    *total = scratch[32];
    __syncthreads();
    return r;
}

}  // namespace raster
