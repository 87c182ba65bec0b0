// Deterministic CTA and grid reductions shared by the kernels that fuse an
// inner product (the Bi-CG scalars of Alg. 2).  A fixed grid reduces its
// per-CTA partials in CTA order in the last CTA to finish (atomic ticket), so
// equal inputs always give equal bits.
#pragma once

#include <cuda_runtime.h>

namespace excmg {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over the CTA (valid in thread 0).  sh: 32 values of shared memory.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int lane = tid & 31, wid = tid >> 5;
    v = warp_sum(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T t = T(0);
    if (wid == 0) {
        t = lane < (nthreads >> 5) ? sh[lane] : T(0);
        t = warp_sum(t);
    }
    __syncthreads();
    return t;
}

__device__ __forceinline__ int flat_block() {
    return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}
__device__ __forceinline__ int flat_grid() { return gridDim.x * gridDim.y * gridDim.z; }
__device__ __forceinline__ bool thread0() { return threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0; }

// Publish this CTA's `count` partial sums and report (to every thread)
// whether this CTA is the last one to do so.
__device__ __forceinline__ bool publish_partials(const double* vals, int count, double* partials,
                                                 unsigned int* ticket, bool* am_last) {
    if (thread0()) {
        const int G = flat_grid(), b = flat_block();
        for (int c = 0; c < count; ++c) partials[c * G + b] = vals[c];
        __threadfence();
        const unsigned int t = atomicAdd(ticket, 1u);
        *am_last = (t == (unsigned)G - 1u);
    }
    __syncthreads();
    return *am_last;
}

// In the last CTA: the total of component c over all CTAs, in CTA order.
__device__ __forceinline__ double gather_partials(const double* partials, int c, double* sh) {
    const int G = flat_grid();
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    double v = 0.0;
    for (int b = tid; b < G; b += nthreads) v += __ldcg(&partials[c * G + b]);
    return block_sum(v, sh);
}

}  // namespace excmg
