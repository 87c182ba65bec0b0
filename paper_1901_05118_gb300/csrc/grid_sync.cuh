// Bounded grid-wide barrier of the cooperative kernels (the small-grid Bi-CG
// and the batch engine).  Every wait is limited: a CTA that has spun
// `spin_limit` times without seeing the barrier open sets the error word and
// leaves, and every CTA that later reaches a barrier sees the word and
// leaves too, so a kernel whose barrier cannot complete returns (with the
// error word set, which the host reports as EXCMG_ERR_TIMEOUT) instead of
// hanging the GPU.
#pragma once

#include <cuda_runtime.h>

namespace excmg {

struct GridBarrier {
    unsigned int* count;   // arrivals at the current barrier
    unsigned int* gen;     // barriers completed so far
    int* err;              // set once a wait gave up
    long long spin_limit;  // polls of `gen` before giving up (>= 32 ns each)
};

// Production limit: 2^22 polls of at least 32 ns each, well over 0.1 s.
constexpr long long kBarrierSpinLimit = 1ll << 22;

// All CTAs of a cooperative launch of `nblocks` CTAs: returns true once every
// CTA has arrived, false (in every thread) when a wait gave up.
__device__ __forceinline__ bool grid_sync(const GridBarrier& gb, unsigned int nblocks) {
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
        volatile unsigned int* gen = gb.gen;
        volatile int* err = gb.err;
        const unsigned int g = *gen;
        __threadfence();
        if (atomicAdd(gb.count, 1u) == nblocks - 1u) {
            atomicExch(gb.count, 0u);
            __threadfence();
            atomicAdd(gb.gen, 1u);
        } else {
            long long spins = 0;
            while (*gen == g) {
                if (*err) break;
                if (++spins > gb.spin_limit) {
                    atomicExch(gb.err, 1);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int*)gb.err == 0;
}

}  // namespace excmg
