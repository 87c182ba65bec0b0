// Bounded grid-wide barrier of the cooperative kernels (the small-grid Bi-CG
// and the batch engine).
//
// One arrival counter serves every barrier of a launch.  Each CTA adds 1 to
// it, except CTA 0, which adds 2^31 - (G - 1): once all G CTAs of a barrier
// have arrived the counter has grown by exactly 2^31, so its top bit has
// flipped and its low bits are back where they started.  A CTA therefore
// waits until the top bit differs from the one its own atomic returned --
// one atomic per CTA and plain polls of the same word, no reset and no
// second word on the critical path.  Every wait is limited: a CTA that has
// polled `spin_limit` times without seeing the flip sets the error word and
// leaves, and every CTA that later reaches a barrier (or polls while
// waiting) sees the word and leaves too, so a kernel whose barrier cannot
// complete returns (the host reports EXCMG_ERR_TIMEOUT) instead of hanging
// the GPU.  The counter must be zero when the launch starts.
#pragma once

#include <cuda_runtime.h>

namespace excmg {

struct GridBarrier {
    unsigned int* count;   // arrival counter (zero at launch)
    unsigned int* gen;     // unused by the wait; kept zero
    int* err;              // set once a wait gave up
    long long spin_limit;  // polls of the counter before giving up
};

// Production limit: 2^22 polls, each an L2 round trip of hundreds of
// nanoseconds: about a second, far beyond any barrier of these kernels.
constexpr long long kBarrierSpinLimit = 1ll << 22;

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// All CTAs of a cooperative launch of `nblocks` CTAs: returns true once every
// CTA has arrived, false (in every thread) when a wait gave up.
__device__ __forceinline__ bool grid_sync(const GridBarrier& gb, unsigned int nblocks) {
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
        const bool master = blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
        const unsigned inc = master ? 0x80000000u - (nblocks - 1u) : 1u;
        __threadfence();   // this CTA's writes before its arrival
        const unsigned old = atomicAdd(gb.count, inc);
        long long spins = 0;
        while (((old ^ ld_acquire_gpu(gb.count)) & 0x80000000u) == 0u) {
            if ((++spins & 255) == 0) {
                if (*(volatile int*)gb.err) break;
                if (spins > gb.spin_limit) {
                    atomicExch(gb.err, 1);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int*)gb.err == 0;
}

}  // namespace excmg
