// Failure-path self-test: make one of the library's bounded device-side
// waits run out on purpose, without a fault, trap or hang, so that the path
// that turns a wait that gave up into EXCMG_ERR_TIMEOUT can be tested.  The
// wait is the one the cooperative kernels use (grid_sync); only the arrival
// it waits for is one that nothing makes.
#include "excmg_internal.cuh"
#include "grid_sync.cuh"

namespace excmg {
namespace {

constexpr int kSelftestCtas = 8;

// barrier words (count, generation, error) and the outcome; fixed device
// memory, so the self-test allocates nothing
__device__ unsigned int g_selftest_barrier[4];
__device__ int g_selftest_status;

// Every CTA of a cooperative launch waits at a barrier that expects one CTA
// more than the launch holds.
__global__ void barrier_timeout_kernel(GridBarrier gb) {
    const bool ok = grid_sync(gb, gridDim.x + 1u);
    if (blockIdx.x == 0 && threadIdx.x == 0) g_selftest_status = ok ? kConverged : kTimeout;
}

}  // namespace
}  // namespace excmg

using namespace excmg;

extern "C" int excmg_selftest_wait_timeout(int which, long long limit) {
    if (which != 0 || limit < 1 || limit > 100000000ll) return EXCMG_ERR_ARG;
    void* words = nullptr;
    void* status = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&words, g_selftest_barrier);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&status, g_selftest_status);
    if (e == cudaSuccess) e = cudaMemsetAsync(words, 0, sizeof(g_selftest_barrier), nullptr);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0xFF, sizeof(int), nullptr);
    if (e == cudaSuccess) {
        unsigned int* w = (unsigned int*)words;
        GridBarrier gb{w, w + 1, (int*)(w + 2), limit};
        void* args[] = {&gb};
        e = cudaLaunchCooperativeKernel((const void*)barrier_timeout_kernel, dim3(kSelftestCtas), dim3(32), args, 0,
                                        nullptr);
        note_launches(1);
    }
    int out = -1;
    if (e == cudaSuccess) e = cudaMemcpy(&out, status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return EXCMG_ERR_CUDA;
    }
    return out == kTimeout ? EXCMG_ERR_TIMEOUT : EXCMG_OK;
}
