// Instruction issue rates of one GPU: each thread runs 8 independent chains
// of one PTX operation for ITER iterations and writes one value (out has
// exactly blocks * threads entries).  Built and run by
//     python -m paper_1901_05118_gb300.cases issue-rates
// It measures why the 25-point operator is summed in 64-bit integers on
// GB300: FP64 FMA/add issue far below the integer and FP32 rates.
#include <cstdio>
#include <cuda_runtime.h>

constexpr int ITER = 4096;

#define CHAINS 8

__global__ void k_dfma(double* out, double a, double b) {
    double x[CHAINS];
    for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x + c;
    for (int it = 0; it < ITER; ++it)
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(x[c]) : "d"(a), "d"(b));
    double s = 0;
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void k_dadd(double* out, double a, double b) {
    double x[CHAINS];
    for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x + c;
    for (int it = 0; it < ITER; ++it)
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(x[c]) : "d"(a));
    double s = 0;
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void k_ffma(double* out, double a, double b) {
    float x[CHAINS];
    float fa = (float)a, fb = (float)b;
    for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x + c;
    for (int it = 0; it < ITER; ++it)
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[c]) : "f"(fa), "f"(fb));
    double s = 0;
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void k_iadd32(double* out, double a, double b) {
    int x[CHAINS];
    int y = (int)a;
    for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x + c;
    for (int it = 0; it < ITER; ++it)
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) asm volatile("add.s32 %0, %0, %1;" : "+r"(x[c]) : "r"(y));
    double s = 0;
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void k_iadd64(double* out, double a, double b) {
    long long x[CHAINS];
    long long y = (long long)a;
    for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x + c;
    for (int it = 0; it < ITER; ++it)
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) asm volatile("add.s64 %0, %0, %1;" : "+l"(x[c]) : "l"(y));
    double s = 0;
    for (int c = 0; c < CHAINS; ++c) s += (double)x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void k_imad32(double* out, double a, double b) {
    int x[CHAINS];
    int y = (int)a, z = (int)b;
    for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x + c;
    for (int it = 0; it < ITER; ++it)
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) asm volatile("mad.lo.s32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(y), "r"(z));
    double s = 0;
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void k_shf(double* out, double a, double b) {
    unsigned x[CHAINS];
    unsigned y = (unsigned)a;
    for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x + c;
    for (int it = 0; it < ITER; ++it)
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) asm volatile("shf.r.clamp.b32 %0, %0, %1, 3;" : "+r"(x[c]) : "r"(y));
    double s = 0;
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void k_i2f64(double* out, double a, double b) {
    unsigned long long x[CHAINS];
    long long y = (long long)a;
    for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x + c;
    for (int it = 0; it < ITER; ++it)
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) {
            double t;
            asm volatile("cvt.rn.f64.s64 %0, %1;" : "=d"(t) : "l"((long long)x[c]));
            x[c] = (unsigned long long)__double_as_longlong(t);   // dependency chain through the conversion
        }
    double s = 0;
    for (int c = 0; c < CHAINS; ++c) s += (double)x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void k_shr64(double* out, double a, double b) {
    unsigned long long x[CHAINS];
    unsigned y = (unsigned)a;
    for (int c = 0; c < CHAINS; ++c) x[c] = 0x123456789abcdefull + threadIdx.x + c;
    for (int it = 0; it < ITER; ++it)
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) asm volatile("shr.b64 %0, %0, %1;" : "+l"(x[c]) : "r"(y));
    double s = 0;
    for (int c = 0; c < CHAINS; ++c) s += (double)x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void k_iadd3(double* out, double a, double b) {
    int x[CHAINS];
    int y = (int)a, z = (int)b;
    for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x + c;
    for (int it = 0; it < ITER; ++it)
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) asm volatile("{.reg .s32 t; add.s32 t, %1, %2; add.s32 %0, %0, t;}" : "+r"(x[c]) : "r"(y), "r"(z + it));
    double s = 0;
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void k_mad64(double* out, double a, double b) {
    long long x[CHAINS];
    long long y = (long long)a;
    for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x + c;
    for (int it = 0; it < ITER; ++it)
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) asm volatile("mad.lo.s64 %0, %0, 12, %1;" : "+l"(x[c]) : "l"(y));
    double s = 0;
    for (int c = 0; c < CHAINS; ++c) s += (double)x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void k_madwide(double* out, double a, double b) {
    long long x[CHAINS];
    int y = (int)a;
    for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x + c;
    for (int it = 0; it < ITER; ++it)
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) asm volatile("mad.wide.s32 %0, %1, 12, %0;" : "+l"(x[c]) : "r"(y + c));
    double s = 0;
    for (int c = 0; c < CHAINS; ++c) s += (double)x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

typedef void (*kfn)(double*, double, double);

int main() {
    const int blocks = 152 * 8, threads = 256;
    double* out;
    cudaMalloc(&out, sizeof(double) * blocks * threads);
    struct { const char* name; kfn f; } ks[] = {{"dfma", k_dfma}, {"dadd", k_dadd}, {"ffma", k_ffma},
        {"iadd32", k_iadd32}, {"iadd64", k_iadd64}, {"imad32", k_imad32}, {"shf32", k_shf}, {"i2f64", k_i2f64}, {"shr64", k_shr64}, {"iadd_x2", k_iadd3}, {"mad64c", k_mad64}, {"madwide", k_madwide}};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int dev; cudaGetDevice(&dev);
    int clk; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    printf("sms %d clock_khz %d\n", sms, clk);
    for (auto& k : ks) {
        k.f<<<blocks, threads>>>(out, 1.0000001, 0.5);
        cudaDeviceSynchronize();
        cudaEventRecord(e0);
        for (int r = 0; r < 3; ++r) k.f<<<blocks, threads>>>(out, 1.0000001, 0.5);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms;
        cudaEventElapsedTime(&ms, e0, e1);
        double ops = 3.0 * blocks * threads * (double)ITER * CHAINS;
        printf("%-8s %.3f ms  %.3e ops/s  %.1f ops/clk/SM (at %d MHz)\n", k.name, ms, ops / (ms * 1e-3),
               ops / (ms * 1e-3) / sms / (clk * 1e3), clk / 1000);
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) { printf("error %s\n", cudaGetErrorString(err)); return 1; }
    }
    return 0;
}
