// Level-transfer steps of Alg. 1.
//
// EXP_finite (Sec. 4.2.2-4.2.3).  On one cell of the coarsest of three
// nested grids, Steps 1-4 give the 27 nodes shared with the middle grid:
// the corner rule (secfff) is u1 + (u1 - u0)/4, the edge rule (bfsec) adds
// (1/8) of the two end differences, and Steps 3-4 average (bfsec) over the
// 2 face diagonals / 4 space diagonals.  All four are one formula,
//     W = u1 + (1/4) * (mean of d = u1 - u0 over the 2^m coarse nodes
//                       around the node, m = number of odd coordinates),
// which the first kernel evaluates once per middle-grid node (shared cells
// agree by construction).  Step 5 is tri-quadratic Lagrange interpolation
// (eqs. (inter)-(iinter)) of W at the fine nodes: per axis the natural
// coordinate 0, 1/4, 1/2, 3/4, 1 has weights (1,0,0), (3/8,3/4,-1/8),
// (0,1,0), (-1/8,3/4,3/8), (0,0,1) on the cell's three middle-grid nodes.
//
// EXP_true (Sec. 4.2.1, eqs. (t1), (chenlin); Alg. 1 line 11):
//     u~ = u_h + (1/3) * (mean of u_h - u_2h over the 2^m coarse nodes
//                         around the node),
// which is (4 u_h - u_2h)/3 at coarse nodes and (chenlin) at 1D midpoints.
#include <mutex>

#include "excmg_internal.cuh"

namespace excmg {
namespace {

__device__ __forceinline__ size_t nidx(int np, int i, int j, int k) {
    return ((size_t)k * np + j) * np + i;
}

// coarse indices around fine index v on one axis: 1 (v even) or 2 (v odd)
__device__ __forceinline__ int around(int v, int* c) {
    if (v & 1) {
        c[0] = (v - 1) >> 1;
        c[1] = (v + 1) >> 1;
        return 2;
    }
    c[0] = v >> 1;
    return 1;
}

__global__ void exp_finite_w_kernel(double* __restrict__ W, const double* __restrict__ u1,
                                    const double* __restrict__ u0, int n1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    const int np1 = n1 + 1, np0 = n1 / 2 + 1;
    if (i >= np1 || j >= np1 || k >= np1) return;
    int ci[2], cj[2], ck[2];
    const int ni = around(i, ci), nj = around(j, cj), nk = around(k, ck);
    double sum = 0.0;
    for (int c = 0; c < nk; ++c)
        for (int b = 0; b < nj; ++b)
            for (int a = 0; a < ni; ++a)
                sum += u1[nidx(np1, 2 * ci[a], 2 * cj[b], 2 * ck[c])] - u0[nidx(np0, ci[a], cj[b], ck[c])];
    // 1/(4 * 2^m), m = number of odd coordinates: a power of two, so the
    // product is exact; an FP64 division would cost many of GB300's scarce
    // FP64 instructions per node
    const int m = (i & 1) + (j & 1) + (k & 1);
    const double w = m == 0 ? 0.25 : (m == 1 ? 0.125 : (m == 2 ? 0.0625 : 0.03125));
    W[nidx(np1, i, j, k)] = u1[nidx(np1, i, j, k)] + sum * w;
}

// Lagrange weights on the cell's middle-grid nodes for local offset o (0..4)
__device__ __forceinline__ int quad_weights(int v, int n0, int* idx, double* w) {
    int c = v >> 2;
    if (c > n0 - 1) c = n0 - 1;
    const int o = v - 4 * c;
    if ((o & 1) == 0) {
        idx[0] = 2 * c + (o >> 1);
        w[0] = 1.0;
        return 1;
    }
    idx[0] = 2 * c;
    idx[1] = 2 * c + 1;
    idx[2] = 2 * c + 2;
    if (o == 1) { w[0] = 0.375; w[1] = 0.75; w[2] = -0.125; }
    else { w[0] = -0.125; w[1] = 0.75; w[2] = 0.375; }
    return 3;
}

__global__ void exp_finite_interp_kernel(double* __restrict__ w, const double* __restrict__ W, int nf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    const int np = nf + 1, n0 = nf / 4, np1 = nf / 2 + 1;
    if (i >= np || j >= np || k >= np) return;
    int xi[3], yi[3], zi[3];
    double xw[3], yw[3], zw[3];
    const int nx = quad_weights(i, n0, xi, xw);
    const int ny = quad_weights(j, n0, yi, yw);
    const int nz = quad_weights(k, n0, zi, zw);
    double v = 0.0;
    for (int c = 0; c < nz; ++c) {
        double vy = 0.0;
        for (int b = 0; b < ny; ++b) {
            double vx = 0.0;
            for (int a = 0; a < nx; ++a) vx += xw[a] * W[nidx(np1, xi[a], yi[b], zi[c])];
            vy += yw[b] * vx;
        }
        v += zw[c] * vy;
    }
    w[nidx(np, i, j, k)] = v;
}

__global__ void exp_true_kernel(double* __restrict__ ut, const double* __restrict__ uh,
                                const double* __restrict__ u2h, int nf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    const int np = nf + 1, npc = nf / 2 + 1;
    if (i >= np || j >= np || k >= np) return;
    int ci[2], cj[2], ck[2];
    const int ni = around(i, ci), nj = around(j, cj), nk = around(k, ck);
    double sum = 0.0;
    for (int c = 0; c < nk; ++c)
        for (int b = 0; b < nj; ++b)
            for (int a = 0; a < ni; ++a)
                sum += uh[nidx(np, 2 * ci[a], 2 * cj[b], 2 * ck[c])] - u2h[nidx(npc, ci[a], cj[b], ck[c])];
    // weight 1/(3 * 2^m), m = number of odd coordinates (one table load
    // instead of an FP64 division per node)
    const int m = (i & 1) + (j & 1) + (k & 1);
    const double w = m == 0 ? 1.0 / 3.0 : (m == 1 ? 1.0 / 6.0 : (m == 2 ? 1.0 / 12.0 : 1.0 / 24.0));
    ut[nidx(np, i, j, k)] = uh[nidx(np, i, j, k)] + sum * w;
}

}  // namespace

cudaError_t launch_exp_finite(double* w, const double* u1, const double* u0, double* W_scratch,
                              int n_fine, cudaStream_t s) {
    const int n1 = n_fine / 2;
    dim3 block(32, 4, 1);
    dim3 g1((n1 + 1 + 31) / 32, (n1 + 1 + 3) / 4, n1 + 1);
    exp_finite_w_kernel<<<g1, block, 0, s>>>(W_scratch, u1, u0, n1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 g2((n_fine + 1 + 31) / 32, (n_fine + 1 + 3) / 4, n_fine + 1);
    exp_finite_interp_kernel<<<g2, block, 0, s>>>(w, W_scratch, n_fine);
    return cudaGetLastError();
}

cudaError_t launch_exp_true(double* ut, const double* uh, const double* u2h, int n_fine,
                            cudaStream_t s) {
    dim3 block(32, 4, 1);
    dim3 g((n_fine + 1 + 31) / 32, (n_fine + 1 + 3) / 4, n_fine + 1);
    exp_true_kernel<<<g, block, 0, s>>>(ut, uh, u2h, n_fine);
    return cudaGetLastError();
}

}  // namespace excmg

// ---------------------------------------------------------------------------
// EXP_finite without allocation.
//
// Some callers cannot allocate device memory when they need this step: code
// whose device memory is all owned by an arena or planner that hands out no
// further blocks (a serving process that sized its pools up front, a job
// held to a hard device-memory budget), or code running where entering the
// CUDA allocator is not allowed (cudaMalloc and cudaFree may synchronise the
// device, which a callback or a latency-critical path must not do).  This
// variant keeps its only scratch -- the middle-grid values W -- in a fixed
// array compiled into the library.  Every GPU that loads the library holds
// that array (2.2 MB) until the process exits.
namespace {

constexpr int kNoAllocMaxFine = 128;
constexpr size_t kNoAllocW =
    (size_t)(kNoAllocMaxFine / 2 + 1) * (kNoAllocMaxFine / 2 + 1) * (kNoAllocMaxFine / 2 + 1);

static __device__ __align__(256) double g_noalloc_W[kNoAllocW];

std::mutex g_noalloc_mu;
double* g_noalloc_addr[64] = {};   // device address of g_noalloc_W, per device

// The array's device address on the current device, looked up once per
// device (the name g_noalloc_W is only a host-side stand-in in host code).
int noalloc_scratch(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return EXCMG_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_W);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return EXCMG_ERR_CUDA;
        }
        g_noalloc_addr[dev] = (double*)p;
    }
    *out = g_noalloc_addr[dev];
    return EXCMG_OK;
}

}  // namespace

extern "C" int extrapolate_interpolate_noalloc(int n_fine, const double* u_2h, const double* u_4h,
                                               double* w_h) {
    if (n_fine < 8 || n_fine % 4 || !u_2h || !u_4h || !w_h) return EXCMG_ERR_ARG;
    if (n_fine > kNoAllocMaxFine) return EXCMG_ERR_SIZE;
    double* W = nullptr;
    const int st = noalloc_scratch(&W);
    if (st != EXCMG_OK) return st;
    // every entry of W is written before it is read: nothing to clear
    cudaError_t e = excmg::launch_exp_finite(w_h, u_2h, u_4h, W, n_fine, nullptr);
    excmg::note_launches(2);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return EXCMG_ERR_CUDA;
    }
    return EXCMG_OK;
}
