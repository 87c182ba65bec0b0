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
// EXP_true (Sec. 4.2.1, eqs. (t1), (chenlin); Alg. 1's final extrapolation):
//     u~ = u_h + (1/3) * (mean of u_h - u_2h over the 2^m coarse nodes
//                         around the node),
// which is (4 u_h - u_2h)/3 at coarse nodes and (chenlin) at 1D midpoints.

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

// Tiled, separable forms of the two fine-grid passes.  A CTA of 32 x 8
// threads owns a tile of TX x TY x TZ fine nodes; the coarse values its
// nodes need are staged in shared memory and interpolated along x, then y,
// then z, so each intermediate value is formed once instead of once per
// fine node that uses it (about 4 instead of 14 FP64 operations per node for
// Step 5; FP64 issue is scarce on GB300).
constexpr int TT_X = 32, TT_Y = 8, TT_Z = 8;
constexpr int TT_THREADS = 256;
constexpr int TM_X = TT_X / 2 + 1, TM_Y = TT_Y / 2 + 1, TM_Z = TT_Z / 2 + 1;   // coarse extents (17, 5, 5)

// Middle-grid cell of fine index v (Step 5 uses cells of 4 fine intervals).
__device__ __forceinline__ int quad_cell(int v, int n0) { return min(v >> 2, n0 - 1); }

// Step 5 at every fine node of the tile: per fine node the same products and
// sums, in the same order, as the direct tri-quadratic sum with x innermost,
// then y, then z.
__global__ void __launch_bounds__(TT_THREADS)
exp_finite_interp_tiled_kernel(double* __restrict__ w, const double* __restrict__ W, int nf) {
    __shared__ double Ws[TM_Z][TM_Y][TM_X];
    __shared__ double Tx[TM_Z][TM_Y][TT_X];
    __shared__ double Txy[TM_Z][TT_Y][TT_X];
    const int tid = threadIdx.x;
    const int np = nf + 1, n0 = nf / 4, np1 = nf / 2 + 1;
    const int xa = blockIdx.x * TT_X, ya = blockIdx.y * TT_Y, za = blockIdx.z * TT_Z;
    const int xb = min(xa + TT_X, np), yb = min(ya + TT_Y, np), zb = min(za + TT_Z, np);
    // middle-grid nodes used by the tile: from the first node of the first
    // cell to the last node of the last cell (tiles start on cell bounds)
    const int mx0 = 2 * quad_cell(xa, n0), my0 = 2 * quad_cell(ya, n0), mz0 = 2 * quad_cell(za, n0);
    const int nmx = 2 * quad_cell(xb - 1, n0) + 3 - mx0;
    const int nmy = 2 * quad_cell(yb - 1, n0) + 3 - my0;
    const int nmz = 2 * quad_cell(zb - 1, n0) + 3 - mz0;
    for (int e = tid; e < nmz * nmy * nmx; e += TT_THREADS) {
        const int ex = e % nmx, ey = (e / nmx) % nmy, ez = e / (nmx * nmy);
        Ws[ez][ey][ex] = W[nidx(np1, mx0 + ex, my0 + ey, mz0 + ez)];
    }
    __syncthreads();
    // along x: vx at (fine x, middle y, middle z)
    for (int e = tid; e < nmz * nmy * TT_X; e += TT_THREADS) {
        const int fx = e % TT_X, ey = (e / TT_X) % nmy, ez = e / (TT_X * nmy);
        const int i = xa + fx;
        if (i >= xb) continue;
        int xi[3];
        double xw[3];
        const int nx = quad_weights(i, n0, xi, xw);
        double vx = 0.0;
        for (int a = 0; a < nx; ++a) vx += xw[a] * Ws[ez][ey][xi[a] - mx0];
        Tx[ez][ey][fx] = vx;
    }
    __syncthreads();
    // along y: vy at (fine x, fine y, middle z)
    for (int e = tid; e < nmz * TT_Y * TT_X; e += TT_THREADS) {
        const int fx = e % TT_X, fy = (e / TT_X) % TT_Y, ez = e / (TT_X * TT_Y);
        const int i = xa + fx, j = ya + fy;
        if (i >= xb || j >= yb) continue;
        int yi[3];
        double yw[3];
        const int ny = quad_weights(j, n0, yi, yw);
        double vy = 0.0;
        for (int b = 0; b < ny; ++b) vy += yw[b] * Tx[ez][yi[b] - my0][fx];
        Txy[ez][fy][fx] = vy;
    }
    __syncthreads();
    // along z: the fine values
    for (int e = tid; e < TT_Z * TT_Y * TT_X; e += TT_THREADS) {
        const int fx = e % TT_X, fy = (e / TT_X) % TT_Y, fz = e / (TT_X * TT_Y);
        const int i = xa + fx, j = ya + fy, k = za + fz;
        if (i >= xb || j >= yb || k >= zb) continue;
        int zi[3];
        double zw[3];
        const int nz = quad_weights(k, n0, zi, zw);
        double v = 0.0;
        for (int c = 0; c < nz; ++c) v += zw[c] * Txy[zi[c] - mz0][fy][fx];
        w[nidx(np, i, j, k)] = v;
    }
}

// EXP_true at every fine node of the tile: d = u_h - u_2h at the coarse
// nodes, then its sums over the 1, 2, 4 or 8 coarse nodes around each fine
// node, formed along x, then y, then z.
__global__ void __launch_bounds__(TT_THREADS)
exp_true_tiled_kernel(double* __restrict__ ut, const double* __restrict__ uh, const double* __restrict__ u2h,
                      int nf) {
    __shared__ double Ds[TM_Z][TM_Y][TM_X];
    __shared__ double Sx[TM_Z][TM_Y][TT_X];
    __shared__ double Sxy[TM_Z][TT_Y][TT_X];
    const int tid = threadIdx.x;
    const int np = nf + 1, npc = nf / 2 + 1;
    const int xa = blockIdx.x * TT_X, ya = blockIdx.y * TT_Y, za = blockIdx.z * TT_Z;
    const int xb = min(xa + TT_X, np), yb = min(ya + TT_Y, np), zb = min(za + TT_Z, np);
    // coarse nodes around the tile's fine nodes: floor(v/2) .. ceil(v/2)
    const int cx0 = xa >> 1, cy0 = ya >> 1, cz0 = za >> 1;
    const int ncx = (xb >> 1) + 1 - cx0, ncy = (yb >> 1) + 1 - cy0, ncz = (zb >> 1) + 1 - cz0;
    for (int e = tid; e < ncz * ncy * ncx; e += TT_THREADS) {
        const int ex = e % ncx, ey = (e / ncx) % ncy, ez = e / (ncx * ncy);
        const int ci = cx0 + ex, cj = cy0 + ey, ck = cz0 + ez;
        if (ci < npc && cj < npc && ck < npc)
            Ds[ez][ey][ex] = uh[nidx(np, 2 * ci, 2 * cj, 2 * ck)] - u2h[nidx(npc, ci, cj, ck)];
    }
    __syncthreads();
    for (int e = tid; e < ncz * ncy * TT_X; e += TT_THREADS) {
        const int fx = e % TT_X, ey = (e / TT_X) % ncy, ez = e / (TT_X * ncy);
        const int i = xa + fx;
        if (i >= xb || cy0 + ey >= npc || cz0 + ez >= npc) continue;
        const int c = (i >> 1) - cx0;
        Sx[ez][ey][fx] = (i & 1) ? Ds[ez][ey][c] + Ds[ez][ey][c + 1] : Ds[ez][ey][c];
    }
    __syncthreads();
    for (int e = tid; e < ncz * TT_Y * TT_X; e += TT_THREADS) {
        const int fx = e % TT_X, fy = (e / TT_X) % TT_Y, ez = e / (TT_X * TT_Y);
        const int i = xa + fx, j = ya + fy;
        if (i >= xb || j >= yb || cz0 + ez >= npc) continue;
        const int c = (j >> 1) - cy0;
        Sxy[ez][fy][fx] = (j & 1) ? Sx[ez][c][fx] + Sx[ez][c + 1][fx] : Sx[ez][c][fx];
    }
    __syncthreads();
    for (int e = tid; e < TT_Z * TT_Y * TT_X; e += TT_THREADS) {
        const int fx = e % TT_X, fy = (e / TT_X) % TT_Y, fz = e / (TT_X * TT_Y);
        const int i = xa + fx, j = ya + fy, k = za + fz;
        if (i >= xb || j >= yb || k >= zb) continue;
        const int c = (k >> 1) - cz0;
        const double sum = (k & 1) ? Sxy[c][fy][fx] + Sxy[c + 1][fy][fx] : Sxy[c][fy][fx];
        const int m = (i & 1) + (j & 1) + (k & 1);
        const double wt = m == 0 ? 1.0 / 3.0 : (m == 1 ? 1.0 / 6.0 : (m == 2 ? 1.0 / 12.0 : 1.0 / 24.0));
        const size_t o = nidx(np, i, j, k);
        ut[o] = uh[o] + sum * wt;
    }
}

dim3 tiled_grid(int nf) {
    const int np = nf + 1;
    return dim3((np + TT_X - 1) / TT_X, (np + TT_Y - 1) / TT_Y, (np + TT_Z - 1) / TT_Z);
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
    exp_finite_interp_tiled_kernel<<<tiled_grid(n_fine), TT_THREADS, 0, s>>>(w, W_scratch, n_fine);
    return cudaGetLastError();
}

cudaError_t launch_exp_true(double* ut, const double* uh, const double* u2h, int n_fine,
                            cudaStream_t s) {
    exp_true_tiled_kernel<<<tiled_grid(n_fine), TT_THREADS, 0, s>>>(ut, uh, u2h, n_fine);
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

// The array's device address on the current device.  In host code the name
// g_noalloc_W is only a host-side stand-in, so the address is looked up on
// every call: a cached address would go stale if the device's context were
// reset and the library's device code loaded again elsewhere.  The lookup
// allocates nothing; on a device's first call it also loads the library's
// device code there.
int noalloc_scratch(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_W);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return EXCMG_ERR_CUDA;
    }
    *out = (double*)p;
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
