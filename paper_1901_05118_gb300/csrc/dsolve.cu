// DSOLVE of Alg. 1: the two coarsest grids are solved directly.
//
// A_h (the 25-point rows with reflections folded in) is assembled densely in
// lexicographic order of the unknowns (x fastest), inverted once per
// (N, bc_kind) by Gauss-Jordan elimination without pivoting (A_h is
// symmetric positive definite, so every pivot is positive), and kept in the
// context.  Each DSOLVE is then one dense matrix-vector product.  The grids
// involved are small (at most 15^3 = 3375 unknowns: a 91 MB inverse).
#include "excmg_internal.cuh"

namespace excmg {
namespace {

__global__ void dense_assemble_kernel(double* __restrict__ A, int n, double sigma) {
    const int m = n - 1;
    const int nu = m * m * m;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= nu) return;
    const int i = row % m + 1, j = (row / m) % m + 1, k = row / (m * m) + 1;
    double* Ar = A + (size_t)row * nu;
    auto put = [&](int qi, int qj, int qk, double c) {
        if (qi < 1 || qi > m || qj < 1 || qj > m || qk < 1 || qk > m) return;  // known value
        Ar[((qk - 1) * m + (qj - 1)) * m + (qi - 1)] += c;
    };
    put(i, j, k, 42.0);
    const int p[3] = {i, j, k};
    for (int ax = 0; ax < 3; ++ax)
        for (int s = -1; s <= 1; s += 2) {
            int q[3] = {p[0], p[1], p[2]};
            q[ax] = p[ax] + s;
            put(q[0], q[1], q[2], -12.0);
            q[ax] = p[ax] + 2 * s;
            if (q[ax] < 0 || q[ax] > n)
                put(i, j, k, sigma);   // ghost folded onto its mirror, the row's own node
            else
                put(q[0], q[1], q[2], 1.0);
        }
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            for (int sa = -1; sa <= 1; sa += 2)
                for (int sb = -1; sb <= 1; sb += 2) {
                    int q[3] = {p[0], p[1], p[2]};
                    q[a] += sa;
                    q[b] += sb;
                    put(q[0], q[1], q[2], 2.0);
                }
}

// Gauss-Jordan step k, part 1: the pivot row scaled by 1/pivot, the pivot
// column, and 1/pivot.
__global__ void gj_prep_kernel(const double* __restrict__ A, int m, int k, double* __restrict__ rowk,
                               double* __restrict__ colk) {
    const double piv = A[(size_t)k * m + k];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
        rowk[t] = A[(size_t)k * m + t] / piv;
        colk[t] = A[(size_t)t * m + k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rowk[m] = 1.0 / piv;
}

// Part 2: eliminate column k from every other row, in place.
__global__ void gj_update_kernel(double* __restrict__ A, int m, int k, const double* __restrict__ rowk,
                                 const double* __restrict__ colk) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= m || j >= m) return;
    const double inv = rowk[m];
    double* a = A + (size_t)i * m + j;
    if (i == k && j == k) *a = inv;
    else if (i == k) *a = rowk[j];
    else if (j == k) *a = -colk[i] * inv;
    else *a = *a - colk[i] * rowk[j];
}

// u_interior = Ainv * fh_interior; one warp per row.
__global__ void dense_apply_kernel(const double* __restrict__ Ainv, const double* __restrict__ fh,
                                   double* __restrict__ u, int n) {
    const int m = n - 1, nu = m * m * m, np = n + 1;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nu) return;
    const double* Ar = Ainv + (size_t)warp * nu;
    double v = 0.0;
    for (int c = lane; c < nu; c += 32) {
        const int ci = c % m + 1, cj = (c / m) % m + 1, ck = c / (m * m) + 1;
        v += Ar[c] * fh[((size_t)ck * np + cj) * np + ci];
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) {
        const int i = warp % m + 1, j = (warp / m) % m + 1, k = warp / (m * m) + 1;
        u[((size_t)k * np + j) * np + i] = v;
    }
}

}  // namespace

cudaError_t launch_dense_assemble(double* A, int n, int bc_kind, cudaStream_t s) {
    const int m = n - 1, nu = m * m * m;
    cudaError_t e = cudaMemsetAsync(A, 0, (size_t)nu * nu * sizeof(double), s);
    if (e != cudaSuccess) return e;
    dense_assemble_kernel<<<(nu + 127) / 128, 128, 0, s>>>(A, n, bc_kind == 1 ? 1.0 : -1.0);
    return cudaGetLastError();
}

cudaError_t launch_gauss_jordan_step(double* A, int m, int k, double* rowk, double* colk,
                                     cudaStream_t s) {
    gj_prep_kernel<<<(m + 255) / 256, 256, 0, s>>>(A, m, k, rowk, colk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 block(32, 8, 1);
    dim3 grid((m + 31) / 32, (m + 7) / 8, 1);
    gj_update_kernel<<<grid, block, 0, s>>>(A, m, k, rowk, colk);
    return cudaGetLastError();
}

cudaError_t launch_dense_apply(const double* Ainv, const double* fh, double* u, int n, cudaStream_t s) {
    const int m = n - 1, nu = m * m * m;
    const long long threads = (long long)nu * 32;
    dense_apply_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(Ainv, fh, u, n);
    return cudaGetLastError();
}

int dsolve_run(excmg_ctx* ctx, int n, int bc_kind, const double* fh, double* u) {
    if (n < 4 || n > 16) return ctx_fail(ctx, EXCMG_ERR_ARG, "DSOLVE supports 4 <= N <= 16");
    const int m = n - 1, nu = m * m * m;
    const auto key = std::make_pair(n, bc_kind);
    auto it = ctx->inverses.find(key);
    if (it == ctx->inverses.end()) {
        const size_t bytes = (size_t)nu * nu * sizeof(double);
        if (ctx->budget && ctx->bytes + bytes > ctx->budget)
            return ctx_fail(ctx, EXCMG_ERR_BUDGET, "HBM budget too small for the DSOLVE inverse");
        excmg_buffer buf;
        if (cudaMalloc(&buf.ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            return ctx_fail(ctx, EXCMG_ERR_OOM, "cudaMalloc of the DSOLVE inverse failed");
        }
        buf.bytes = bytes;
        ctx->bytes += bytes;
        it = ctx->inverses.emplace(key, buf).first;
        int st = EXCMG_OK;
        double* rk = ctx_buffer(ctx, "gj_row", (size_t)(nu + 1) * sizeof(double), &st);
        if (st) return st;
        double* ck = ctx_buffer(ctx, "gj_col", (size_t)(nu + 1) * sizeof(double), &st);
        if (st) return st;
        double* A = (double*)buf.ptr;
        cudaError_t e = launch_dense_assemble(A, n, bc_kind, ctx->stream);
        for (int k = 0; k < nu && e == cudaSuccess; ++k)
            e = launch_gauss_jordan_step(A, nu, k, rk, ck, ctx->stream);
        note_launches(1 + 2LL * nu);
        if (e != cudaSuccess) return ctx_cuda(ctx, e, "DSOLVE factorisation");
    }
    note_launches(1);
    return ctx_cuda(ctx, launch_dense_apply((const double*)it->second.ptr, fh, u, n, ctx->stream),
                    "DSOLVE apply");
}

}  // namespace excmg
