// The two-dimensional problem, eq. (bvp2d): Delta^2 u = f on (0,1)^2 with
// Dirichlet data of the first kind (u = g1, du/dn = g2) or the second kind
// (u = g1, d2u/dn2 = g2), solved by the same method as the 3D problem.
//
// The paper names the 13-point discretisation of the 2D equation without
// printing it; the scheme here is the 13-point one built as eq. (method1) is
// built for 3D (the square of the five-point Laplacian):
//     20 u - 8 (4 axis neighbours) + (4 neighbours at distance 2)
//          + 2 (4 diagonal neighbours) = h^4 f,
// with the fictitious node of a row one step from an edge folded onto the
// row's own node by the reflection formulas of Sec. 2 (first kind: ghost =
// mirror + 2h du/dn, so +1 on the diagonal per near-edge axis; second kind:
// ghost = 2 u_edge - mirror + h^2 d2u/dn2, so -1), the known parts moved to
// the right-hand side.  Alg. 1 and Alg. 2 run as in 3D (the flat vector
// kernels of Bi-CG are shared: they act on node arrays of any length); the
// transfer steps are the 2D forms of Sec. 4.2 (Richardson extrapolation at
// the coarse nodes, eq. (bfsec) at edge midpoints, the mean of the two
// diagonal rules at cell centres, bi-quadratic interpolation; EXP_true with
// bilinear interpolation).
//
// Layout: node arrays of (N+1)^2 doubles, x fastest (idx = j (N+1) + i); g2
// holds 4 edges of N+1 doubles: x=0, x=1, y=0, y=1, indexed by the other
// coordinate.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "excmg_internal.cuh"
#include "march_fx.cuh"
#include "reduce.cuh"

namespace excmg {
namespace {

constexpr int Q_TX = 32, Q_TY = 8, Q_OY = 16;       // 32 x 16 output nodes per CTA
constexpr int Q_HX = Q_TX + 4, Q_HY = Q_OY + 4;      // 36 x 20 halo
constexpr int Q_NT = Q_TX * Q_TY;
constexpr int Q_SLOTS = (Q_HX * Q_HY + Q_NT - 1) / Q_NT;

__device__ __forceinline__ size_t i2(int np, int i, int j) { return (size_t)j * np + i; }

// Largest biased exponent over the CTA (all threads get it).
__device__ __forceinline__ int block_max_exp(int e, int* sh) {
    const int tid = threadIdx.x + Q_TX * threadIdx.y, lane = tid & 31, warp = tid >> 5;
    e = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
    if (lane == 0) sh[warp] = e;
    __syncthreads();
    e = (int)__reduce_max_sync(0xffffffffu, (unsigned)sh[lane & (Q_NT / 32 - 1)]);
    __syncthreads();
    return e;
}

// y = A u (or y = b - A u) for NF fields on one 32 x 16 tile, in the
// integer arithmetic of the 3D operator: the tile's inputs on one
// power-of-two scale (its largest exponent), the 13 integer-weighted taps
// summed exactly, each output rounded once; error below 67 units of
// 2^(E-1075), E the tile's largest exponent.  A^T u gathers over the mirrored
// tap set, which has the same weights: the same integers, the same result.
// With kDot (NF = 2: p, p*) the CTA also forms its share of sigma = (p*, A p)
// and the last CTA alpha = rho / sigma (Alg. 2).  Where the two fields agree
// bit for bit over the whole tile, the second one's outputs are the first's.
template <int NF, bool kDot>
__global__ void __launch_bounds__(Q_NT)
stencil2d_kernel(const double* __restrict__ u0, const double* __restrict__ u1, double* __restrict__ y0,
                 double* __restrict__ y1, const double* __restrict__ b, int n, int sigma, double* partials,
                 BicgState* st) {
    if (kDot && st->done) return;
    __shared__ long long tile[NF][Q_HY * Q_HX];
    __shared__ int shx[Q_NT / 32];
    const int np = n + 1;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * Q_TX + tx;
    const int i0 = 1 + blockIdx.x * Q_TX, j0 = 1 + blockIdx.y * Q_OY;
    const double* in[2] = {u0, u1};
    double* out[2] = {y0, y1};
    double v[NF][Q_SLOTS];
    bool same = true;
#pragma unroll
    for (int s = 0; s < Q_SLOTS; ++s) {
        const int e = tid + s * Q_NT;
        const int ly = e / Q_HX, lx = e - ly * Q_HX;
        const int gi = i0 - 2 + lx, gj = j0 - 2 + ly;
        const bool ok = e < Q_HX * Q_HY && gi >= 1 && gi <= n - 1 && gj >= 1 && gj <= n - 1;
#pragma unroll
        for (int f = 0; f < NF; ++f) v[f][s] = ok ? in[f][i2(np, gi, gj)] : 0.0;
        if (NF == 2) same = same && __double_as_longlong(v[0][s]) == __double_as_longlong(v[NF - 1][s]);
    }
    const bool twin = NF == 2 && __syncthreads_and(same);
    int E[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        if (f > 0 && twin) {
            E[f] = E[0];
            continue;
        }
        int em = 0;
#pragma unroll
        for (int s = 0; s < Q_SLOTS; ++s) em = max(em, exponent_of(v[f][s]));
        E[f] = max(1, block_max_exp(em, shx));
#pragma unroll
        for (int s = 0; s < Q_SLOTS; ++s) {
            const int e = tid + s * Q_NT;
            if (e < Q_HX * Q_HY) tile[f][e] = to_fixed(v[f][s], E[f]);
        }
    }
    __syncthreads();
    const int i = i0 + tx, ja = j0 + 2 * ty;
    const int ry = 2 * ty + 2, rx = tx + 2;
    const int cx = (i == 1) + (i == n - 1);
    double dot = 0.0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int j = ja + q;
        if (i > n - 1 || j > n - 1) continue;
        const int cnt = cx + (j == 1) + (j == n - 1);
        const size_t o = i2(np, i, j);
        double val0 = 0.0;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            double val;
            if (f > 0 && twin) {
                val = val0;
            } else {
                const long long* T = tile[f];
                auto at = [&](int yy, int xx) { return T[(ry + q + yy) * Q_HX + rx + xx]; };
                const long long c = at(0, 0);
                const long long n4 = at(0, -1) + at(0, 1) + at(-1, 0) + at(1, 0);
                const long long f4 = at(0, -2) + at(0, 2) + at(-2, 0) + at(2, 0);
                const long long d4 = at(-1, -1) + at(-1, 1) + at(1, -1) + at(1, 1);
                const long long Y = (long long)(20 + sigma * cnt) * c - 8 * n4 + f4 + 2 * d4;
                val = fx_result(Y, E[f], E[f] == 0x7FF);
            }
            if (f == 0) val0 = val;
            if (NF == 1 && b != nullptr) val = b[o] - val;
            out[f][o] = val;
        }
        if (kDot) dot += in[NF - 1][o] * val0;   // (p*, A p)
    }
    if (kDot) {
        __shared__ double sh[32];
        __shared__ bool am_last;
        const double sdot = block_sum(dot, sh);
        if (publish_partials(&sdot, 1, partials, &st->ticket, &am_last)) {
            const double sg = gather_partials(partials, 0, sh);
            if (thread0()) {
                const double rho = st->rho;
                st->sigma = sg;
                if (!(rho != 0.0 && isfinite(rho)) || !(sg != 0.0 && isfinite(sg))) {
                    st->status = kBreakdown;
                    st->done = 1;
                } else {
                    st->alpha = rho / sg;
                }
                st->ticket = 0;
            }
        }
    }
}

dim3 grid2d(int n) { return dim3((n - 1 + Q_TX - 1) / Q_TX, (n - 1 + Q_OY - 1) / Q_OY, 1); }

__global__ void zero_boundary2d_kernel(double* __restrict__ y, int n) {
    const int np = n + 1;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 4 * np; t += gridDim.x * blockDim.x) {
        const int e = t / np, a = t - e * np;
        const int i = e < 2 ? (e & 1) * n : a, j = e < 2 ? a : (e & 1) * n;
        y[i2(np, i, j)] = 0.0;
    }
}

// f_h of the 2D scheme: h^4 f minus the known values each interior row
// touches (g1 at boundary nodes; through the reflection formulas, 2h g2 (first
// kind) or 2 g1 + h^2 g2 (second kind) at ghost nodes).  The level takes
// every stride-th node / edge value of arrays with n * stride intervals.
__global__ void assemble_rhs2d_kernel(double* __restrict__ fh, int n, int bc_kind, const double* __restrict__ f,
                                      const double* __restrict__ g1, const double* __restrict__ g2, int stride) {
    const int np = n + 1, nps = n * stride + 1;
    const double h = 1.0 / (double)n, h4 = h * h * h * h;
    const int total = np * np;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int i = t % np, j = t / np;
        if (i < 1 || i > n - 1 || j < 1 || j > n - 1) {
            fh[t] = 0.0;
            continue;
        }
        double rhs = h4 * f[i2(nps, i * stride, j * stride)];
        const int dxs[13] = {0, -1, 1, 0, 0, -2, 2, 0, 0, -1, -1, 1, 1};
        const int dys[13] = {0, 0, 0, -1, 1, 0, 0, -2, 2, -1, 1, -1, 1};
        const double cs[13] = {20, -8, -8, -8, -8, 1, 1, 1, 1, 2, 2, 2, 2};
        for (int k = 0; k < 13; ++k) {
            const int qi = i + dxs[k], qj = j + dys[k];
            if (qi < 0 || qi > n || qj < 0 || qj > n) {
                // ghost one step outside edge (axis, side); datum at the edge node
                const int axis = (qi < 0 || qi > n) ? 0 : 1, side = (axis == 0 ? qi > n : qj > n) ? 1 : 0;
                const int bi = axis == 0 ? side * n : qi, bj = axis == 0 ? qj : side * n;
                const int edge = 2 * axis + side, a = axis == 0 ? bj : bi;
                const double gb = g2[(size_t)edge * nps + (size_t)a * stride];
                const double known =
                    bc_kind == 1 ? 2.0 * h * gb : 2.0 * g1[i2(nps, bi * stride, bj * stride)] + h * h * gb;
                rhs -= cs[k] * known;
            } else if (qi == 0 || qi == n || qj == 0 || qj == n) {
                rhs -= cs[k] * g1[i2(nps, qi * stride, qj * stride)];
            }
        }
        fh[t] = rhs;
    }
}

// boundary nodes of u <- g1 (every stride-th node of g1)
__global__ void set_boundary2d_kernel(double* __restrict__ u, int n, const double* __restrict__ g1, int stride) {
    const int np = n + 1, nps = n * stride + 1;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 4 * np; t += gridDim.x * blockDim.x) {
        const int e = t / np, a = t - e * np;
        const int i = e < 2 ? (e & 1) * n : a, j = e < 2 ? a : (e & 1) * n;
        u[i2(np, i, j)] = g1[i2(nps, i * stride, j * stride)];
    }
}

// EXP_finite, Steps 1-3 on the middle grid: W = u1 + (1/4) (mean of
// d = u1 - u0 over the 2^m coarse nodes around the node, m = number of odd
// coordinates) -- eq. (secfff) at coarse nodes, (bfsec) at edge midpoints,
// the mean of the two diagonal rules at cell centres.
__global__ void exp_finite_w2d_kernel(double* __restrict__ W, const double* __restrict__ u1,
                                      const double* __restrict__ u0, int n1) {
    const int np1 = n1 + 1, np0 = n1 / 2 + 1;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < np1 * np1; t += gridDim.x * blockDim.x) {
        const int i = t % np1, j = t / np1;
        const int ci[2] = {i >> 1, (i + 1) >> 1}, cj[2] = {j >> 1, (j + 1) >> 1};
        const int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1;
        double sum = 0.0;
        for (int bb = 0; bb < nj; ++bb)
            for (int aa = 0; aa < ni; ++aa)
                sum += u1[i2(np1, 2 * ci[aa], 2 * cj[bb])] - u0[i2(np0, ci[aa], cj[bb])];
        const int m = (i & 1) + (j & 1);
        const double w = m == 0 ? 0.25 : (m == 1 ? 0.125 : 0.0625);
        W[t] = u1[t] + sum * w;
    }
}

// weights of the middle-grid nodes of the cell holding fine index v
__device__ __forceinline__ int quad_w2(int v, int n0, int* idx, double* w) {
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

// Step 4: bi-quadratic Lagrange interpolation of W at every fine node.
__global__ void exp_finite_interp2d_kernel(double* __restrict__ w, const double* __restrict__ W, int nf) {
    const int np = nf + 1, np1 = nf / 2 + 1, n0 = nf / 4;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < np * np; t += gridDim.x * blockDim.x) {
        const int i = t % np, j = t / np;
        int xi[3], yi[3];
        double xw[3], yw[3];
        const int nx = quad_w2(i, n0, xi, xw), ny = quad_w2(j, n0, yi, yw);
        double v = 0.0;
        for (int bb = 0; bb < ny; ++bb) {
            double vx = 0.0;
            for (int aa = 0; aa < nx; ++aa) vx += xw[aa] * W[i2(np1, xi[aa], yi[bb])];
            v += yw[bb] * vx;
        }
        w[t] = v;
    }
}

// EXP_true: u~ = u_h + (1/3) bilinear interpolation of u_h - u_2h.
__global__ void exp_true2d_kernel(double* __restrict__ ut, const double* __restrict__ uh,
                                  const double* __restrict__ u2h, int nf) {
    const int np = nf + 1, npc = nf / 2 + 1;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < np * np; t += gridDim.x * blockDim.x) {
        const int i = t % np, j = t / np;
        const int ci[2] = {i >> 1, (i + 1) >> 1}, cj[2] = {j >> 1, (j + 1) >> 1};
        double sum = 0.0;
        for (int bb = 0; bb < 2; ++bb)
            for (int aa = 0; aa < 2; ++aa)
                sum += uh[i2(np, 2 * ci[aa], 2 * cj[bb])] - u2h[i2(npc, ci[aa], cj[bb])];
        ut[t] = uh[t] + (sum * 0.25) / 3.0;
    }
}

// DSOLVE: rows of the dense A_h over the unknowns (x fastest).
__global__ void dense_assemble2d_kernel(double* __restrict__ A, int n, double sigma) {
    const int m = n - 1, nu = m * m;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= nu) return;
    const int i = row % m + 1, j = row / m + 1;
    double* Ar = A + (size_t)row * nu;
    auto put = [&](int qi, int qj, double c) {
        if (qi < 1 || qi > m || qj < 1 || qj > m) return;
        Ar[(qj - 1) * m + (qi - 1)] += c;
    };
    put(i, j, 20.0);
    const int p[2] = {i, j};
    for (int ax = 0; ax < 2; ++ax)
        for (int s = -1; s <= 1; s += 2) {
            int q[2] = {p[0], p[1]};
            q[ax] = p[ax] + s;
            put(q[0], q[1], -8.0);
            q[ax] = p[ax] + 2 * s;
            if (q[ax] < 0 || q[ax] > n) put(i, j, sigma);
            else put(q[0], q[1], 1.0);
        }
    for (int sa = -1; sa <= 1; sa += 2)
        for (int sb = -1; sb <= 1; sb += 2) put(i + sa, j + sb, 2.0);
}

__global__ void dense_apply2d_kernel(const double* __restrict__ Ainv, const double* __restrict__ fh,
                                     double* __restrict__ u, int n) {
    const int m = n - 1, nu = m * m, np = n + 1;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= nu) return;
    const double* Ar = Ainv + (size_t)warp * nu;
    double v = 0.0;
    for (int c = lane; c < nu; c += 32) v += Ar[c] * fh[i2(np, c % m + 1, c / m + 1)];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) u[i2(np, warp % m + 1, warp / m + 1)] = v;
}

int blocks_for(size_t work) {
    size_t b = (work + 255) / 256;
    if (b > 4096) b = 4096;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_stencil2d(const double* u, double* y, const double* b, int n, int bc_kind, cudaStream_t s) {
    stencil2d_kernel<1, false><<<grid2d(n), dim3(Q_TX, Q_TY), 0, s>>>(u, nullptr, y, nullptr, b, n,
                                                                      bc_kind == 1 ? 1 : -1, nullptr, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        zero_boundary2d_kernel<<<blocks_for(4 * (size_t)(n + 1)), 256, 0, s>>>(y, n);
        e = cudaGetLastError();
    }
    return e;
}

int dsolve2d(excmg_ctx* ctx, int n, int bc_kind, const double* fh, double* u) {
    if (n < 4 || n > 32) return ctx_fail(ctx, EXCMG_ERR_ARG, "2D DSOLVE supports 4 <= N <= 32");
    const int m = n - 1, nu = m * m;
    const auto key = std::make_pair(-n, bc_kind);   // 2D inverses: negative grid sizes
    auto it = ctx->inverses.find(key);
    if (it == ctx->inverses.end()) {
        const size_t bytes = (size_t)nu * nu * sizeof(double);
        if (ctx->budget && ctx->bytes + bytes > ctx->budget)
            return ctx_fail(ctx, EXCMG_ERR_BUDGET, "HBM budget too small for the 2D DSOLVE inverse");
        excmg_buffer buf;
        if (cudaMalloc(&buf.ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            return ctx_fail(ctx, EXCMG_ERR_OOM, "cudaMalloc of the 2D DSOLVE inverse failed");
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
        cudaError_t e = cudaMemsetAsync(A, 0, bytes, ctx->stream);
        if (e == cudaSuccess) {
            dense_assemble2d_kernel<<<(nu + 127) / 128, 128, 0, ctx->stream>>>(A, n, bc_kind == 1 ? 1.0 : -1.0);
            e = cudaGetLastError();
        }
        for (int k = 0; k < nu && e == cudaSuccess; ++k) e = launch_gauss_jordan_step(A, nu, k, rk, ck, ctx->stream);
        note_launches(1 + 2LL * nu);
        if (e != cudaSuccess) return ctx_cuda(ctx, e, "2D DSOLVE factorisation");
    }
    dense_apply2d_kernel<<<(unsigned)(((long long)nu * 32 + 255) / 256), 256, 0, ctx->stream>>>(
        (const double*)it->second.ptr, fh, u, n);
    note_launches(1);
    return ctx_cuda(ctx, cudaGetLastError(), "2D DSOLVE apply");
}

double host_norm(excmg_ctx* ctx, const double* a, size_t len, int* st) {
    cudaError_t e = launch_dot(a, a, len, ctx->partials, ctx->ticket, ctx->scalar, ctx->stream);
    note_launches(1);
    if (e == cudaSuccess)
        e = ctx_read_back(ctx, ctx->host_scalar, ctx->scalar, sizeof(double));
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        *st = ctx_cuda(ctx, e, "2D norm");
        return 0.0;
    }
    return sqrt(*ctx->host_scalar);
}

// ||b - A x|| over the unknowns, through the context's residual buffer.
double residual2d(excmg_ctx* ctx, int n, int bc_kind, const double* b, const double* x, int* st) {
    const size_t len = (size_t)(n + 1) * (n + 1);
    double* r = ctx_buffer(ctx, "res2d", len * sizeof(double), st);
    if (*st) return 0.0;
    cudaError_t e = launch_stencil2d(x, r, b, n, bc_kind, ctx->stream);
    note_launches(2);
    if (e != cudaSuccess) {
        *st = ctx_cuda(ctx, e, "2D residual");
        return 0.0;
    }
    return host_norm(ctx, r, len, st);
}

// Alg. 2 (M = I, r*_0 = r_0) on the 2D system: the operator pair with sigma
// and alpha, then the flat update and direction-update kernels of the 3D
// solver; the host looks at the device state every check_every iterations.
int bicg2d_run(excmg_ctx* ctx, int n, int bc_kind, const double* b, double* x, double tol, double bnorm, int max_iter,
               int check_every, int* iters_out, double* relres_out) {
    const size_t len = (size_t)(n + 1) * (n + 1), bytes = len * sizeof(double);
    int st = EXCMG_OK;
    double* r = ctx_buffer(ctx, "b2_r", bytes, &st);
    double* rs = st ? nullptr : ctx_buffer(ctx, "b2_rs", bytes, &st);
    double* p = st ? nullptr : ctx_buffer(ctx, "b2_p", bytes, &st);
    double* ps = st ? nullptr : ctx_buffer(ctx, "b2_ps", bytes, &st);
    double* q = st ? nullptr : ctx_buffer(ctx, "b2_q", bytes, &st);
    double* qs = st ? nullptr : ctx_buffer(ctx, "b2_qs", bytes, &st);
    if (st) return st;
    const dim3 g = grid2d(n);
    if ((int)(g.x * g.y) > kMaxPartials) return ctx_fail(ctx, EXCMG_ERR_ARG, "2D grid too large");
    cudaStream_t s = ctx->stream;
    BicgState init{};
    init.bnorm = bnorm;
    init.tol = tol;
    init.max_iter = max_iter;
    *ctx->host_state = init;
    cudaError_t e = cudaMemcpyAsync(ctx->state, ctx->host_state, sizeof(BicgState), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(q, 0, bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(qs, 0, bytes, s);
    if (e == cudaSuccess) e = launch_stencil2d(x, r, b, n, bc_kind, s);
    if (e == cudaSuccess) e = launch_bicg_init(r, nullptr, rs, p, ps, len, ctx->partials, ctx->state, s);
    note_launches(3);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "2D Bi-CG setup");
    const int sg = bc_kind == 1 ? 1 : -1;
    if (check_every < 1) check_every = 1;
    for (;;) {
        e = ctx_read_back(ctx, ctx->host_state, ctx->state, sizeof(BicgState));
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return ctx_cuda(ctx, e, "2D Bi-CG state read");
        if (ctx->host_state->done) break;
        int batch = check_every;
        const int left = max_iter - ctx->host_state->iter;
        if (batch > left) batch = left;
        for (int it = 0; it < batch && e == cudaSuccess; ++it) {
            stencil2d_kernel<2, true><<<g, dim3(Q_TX, Q_TY), 0, s>>>(p, ps, q, qs, nullptr, n, sg, ctx->partials,
                                                                     ctx->state);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = launch_bicg_update(x, p, r, q, rs, qs, len, ctx->partials, ctx->state, s);
            if (e == cudaSuccess) e = launch_bicg_pupdate(p, r, ps, rs, len, ctx->state, s);
        }
        note_launches(3LL * batch);
        if (e != cudaSuccess) return ctx_cuda(ctx, e, "2D Bi-CG iteration");
    }
    const BicgState& h = *ctx->host_state;
    if (iters_out) *iters_out = h.iter;
    const double rn = sqrt(h.rr);
    if (relres_out) *relres_out = bnorm > 0.0 ? rn / bnorm : rn;
    if (!std::isfinite(h.rr)) return ctx_fail(ctx, EXCMG_ERR_NAN, "2D Bi-CG residual is not finite");
    if (h.status == kBreakdown) return ctx_fail(ctx, EXCMG_ERR_BREAKDOWN, "2D Bi-CG breakdown");
    if (h.status == kCapped) return EXCMG_ERR_NOCONV;
    return EXCMG_OK;
}

cudaError_t launch_exp_finite2d(double* w, const double* u1, const double* u0, double* W, int nf, cudaStream_t s) {
    const int n1 = nf / 2;
    exp_finite_w2d_kernel<<<blocks_for((size_t)(n1 + 1) * (n1 + 1)), 256, 0, s>>>(W, u1, u0, n1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        exp_finite_interp2d_kernel<<<blocks_for((size_t)(nf + 1) * (nf + 1)), 256, 0, s>>>(w, W, nf);
        e = cudaGetLastError();
    }
    return e;
}

bool pow2_steps(int fine, int coarse, int* steps) {
    if (coarse <= 0 || fine < coarse) return false;
    int k = 0, v = coarse;
    while (v < fine) {
        v *= 2;
        ++k;
    }
    *steps = k;
    return v == fine;
}

}  // namespace
}  // namespace excmg

using namespace excmg;

extern "C" {

int excmg2d_stencil_apply(excmg_ctx* ctx, int n, int bc_kind, int transpose, const double* u, double* y) {
    (void)transpose;   // A^T u == A u bit for bit here (mirrored taps, equal weights)
    if (!ctx || !u || !y || n < 4 || (bc_kind != 1 && bc_kind != 2)) return EXCMG_ERR_ARG;
    if (u == y) return ctx_fail(ctx, EXCMG_ERR_ARG, "excmg2d_stencil_apply: u and y must not overlap");
    cudaError_t e = launch_stencil2d(u, y, nullptr, n, bc_kind, ctx->stream);
    note_launches(2);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return ctx_cuda(ctx, e, "excmg2d_stencil_apply");
}

int excmg2d_bicg_solve(excmg_ctx* ctx, int n, int bc_kind, const double* b, double* x_inout, double tol,
                       int max_iter, int* iters_out, double* relres_out) {
    if (!ctx || !b || !x_inout || n < 4 || (bc_kind != 1 && bc_kind != 2)) return EXCMG_ERR_ARG;
    if (!(tol >= 0.0) || max_iter < 0) return ctx_fail(ctx, EXCMG_ERR_ARG, "excmg2d_bicg_solve: bad tol / max_iter");
    // ||b|| over the unknowns: b's boundary entries are not part of the system
    const size_t len = (size_t)(n + 1) * (n + 1);
    int st = EXCMG_OK;
    double* bi = ctx_buffer(ctx, "b2_bint", len * sizeof(double), &st);
    if (st) return st;
    cudaError_t e = cudaMemcpyAsync(bi, b, len * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) {
        zero_boundary2d_kernel<<<blocks_for(4 * (size_t)(n + 1)), 256, 0, ctx->stream>>>(bi, n);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "excmg2d_bicg_solve");
    const double bnorm = host_norm(ctx, bi, len, &st);
    if (st) return st;
    return bicg2d_run(ctx, n, bc_kind, b, x_inout, tol, bnorm, max_iter, 16, iters_out, relres_out);
}

int excmg2d_extrapolate_interpolate(excmg_ctx* ctx, int n_fine, const double* u_2h, const double* u_4h,
                                    const double* g1_fine, double* w_h) {
    if (!ctx || !u_2h || !u_4h || !w_h || n_fine < 8 || n_fine % 4) return EXCMG_ERR_ARG;
    int st = EXCMG_OK;
    double* W = ctx_buffer(ctx, "exp2d_W", (size_t)(n_fine / 2 + 1) * (n_fine / 2 + 1) * sizeof(double), &st);
    if (st) return st;
    cudaError_t e = launch_exp_finite2d(w_h, u_2h, u_4h, W, n_fine, ctx->stream);
    note_launches(2);
    if (e == cudaSuccess && g1_fine) {
        set_boundary2d_kernel<<<blocks_for(4 * (size_t)(n_fine + 1)), 256, 0, ctx->stream>>>(w_h, n_fine, g1_fine, 1);
        e = cudaGetLastError();
        note_launches(1);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return ctx_cuda(ctx, e, "excmg2d_extrapolate_interpolate");
}

int excmg2d_midpoint_extrapolate(excmg_ctx* ctx, int n_fine, const double* u_h, const double* u_2h,
                                 double* u_tilde) {
    if (!ctx || !u_h || !u_2h || !u_tilde || n_fine < 4 || n_fine % 2) return EXCMG_ERR_ARG;
    exp_true2d_kernel<<<blocks_for((size_t)(n_fine + 1) * (n_fine + 1)), 256, 0, ctx->stream>>>(u_tilde, u_h, u_2h,
                                                                                               n_fine);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return ctx_cuda(ctx, e, "excmg2d_midpoint_extrapolate");
}

int excmg2d_solve(excmg_ctx* ctx, int n_finest, int n_coarsest, int bc_kind, const double* f, const double* g1,
                  const double* g2, const excmg_params* params, double* u_h_out, double* u_tilde_out,
                  excmg_stats* stats) {
    if (!ctx || !f || !g1 || !g2 || !params) return EXCMG_ERR_ARG;
    if (bc_kind != 1 && bc_kind != 2) return ctx_fail(ctx, EXCMG_ERR_ARG, "bc_kind must be 1 or 2");
    int steps = 0;
    if (n_coarsest < 4 || 2 * n_coarsest > 32)
        return ctx_fail(ctx, EXCMG_ERR_ARG, "n_coarsest must be 4..16 (2D DSOLVE grids up to 32 intervals)");
    if (!pow2_steps(n_finest, n_coarsest, &steps) || steps < 2)
        return ctx_fail(ctx, EXCMG_ERR_ARG, "n_finest must be n_coarsest * 2^(L+1) with L >= 1");
    if (!(params->tol > 0.0) || params->max_iter < 1 || params->max_total < 1)
        return ctx_fail(ctx, EXCMG_ERR_ARG, "excmg2d_solve: tol > 0, max_iter >= 1, max_total >= 1");
    if (params->precision != EXCMG_PRECISION_FP64)
        return ctx_fail(ctx, EXCMG_ERR_ARG, "excmg2d_solve: FP64 only");
    const int nl = steps + 1, L = nl - 2;
    if (nl > EXCMG_MAX_LEVELS) return ctx_fail(ctx, EXCMG_ERR_ARG, "too many levels");
    cudaStream_t s = ctx->stream;
    int st = EXCMG_OK;
    double* lvl[EXCMG_MAX_LEVELS] = {};
    for (int l = 0; l < nl; ++l) {
        char name[32];
        snprintf(name, sizeof name, "l2d_u%d", l);
        const int N = n_coarsest << l;
        lvl[l] = ctx_buffer(ctx, name, (size_t)(N + 1) * (N + 1) * sizeof(double), &st);
        if (st) return st;
    }
    const size_t lenf = (size_t)(n_finest + 1) * (n_finest + 1);
    double* fh = ctx_buffer(ctx, "l2d_fh", lenf * sizeof(double), &st);
    double* W = st ? nullptr : ctx_buffer(ctx, "exp2d_W", (size_t)(n_finest / 2 + 1) * (n_finest / 2 + 1) * 8, &st);
    if (st) return st;
    if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->levels = nl;
    }
    for (int l = 0; l < nl; ++l) {
        const int N = n_coarsest << l, stride = n_finest / N;
        const size_t len = (size_t)(N + 1) * (N + 1);
        double* u = lvl[l];
        int iters = 0, calls = 0, stag = 0, bad = 0;
        double rel = 0.0;
        assemble_rhs2d_kernel<<<blocks_for(len), 256, 0, s>>>(fh, N, bc_kind, f, g1, g2, stride);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && l >= 2) e = launch_exp_finite2d(u, lvl[l - 1], lvl[l - 2], W, N, s);
        if (e == cudaSuccess) {
            set_boundary2d_kernel<<<blocks_for(4 * (size_t)(N + 1)), 256, 0, s>>>(u, N, g1, stride);
            e = cudaGetLastError();
        }
        note_launches(l >= 2 ? 4 : 2);
        if (e != cudaSuccess) return ctx_cuda(ctx, e, "2D level setup");
        const double fnorm = host_norm(ctx, fh, len, &st);
        if (st) return st;
        if (!std::isfinite(fnorm)) return ctx_fail(ctx, EXCMG_ERR_NAN, "2D right-hand side is not finite");
        if (l <= 1) {   // Alg. 1's direct solves
            if ((st = dsolve2d(ctx, N, bc_kind, fh, u))) return st;
            const double rn = residual2d(ctx, N, bc_kind, fh, u, &st);
            if (st) return st;
            rel = fnorm > 0.0 ? rn / fnorm : 0.0;
        } else {
            const int i = l - 1;
            const double eps = params->tol_mode == EXCMG_TOL_PAPER ? params->tol * std::pow(10.0, (double)(i - L))
                                                                   : params->tol;
            double rn = residual2d(ctx, N, bc_kind, fh, u, &st);
            if (st) return st;
            rel = fnorm > 0.0 ? rn / fnorm : 0.0;
            if (!std::isfinite(rel)) return ctx_fail(ctx, EXCMG_ERR_NAN, "2D residual is not finite");
            while (rel > eps && iters < params->max_total) {   // Alg. 1's WHILE loop
                int it = 0;
                double rr = 0.0;
                const double prev = rel;
                int cap = params->max_total - iters;
                if (cap > params->max_iter) cap = params->max_iter;
                const int bs = bicg2d_run(ctx, N, bc_kind, fh, u, eps, fnorm, cap, params->check_every, &it, &rr);
                iters += it;
                ++calls;
                if (bs != EXCMG_OK && bs != EXCMG_ERR_NOCONV) return bs;
                rn = residual2d(ctx, N, bc_kind, fh, u, &st);
                if (st) return st;
                rel = rn / fnorm;
                if (!std::isfinite(rel)) return ctx_fail(ctx, EXCMG_ERR_NAN, "2D residual is not finite");
                if (rel > 0.5 * prev) {
                    if (++bad >= 2) {
                        stag = 1;
                        break;
                    }
                } else {
                    bad = 0;
                }
            }
        }
        if (stats) {
            stats->n[l] = N;
            stats->iters[l] = iters;
            stats->calls[l] = calls;
            stats->stagnated[l] = stag;
            stats->relres[l] = rel;
        }
    }
    cudaError_t e = cudaSuccess;
    if (u_h_out) e = cudaMemcpyAsync(u_h_out, lvl[nl - 1], lenf * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && u_tilde_out) {   // Alg. 1's final extrapolation
        exp_true2d_kernel<<<blocks_for(lenf), 256, 0, s>>>(u_tilde_out, lvl[nl - 1], lvl[nl - 2], n_finest);
        e = cudaGetLastError();
        note_launches(1);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return ctx_cuda(ctx, e, "excmg2d_solve output");
}

}  // extern "C"
