// FP32 inner solves with FP64 iterative refinement.
//
// On a level, the FP64 outer loop forms the true residual r = f_h - A u
// (integer operator on the FP64 iterate), scales it to unit 2-norm, solves
// the correction equation A e = r / ||r|| approximately with Bi-CG (Alg. 2,
// M = I, r*_0 = r_0) entirely in FP32 -- FP32 vectors, FP32 operator, FP32
// accumulation inside threads and CTAs -- and updates u += ||r|| e in FP64.
// The loop ends on the FP64 true residual test of Alg. 1, with the
// same stagnation rule as the FP64 solver.  The FP32 operator applies A^T
// with the same code as A: A_h is symmetric, so the two are one operator.
//
// Entries of A u for a smooth u are many orders of magnitude below the
// individual terms of the 25-point sum, so FP32 never touches u itself:
// only the correction, whose size shrinks with every outer step.
#include <cmath>

#include "excmg_internal.cuh"
#include "march_f32.cuh"
#include "reduce.cuh"

namespace excmg {
namespace {

// NF = 1: y = A u.  NF = 2 with kDot: q = A p, qs = A ps and
// sigma = (ps, q), alpha = rho / sigma in the last CTA.
template <int NF, bool kDot>
__global__ void __launch_bounds__(S_NT)
stencil_f32_kernel(const float* __restrict__ in0, const float* __restrict__ in1, float* __restrict__ out0,
                   float* __restrict__ out1, int n, float sigma, int kz_per_cta, const int* __restrict__ skip,
                   double* partials, BicgState* st) {
    if (skip != nullptr && *skip) return;
    const int kz0 = 1 + blockIdx.z * kz_per_cta;
    const int kz1 = min(kz0 + kz_per_cta, n);
    const float dot = f32_march<NF, kDot>(in0, in1, out0, out1, n, sigma, blockIdx.x, blockIdx.y, kz0, kz1);
    if (kDot) {
        __shared__ float shf[32];
        __shared__ double sh[32];
        __shared__ bool am_last;
        const double sdot = (double)block_sum(dot, shf);
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

// r*_0 = p_0 = p*_0 = r_0; rho_0 = (r_0, r_0).
__global__ void __launch_bounds__(kVecThreads)
bicg32_init_kernel(const float* __restrict__ r, float* __restrict__ rs, float* __restrict__ p,
                   float* __restrict__ ps, size_t len, double* partials, BicgState* st) {
    __shared__ float shf[32];
    __shared__ double sh[32];
    __shared__ bool am_last;
    float v = 0.f;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len; t += (size_t)gridDim.x * blockDim.x) {
        const float rv = r[t];
        rs[t] = rv;
        p[t] = rv;
        ps[t] = rv;
        v += rv * rv;
    }
    const double s = (double)block_sum(v, shf);
    if (publish_partials(&s, 1, partials, &st->ticket, &am_last)) {
        const double tot = gather_partials(partials, 0, sh);
        if (thread0()) {
            st->rho = tot;
            st->rr = tot;
            st->iter = 0;
            st->alpha = st->beta = st->sigma = 0.0;
            const bool conv = sqrt(tot) <= st->tol * st->bnorm;
            st->done = (conv || st->max_iter <= 0) ? 1 : 0;
            st->status = conv ? kConverged : (st->max_iter <= 0 ? kCapped : kRunning);
            st->ticket = 0;
        }
    }
}

__global__ void __launch_bounds__(kVecThreads)
bicg32_update_kernel(float* __restrict__ x, const float* __restrict__ p, float* __restrict__ r,
                     const float* __restrict__ q, float* __restrict__ rs, const float* __restrict__ qs,
                     size_t len, double* partials, BicgState* st) {
    if (st->done) return;
    __shared__ float shf[32];
    __shared__ double sh[32];
    __shared__ bool am_last;
    const float alpha = (float)st->alpha;
    float vr = 0.f, vrr = 0.f;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len; t += (size_t)gridDim.x * blockDim.x) {
        x[t] = x[t] + alpha * p[t];
        const float rn = r[t] - alpha * q[t];
        const float rsn = rs[t] - alpha * qs[t];
        r[t] = rn;
        rs[t] = rsn;
        vr += rsn * rn;
        vrr += rn * rn;
    }
    double s[2];
    s[0] = (double)block_sum(vr, shf);
    s[1] = (double)block_sum(vrr, shf);
    if (publish_partials(s, 2, partials, &st->ticket, &am_last)) {
        const double rho_new = gather_partials(partials, 0, sh);
        const double rr = gather_partials(partials, 1, sh);
        if (thread0()) {
            st->beta = rho_new / st->rho;
            st->rho = rho_new;
            st->rr = rr;
            st->iter += 1;
            if (sqrt(rr) <= st->tol * st->bnorm) {
                st->status = kConverged;
                st->done = 1;
            } else if (st->iter >= st->max_iter) {
                st->status = kCapped;
                st->done = 1;
            }
            st->ticket = 0;
        }
    }
}

__global__ void __launch_bounds__(kVecThreads)
bicg32_pupdate_kernel(float* __restrict__ p, const float* __restrict__ r, float* __restrict__ ps,
                      const float* __restrict__ rs, size_t len, const BicgState* st) {
    if (st->done) return;
    const float beta = (float)st->beta;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len; t += (size_t)gridDim.x * blockDim.x) {
        p[t] = r[t] + beta * p[t];
        ps[t] = rs[t] + beta * ps[t];
    }
}

// r32 = r / s (s = ||r||_2); the correction e starts at zero.
__global__ void __launch_bounds__(kVecThreads)
scale_to_f32_kernel(const double* __restrict__ r, float* __restrict__ r32, float* __restrict__ e, size_t len,
                    double inv_s) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len; t += (size_t)gridDim.x * blockDim.x) {
        r32[t] = (float)(r[t] * inv_s);
        e[t] = 0.f;
    }
}

// u += s e (FP64); e is zero on the boundary, so u keeps its boundary data.
__global__ void __launch_bounds__(kVecThreads)
add_correction_kernel(double* __restrict__ u, const float* __restrict__ e, size_t len, double s) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len; t += (size_t)gridDim.x * blockDim.x)
        u[t] = u[t] + s * (double)e[t];
}

struct Grid32 {
    dim3 grid, block;
    int kz_per_cta;
};

Grid32 grid32(int n) {
    const int m = n - 1;
    Grid32 g;
    g.block = dim3(S_TX, S_TY, 1);
    const int gx = (m + S_TX - 1) / S_TX, gy = (m + S_OY - 1) / S_OY;
    const int tiles = gx * gy;
    int slabs = (152 * 8 + tiles - 1) / tiles;
    const int max_slabs = (m + 7) / 8;
    if (slabs > max_slabs) slabs = max_slabs;
    if (slabs < 1) slabs = 1;
    g.kz_per_cta = (m + slabs - 1) / slabs;
    slabs = (m + g.kz_per_cta - 1) / g.kz_per_cta;
    g.grid = dim3(gx, gy, slabs);
    return g;
}

}  // namespace

int stencil32_cta_count(int n) {
    const Grid32 g = grid32(n);
    return (int)(g.grid.x * g.grid.y * g.grid.z);
}

// FP32 Bi-CG on A e = b32 from e = 0 (Alg. 2, M = I, r*_0 = r_0).
static int bicg32_run(excmg_ctx* ctx, int n, int bc_kind, const float* b32, float* e, double tol, int max_iter,
                      int check_every, int* iters_out) {
    const size_t len = node_count(n);
    const size_t bytes = len * sizeof(float);
    int st = EXCMG_OK;
    float* r = (float*)ctx_buffer(ctx, "b32_r", bytes, &st);
    float* rs = st ? nullptr : (float*)ctx_buffer(ctx, "b32_rs", bytes, &st);
    float* p = st ? nullptr : (float*)ctx_buffer(ctx, "b32_p", bytes, &st);
    float* ps = st ? nullptr : (float*)ctx_buffer(ctx, "b32_ps", bytes, &st);
    float* q = st ? nullptr : (float*)ctx_buffer(ctx, "b32_q", bytes, &st);
    float* qs = st ? nullptr : (float*)ctx_buffer(ctx, "b32_qs", bytes, &st);
    if (st) return st;
    cudaStream_t s = ctx->stream;
    const Grid32 g = grid32(n);
    if ((int)(g.grid.x * g.grid.y * g.grid.z) > kMaxPartials)
        return ctx_fail(ctx, EXCMG_ERR_ARG, "grid too large for the FP32 solver's reduction buffer");
    const float sigma = bc_kind == 1 ? 1.f : -1.f;
    BicgState init{};
    init.bnorm = 1.0;   // b32 has unit 2-norm
    init.tol = tol;
    init.max_iter = max_iter;
    *ctx->host_state = init;
    cudaError_t err = cudaMemcpyAsync(ctx->state, ctx->host_state, sizeof(BicgState), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) err = cudaMemsetAsync(q, 0, bytes, s);
    if (err == cudaSuccess) err = cudaMemsetAsync(qs, 0, bytes, s);
    // e = 0, so r_0 = b32
    if (err == cudaSuccess) err = cudaMemcpyAsync(r, b32, bytes, cudaMemcpyDeviceToDevice, s);
    if (err == cudaSuccess) {
        bicg32_init_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(r, rs, p, ps, len, ctx->partials, ctx->state);
        err = cudaGetLastError();
    }
    note_launches(1);
    if (err != cudaSuccess) return ctx_cuda(ctx, err, "FP32 Bi-CG setup");
    if (check_every < 1) check_every = 1;
    for (;;) {
        err = ctx_read_back(ctx, ctx->host_state, ctx->state, sizeof(BicgState));
        if (err == cudaSuccess) err = cudaStreamSynchronize(s);
        if (err != cudaSuccess) return ctx_cuda(ctx, err, "FP32 Bi-CG state read");
        if (ctx->host_state->done) break;
        int batch = check_every;
        const int left = max_iter - ctx->host_state->iter;
        if (batch > left) batch = left;
        for (int it = 0; it < batch && err == cudaSuccess; ++it) {
            stencil_f32_kernel<2, true><<<g.grid, g.block, 0, s>>>(p, ps, q, qs, n, sigma, g.kz_per_cta,
                                                                   &ctx->state->done, ctx->partials, ctx->state);
            bicg32_update_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(e, p, r, q, rs, qs, len, ctx->partials,
                                                                    ctx->state);
            bicg32_pupdate_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(p, r, ps, rs, len, ctx->state);
            err = cudaGetLastError();
        }
        note_launches(3LL * batch);
        if (err != cudaSuccess) return ctx_cuda(ctx, err, "FP32 Bi-CG iteration");
    }
    if (iters_out) *iters_out = ctx->host_state->iter;
    if (!std::isfinite(ctx->host_state->rr)) return ctx_fail(ctx, EXCMG_ERR_NAN, "FP32 Bi-CG residual is not finite");
    if (ctx->host_state->status == kBreakdown) return ctx_fail(ctx, EXCMG_ERR_BREAKDOWN, "FP32 Bi-CG breakdown");
    return EXCMG_OK;
}

int mixed_level_solve(excmg_ctx* ctx, int n, int bc_kind, const double* fh, double* u, double fnorm, double eps,
                      double inner_tol, int max_inner, int max_total, int check_every, int* iters_out,
                      int* outer_out, int* stag_out, double* rel_out) {
    const size_t len = node_count(n);
    int st = EXCMG_OK;
    double* r = ctx_buffer(ctx, "res", len * sizeof(double), &st);
    float* r32 = st ? nullptr : (float*)ctx_buffer(ctx, "mx_r32", len * sizeof(float), &st);
    float* e = st ? nullptr : (float*)ctx_buffer(ctx, "mx_e", len * sizeof(float), &st);
    if (st) return st;
    cudaStream_t s = ctx->stream;
    int iters = 0, outer = 0, bad = 0, stag = 0;
    double rel = 0.0;
    for (;;) {
        // FP64 true residual r = f_h - A u and its norm
        cudaError_t err = cudaMemsetAsync(r, 0, len * sizeof(double), s);
        if (err == cudaSuccess) err = launch_stencil(u, r, fh, n, bc_kind, false, nullptr, s, ctx->stencil_variant);
        note_launches(1);
        if (err != cudaSuccess) return ctx_cuda(ctx, err, "refinement residual");
        double rn = 0.0;
        if ((st = interior_norm(ctx, n, r, &rn))) return st;
        const double prev = rel;
        rel = fnorm > 0.0 ? rn / fnorm : 0.0;
        if (!std::isfinite(rel)) return ctx_fail(ctx, EXCMG_ERR_NAN, "residual is not finite");
        if (outer > 0) {
            // a refinement step that removes less than a tenth of the
            // residual twice in a row has met the FP32 solver's limit
            if (rel > 0.9 * prev) {
                if (++bad >= 2) { stag = 1; break; }
            } else {
                bad = 0;
            }
        }
        if (rel <= eps || iters >= max_total || rn == 0.0) break;
        // FP32 correction solve on A e = r / ||r||
        scale_to_f32_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(r, r32, e, len, 1.0 / rn);
        note_launches(1);
        if ((err = cudaGetLastError()) != cudaSuccess) return ctx_cuda(ctx, err, "scale residual");
        int cap = max_total - iters;
        if (cap > max_inner) cap = max_inner;
        int it = 0;
        if ((st = bicg32_run(ctx, n, bc_kind, r32, e, inner_tol, cap, check_every, &it))) return st;
        iters += it;
        ++outer;
        add_correction_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(u, e, len, rn);
        note_launches(1);
        if ((err = cudaGetLastError()) != cudaSuccess) return ctx_cuda(ctx, err, "refinement update");
    }
    *iters_out = iters;
    *outer_out = outer;
    *stag_out = stag;
    *rel_out = rel;
    return EXCMG_OK;
}

}  // namespace excmg
