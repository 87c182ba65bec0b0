// Vector kernels of Bi-CG (Alg. 2, M = I): the inner products, the iterate
// and residual updates and the direction updates, with the scalars alpha and
// beta formed on the device.
//
// Reductions are deterministic: a fixed grid (kVecBlocks x kVecThreads)
// walks the vectors with a grid stride, each CTA reduces its values by a
// fixed shuffle tree, and the last CTA to finish (atomic ticket) adds the
// per-CTA partials in CTA order.  The same inputs therefore always give the
// same bits, independent of scheduling.
#include "excmg_internal.cuh"
#include "reduce.cuh"

namespace excmg {
namespace {

__global__ void __launch_bounds__(kVecThreads)
dot_kernel(const double* __restrict__ a, const double* __restrict__ b, size_t len,
           double* partials, unsigned int* ticket, double* out) {
    __shared__ double sh[32];
    __shared__ bool am_last;
    double v = 0.0;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len;
         t += (size_t)gridDim.x * blockDim.x)
        v += a[t] * b[t];
    double s = block_sum(v, sh);
    if (publish_partials(&s, 1, partials, ticket, &am_last)) {
        const double tot = gather_partials(partials, 0, sh);
        if (thread0()) {
            *out = tot;
            *ticket = 0;
        }
    }
}

// (a, a) over the unknowns (interior nodes) of a grid with n intervals:
// for caller-supplied vectors whose boundary entries need not be zero.
__global__ void __launch_bounds__(kVecThreads)
interior_dot_kernel(const double* __restrict__ a, int n, double* partials, unsigned int* ticket, double* out) {
    __shared__ double sh[32];
    __shared__ bool am_last;
    const long long m = n - 1, np = n + 1;
    const long long pts = m * m * m;
    double v = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < pts;
         t += (long long)gridDim.x * blockDim.x) {
        const long long i = t % m + 1, j = (t / m) % m + 1, k = t / (m * m) + 1;
        const double x = a[(k * np + j) * np + i];
        v += x * x;
    }
    double s = block_sum(v, sh);
    if (publish_partials(&s, 1, partials, ticket, &am_last)) {
        const double tot = gather_partials(partials, 0, sh);
        if (thread0()) {
            *out = tot;
            *ticket = 0;
        }
    }
}

// r*_0 = shadow (or r_0), p_0 = r_0, p*_0 = r*_0; rho_0 = (r*_0, r_0),
// rr = (r_0, r_0).
__global__ void __launch_bounds__(kVecThreads)
bicg_init_kernel(const double* __restrict__ r, const double* __restrict__ shadow, double* __restrict__ rs,
                 double* __restrict__ p, double* __restrict__ ps, size_t len, double* partials, BicgState* st) {
    __shared__ double sh[32];
    __shared__ bool am_last;
    double vr = 0.0, vrr = 0.0;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len;
         t += (size_t)gridDim.x * blockDim.x) {
        const double rv = r[t];
        const double sv = shadow ? shadow[t] : rv;
        rs[t] = sv;
        p[t] = rv;
        ps[t] = sv;
        vr += sv * rv;
        vrr += rv * rv;
    }
    double s2[2];
    s2[0] = block_sum(vr, sh);
    s2[1] = block_sum(vrr, sh);
    if (publish_partials(s2, 2, partials, &st->ticket, &am_last)) {
        const double rho = gather_partials(partials, 0, sh);
        const double rr = gather_partials(partials, 1, sh);
        if (thread0()) {
            st->rho = rho;
            st->rr = rr;
            st->iter = 0;
            st->alpha = st->beta = st->sigma = 0.0;
            const bool conv = sqrt(rr) <= st->tol * st->bnorm;
            st->done = (conv || st->max_iter <= 0) ? 1 : 0;
            st->status = conv ? kConverged : (st->max_iter <= 0 ? kCapped : kRunning);
            st->ticket = 0;
        }
    }
}

// sigma_k = (p*_k, A p_k); alpha_k = rho_k / sigma_k.
__global__ void __launch_bounds__(kVecThreads)
bicg_sigma_kernel(const double* __restrict__ ps, const double* __restrict__ q, size_t len,
                  double* partials, BicgState* st) {
    if (st->done) return;
    __shared__ double sh[32];
    __shared__ bool am_last;
    double v = 0.0;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len;
         t += (size_t)gridDim.x * blockDim.x)
        v += ps[t] * q[t];
    double s = block_sum(v, sh);
    if (publish_partials(&s, 1, partials, &st->ticket, &am_last)) {
        const double sigma = gather_partials(partials, 0, sh);
        if (thread0()) {
            const double rho = st->rho;
            st->sigma = sigma;
            if (!(rho != 0.0 && isfinite(rho)) || !(sigma != 0.0 && isfinite(sigma))) {
                st->status = kBreakdown;
                st->done = 1;
            } else {
                st->alpha = rho / sigma;
            }
            st->ticket = 0;
        }
    }
}

// x += alpha p; r -= alpha A p; r* -= alpha A^T p*;
// rho_{k+1} = (r*, r), beta = rho_{k+1} / rho_k; stopping test on ||r||.
// Where r* and A^T p* equal r and A p bit for bit (always so with
// r*_0 = r_0 and the integer operator) the shadow update gives the same
// bits as the primal one and the product r* r equals r r, so it is formed
// once; a thread that meets a differing entry continues with separate sums
// from the identical partial sums it has so far.  FP64 issue is scarce on
// GB300: this saves two of the five FMAs per entry.
__global__ void __launch_bounds__(kVecThreads)
bicg_update_kernel(double* __restrict__ x, const double* __restrict__ p, double* __restrict__ r,
                   const double* __restrict__ q, double* __restrict__ rs,
                   const double* __restrict__ qs, size_t len, double* partials, BicgState* st) {
    if (st->done) return;
    __shared__ double sh[32];
    __shared__ bool am_last;
    const double alpha = st->alpha;
    double vr = 0.0, vrr = 0.0;
    bool twin = true;   // so far every entry of this thread was a twin: vr == vrr
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len;
         t += (size_t)gridDim.x * blockDim.x) {
        x[t] = x[t] + alpha * p[t];
        const double rv = r[t], qv = q[t], rsv = rs[t], qsv = qs[t];
        const double rn = rv - alpha * qv;
        r[t] = rn;
        if (__double_as_longlong(rsv) == __double_as_longlong(rv) &&
            __double_as_longlong(qsv) == __double_as_longlong(qv)) {
            rs[t] = rn;
            if (twin) {
                vrr += rn * rn;
            } else {
                vr += rn * rn;
                vrr += rn * rn;
            }
        } else {
            if (twin) {
                vr = vrr;
                twin = false;
            }
            const double rsn = rsv - alpha * qsv;
            rs[t] = rsn;
            vr += rsn * rn;
            vrr += rn * rn;
        }
    }
    if (twin) vr = vrr;
    double s[2];
    s[0] = block_sum(vr, sh);
    s[1] = block_sum(vrr, sh);
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

// p_{k+1} = r_{k+1} + beta p_k; p*_{k+1} = r*_{k+1} + beta p*_k (one FMA
// where the shadow entries equal the primal ones bit for bit).
__global__ void __launch_bounds__(kVecThreads)
bicg_pupdate_kernel(double* __restrict__ p, const double* __restrict__ r, double* __restrict__ ps,
                    const double* __restrict__ rs, size_t len, const BicgState* st) {
    if (st->done) return;
    const double beta = st->beta;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len;
         t += (size_t)gridDim.x * blockDim.x) {
        const double rv = r[t], pv = p[t], rsv = rs[t], psv = ps[t];
        const double pn = rv + beta * pv;
        p[t] = pn;
        if (__double_as_longlong(rsv) == __double_as_longlong(rv) && __double_as_longlong(psv) == __double_as_longlong(pv))
            ps[t] = pn;
        else
            ps[t] = rsv + beta * psv;
    }
}

// Shadow-elided mode (not Alg. 2 as printed; r* = r and p* = p are not
// stored).  p_0 = r_0, rho_0 = rr = (r_0, r_0): the sums of
// bicg_init_kernel with r*_0 = r_0, in the same order.
__global__ void __launch_bounds__(kVecThreads)
cg_init_kernel(const double* __restrict__ r, double* __restrict__ p, size_t len, double* partials, BicgState* st) {
    __shared__ double sh[32];
    __shared__ bool am_last;
    double vrr = 0.0;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len;
         t += (size_t)gridDim.x * blockDim.x) {
        const double rv = r[t];
        p[t] = rv;
        vrr += rv * rv;
    }
    double s2[2];
    s2[0] = block_sum(vrr, sh);
    s2[1] = s2[0];
    if (publish_partials(s2, 2, partials, &st->ticket, &am_last)) {
        const double rr = gather_partials(partials, 1, sh);
        if (thread0()) {
            st->rho = rr;
            st->rr = rr;
            st->iter = 0;
            st->alpha = st->beta = st->sigma = 0.0;
            const bool conv = sqrt(rr) <= st->tol * st->bnorm;
            st->done = (conv || st->max_iter <= 0) ? 1 : 0;
            st->status = conv ? kConverged : (st->max_iter <= 0 ? kCapped : kRunning);
            st->ticket = 0;
        }
    }
}

// Shadow-elided update: x += alpha p; r -= alpha A p; rho_{k+1} = rr =
// (r, r); beta; stopping test.  Same arithmetic and summation order as
// bicg_update_kernel on twin entries.
__global__ void __launch_bounds__(kVecThreads)
cg_update_kernel(double* __restrict__ x, const double* __restrict__ p, double* __restrict__ r,
                 const double* __restrict__ q, size_t len, double* partials, BicgState* st) {
    if (st->done) return;
    __shared__ double sh[32];
    __shared__ bool am_last;
    const double alpha = st->alpha;
    double vrr = 0.0;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len;
         t += (size_t)gridDim.x * blockDim.x) {
        x[t] = x[t] + alpha * p[t];
        const double rn = r[t] - alpha * q[t];
        r[t] = rn;
        vrr += rn * rn;
    }
    double s[2];
    s[0] = block_sum(vrr, sh);
    s[1] = s[0];
    if (publish_partials(s, 2, partials, &st->ticket, &am_last)) {
        const double rr = gather_partials(partials, 1, sh);
        if (thread0()) {
            st->beta = rr / st->rho;
            st->rho = rr;
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

// Shadow-elided direction update: p = r + beta p.
__global__ void __launch_bounds__(kVecThreads)
cg_pupdate_kernel(double* __restrict__ p, const double* __restrict__ r, size_t len, const BicgState* st) {
    if (st->done) return;
    const double beta = st->beta;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len;
         t += (size_t)gridDim.x * blockDim.x)
        p[t] = r[t] + beta * p[t];
}

}  // namespace

cudaError_t launch_cg_pupdate(double* p, const double* r, size_t len, const BicgState* st, cudaStream_t s) {
    cg_pupdate_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(p, r, len, st);
    return cudaGetLastError();
}

cudaError_t launch_cg_init(const double* r, double* p, size_t len, double* partials, BicgState* st, cudaStream_t s) {
    cg_init_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(r, p, len, partials, st);
    return cudaGetLastError();
}

cudaError_t launch_cg_update(double* x, const double* p, double* r, const double* q, size_t len, double* partials,
                             BicgState* st, cudaStream_t s) {
    cg_update_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(x, p, r, q, len, partials, st);
    return cudaGetLastError();
}

cudaError_t launch_dot(const double* a, const double* b, size_t len, double* partials,
                       unsigned int* ticket, double* out, cudaStream_t s) {
    dot_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(a, b, len, partials, ticket, out);
    return cudaGetLastError();
}

cudaError_t launch_interior_dot(const double* a, int n, double* partials, unsigned int* ticket, double* out,
                                cudaStream_t s) {
    interior_dot_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(a, n, partials, ticket, out);
    return cudaGetLastError();
}

cudaError_t launch_bicg_init(const double* r, const double* shadow, double* rs, double* p, double* ps, size_t len,
                             double* partials, BicgState* st, cudaStream_t s) {
    bicg_init_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(r, shadow, rs, p, ps, len, partials, st);
    return cudaGetLastError();
}

cudaError_t launch_bicg_sigma(const double* ps, const double* q, size_t len, double* partials,
                              BicgState* st, cudaStream_t s) {
    bicg_sigma_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(ps, q, len, partials, st);
    return cudaGetLastError();
}

cudaError_t launch_bicg_update(double* x, const double* p, double* r, const double* q, double* rs,
                               const double* qs, size_t len, double* partials, BicgState* st,
                               cudaStream_t s) {
    bicg_update_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(x, p, r, q, rs, qs, len, partials, st);
    return cudaGetLastError();
}

cudaError_t launch_bicg_pupdate(double* p, const double* r, double* ps, const double* rs, size_t len,
                                const BicgState* st, cudaStream_t s) {
    bicg_pupdate_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(p, r, ps, rs, len, st);
    return cudaGetLastError();
}

}  // namespace excmg
