// Matrix-free 25-point operator A_h of eq. (sec): the interior scheme of
// eq. (method1) with the fictitious nodes folded onto their mirrors by
// eq. (reflection2) (first kind) or eq. (reflection4) (second kind).
//
// Structure: each CTA owns a TX x TY block of (x, y) columns and marches
// along z.  One z-plane of the input (with a 2-node halo in x and y) sits in
// shared memory at a time; every thread turns it into its plane-local
// partial sums and adds them to five register accumulators, one per output
// plane z-2 .. z+2.  The 25 taps split by plane offset:
//   same plane:  (42 + sigma*c) u  - 12 (4 axis nbrs) + (4 nbrs at 2) + 2 (4 diagonals)
//   planes +-1:  -12 u + 2 (4 axis nbrs)
//   planes +-2:  u
// Values outside the interior (boundary nodes and beyond) read as zero: the
// known boundary values belong to the right-hand side.  A ghost folds onto
// its mirror node, which for every ghost of eq. (method1) is the row's own
// node (the +-2 tap of a node one step from a face), so the folding only
// changes the centre weight by sigma = +1 (first kind) or -1 (second kind)
// per axis on which the node is one step from a face.
//
// The transposed operator gathers over the mirrored tap set (p - d instead
// of p + d).  Each tap d has a partner -d of equal weight and the folding is
// diagonal, so this is the same arithmetic; the flag is kept so that A^T is
// applied as Alg. 2 asks (its shadow recurrence multiplies by A^T).
#include <initializer_list>
#include <utility>

#include "excmg_internal.cuh"
#include "grid_sync.cuh"
#include "march_fx.cuh"
#include "march_pair.cuh"
#include "reduce.cuh"

namespace excmg {
namespace {

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int HX = TX + 4;
constexpr int HY = TY + 4;

template <bool kTranspose>
__global__ void __launch_bounds__(TX * TY)
stencil_f64_kernel(const double* __restrict__ u, double* __restrict__ y, const double* __restrict__ b,
                   int n, double sigma, int kz_per_cta, const int* __restrict__ skip) {
    if (skip != nullptr && *skip) return;
    __shared__ double tile[2][HY][HX];
    const int np = n + 1;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int i0 = 1 + blockIdx.x * TX, j0 = 1 + blockIdx.y * TY;
    const int kz0 = 1 + blockIdx.z * kz_per_cta;
    const int kz1 = min(kz0 + kz_per_cta, n);   // output planes [kz0, kz1)
    const int i = i0 + tx, j = j0 + ty;
    const bool active = (i <= n - 1) && (j <= n - 1);
    const int cxy = (i == 1) + (i == n - 1) + (j == 1) + (j == n - 1);
    // mirrored gather for the transpose: offset -d instead of +d
    const int sgn = kTranspose ? -1 : 1;

    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0, acc4 = 0.0;
    int buf = 0;
    for (int zin = kz0 - 2; zin <= kz1 + 1; ++zin, buf ^= 1) {
        const bool zok = (zin >= 1) && (zin <= n - 1);
        for (int e = tid; e < HX * HY; e += TX * TY) {
            const int ly = e / HX, lx = e - ly * HX;
            const int gi = i0 - 2 + lx, gj = j0 - 2 + ly;
            double v = 0.0;
            if (zok && gi >= 1 && gi <= n - 1 && gj >= 1 && gj <= n - 1)
                v = u[((size_t)zin * np + gj) * np + gi];
            tile[buf][ly][lx] = v;
        }
        __syncthreads();
        const int cy = ty + 2, cx = tx + 2;
        const double a = tile[buf][cy][cx];
        const double n4 = tile[buf][cy][cx - sgn] + tile[buf][cy][cx + sgn] +
                          tile[buf][cy - sgn][cx] + tile[buf][cy + sgn][cx];
        const double f4 = tile[buf][cy][cx - 2 * sgn] + tile[buf][cy][cx + 2 * sgn] +
                          tile[buf][cy - 2 * sgn][cx] + tile[buf][cy + 2 * sgn][cx];
        const double d4 = tile[buf][cy - sgn][cx - sgn] + tile[buf][cy - sgn][cx + sgn] +
                          tile[buf][cy + sgn][cx - sgn] + tile[buf][cy + sgn][cx + sgn];
        const int cz = (zin == 1) + (zin == n - 1);
        const double centre = 42.0 + sigma * (double)(cxy + cz);
        const double p0 = centre * a - 12.0 * n4 + f4 + 2.0 * d4;
        const double p1 = -12.0 * a + 2.0 * n4;
        acc0 += a;
        acc1 += p1;
        acc2 += p0;
        acc3 += p1;
        acc4 += a;
        const int zo = zin - 2;   // this output plane has all five contributions now
        if (active && zo >= kz0 && zo < kz1) {
            const size_t o = ((size_t)zo * np + j) * np + i;
            y[o] = b ? (b[o] - acc0) : acc0;
        }
        acc0 = acc1;
        acc1 = acc2;
        acc2 = acc3;
        acc3 = acc4;
        acc4 = 0.0;
    }
}

// y = A u (or y = b - A u): the single-field march of march_fx.cuh, three
// CTAs per SM (the march waits on each plane's loads, and 24 resident warps
// hide more of that latency than 16).
__global__ void __launch_bounds__(FX_NT, 3)
stencil_fx_kernel(FxFields fl, const double* __restrict__ b, int n, int sigma, int kz_per_cta,
                  const int* __restrict__ skip) {
    if (skip != nullptr && *skip) return;
    const int kz0 = 1 + blockIdx.z * kz_per_cta;
    const int kz1 = min(kz0 + kz_per_cta, n);
    (void)fx_march<1, false>(fl, b, n, sigma, blockIdx.x, blockIdx.y, kz0, kz1);
}

// The operator launch of the default Bi-CG schedule on grids above 64^3:
// q = A p, q* = A^T p*, sigma = (p*, q) and alpha = rho / sigma (Alg. 2),
// with the copy-ahead march of march_pair.cuh (bit for bit the results of
// fx_march<2, true>).  A CTA whose slab holds a node where p*
// differs from p (a caller-chosen r*_0) runs the general two-field march
// instead.  kElide: the shadow-elided mode (p only, q only; the same sums).
constexpr bool kPairCvt = true;   // outputs rounded by the hardware conversion

// the general two-field march, kept out of line: it runs only where p* != p
__device__ __noinline__ double pair_two_field(const double* p, const double* ps, double* q, double* qs, int n,
                                              int sigma, int bx, int by, int kz0, int kz1) {
    const FxFields fl{{p, ps}, {q, qs}, {nullptr, nullptr}, {nullptr, nullptr}, 0.0};
    return fx_march<2, true>(fl, nullptr, n, sigma, bx, by, kz0, kz1);
}

// Launch bounds: the two-field kernel at two CTAs per SM (up to 128
// registers: measured 1.27 ms against 1.41 ms per 512^3 launch at three CTAs
// and 80 registers, where the compiler recomputes values it cannot keep),
// the elided one at three (1.02 against 1.06 ms).
template <bool kElide>
__global__ void __launch_bounds__(PP_NT, kElide ? 3 : 2)
stencil_pair_kernel(const double* __restrict__ p, const double* __restrict__ ps, double* __restrict__ q,
                    double* __restrict__ qs, int n, int sigma, int kz_per_cta, double* partials, BicgState* st) {
    extern __shared__ __align__(128) unsigned char pp_smem[];
    if (st->done) return;
    const int kz0 = 1 + blockIdx.z * kz_per_cta;
    const int kz1 = min(kz0 + kz_per_cta, n);
    double dot = 0.0;
    const bool fast = pp_march<kElide, kPairCvt>(p, ps, q, qs, n, sigma, blockIdx.x, blockIdx.y, kz0, kz1,
                                                pp_smem, &dot);
    if constexpr (!kElide) {
        if (!fast) {
            __syncthreads();
            dot = pair_two_field(p, ps, q, qs, n, sigma, blockIdx.x, blockIdx.y, kz0, kz1);
        }
    }
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

// The fused schedule's operator launch: p = r + beta p_prev (and p*) formed
// on every loaded node, the nodes the CTA owns written to (pn, psn), then
// q = A p, q* = A^T p*, sigma and alpha, with the copy-ahead march (bit for
// bit the results of fx_march<2, true, true>).  A CTA whose slab
// holds a node where r* != r or p*_prev != p_prev runs the general march.
__device__ __noinline__ double pair_two_field_dir(const double* r, const double* rs, const double* pp,
                                                  const double* psp, double* pn, double* psn, double* q, double* qs,
                                                  double beta, int n, int sigma, int kz0, int kz1) {
    FxFields fl{{pp, psp}, {q, qs}, {r, rs}, {pn, psn}, beta};
    return fx_march<2, true, true>(fl, nullptr, n, sigma, blockIdx.x, blockIdx.y, kz0, kz1);
}

template <bool kElide>
__global__ void __launch_bounds__(PP_NT, 2)
stencil_pair_dir_kernel(const double* __restrict__ r, const double* __restrict__ rs, const double* __restrict__ pp,
                        const double* __restrict__ psp, double* __restrict__ pn, double* __restrict__ psn,
                        double* __restrict__ q, double* __restrict__ qs, int n, int sigma, int kz_per_cta,
                        double* partials, BicgState* st) {
    extern __shared__ __align__(128) unsigned char pp_smem[];
    if (st->done) return;
    const int kz0 = 1 + blockIdx.z * kz_per_cta;
    const int kz1 = min(kz0 + kz_per_cta, n);
    const PairDir dir{r, rs, pn, psn, st->beta};
    double dot = 0.0;
    const bool fast = pp_march<kElide, kPairCvt, true>(pp, psp, q, qs, n, sigma, blockIdx.x, blockIdx.y, kz0, kz1,
                                                      pp_smem, &dot, dir);
    if constexpr (!kElide) {
        if (!fast) {
            __syncthreads();
            dot = pair_two_field_dir(r, rs, pp, psp, pn, psn, q, qs, dir.beta, n, sigma, kz0, kz1);
        }
    }
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

// A u at one interior node (i, j, k) with the integer arithmetic, without
// shared memory: the node's own 25 taps are put on the scale of their
// largest exponent and summed exactly.  Used where grids are so small that
// a z-march would be all latency.
__device__ __forceinline__ double fx_point(const double* __restrict__ u, int n, int sigma, int i, int j, int k) {
    const int np = n + 1;
    auto val = [&](int a, int b, int c) -> double {
        if (a < 1 || a > n - 1 || b < 1 || b > n - 1 || c < 1 || c > n - 1) return 0.0;
        return u[((size_t)c * np + b) * np + a];
    };
    const double ctr = val(i, j, k);
    double ax[6], far[6], dg[12];
    ax[0] = val(i - 1, j, k); ax[1] = val(i + 1, j, k); ax[2] = val(i, j - 1, k);
    ax[3] = val(i, j + 1, k); ax[4] = val(i, j, k - 1); ax[5] = val(i, j, k + 1);
    far[0] = val(i - 2, j, k); far[1] = val(i + 2, j, k); far[2] = val(i, j - 2, k);
    far[3] = val(i, j + 2, k); far[4] = val(i, j, k - 2); far[5] = val(i, j, k + 2);
    dg[0] = val(i - 1, j - 1, k); dg[1] = val(i - 1, j + 1, k); dg[2] = val(i + 1, j - 1, k); dg[3] = val(i + 1, j + 1, k);
    dg[4] = val(i - 1, j, k - 1); dg[5] = val(i + 1, j, k - 1); dg[6] = val(i, j - 1, k - 1); dg[7] = val(i, j + 1, k - 1);
    dg[8] = val(i - 1, j, k + 1); dg[9] = val(i + 1, j, k + 1); dg[10] = val(i, j - 1, k + 1); dg[11] = val(i, j + 1, k + 1);
    int E = max(1, exponent_of(ctr));
#pragma unroll
    for (int t = 0; t < 6; ++t) E = max(E, max(exponent_of(ax[t]), exponent_of(far[t])));
#pragma unroll
    for (int t = 0; t < 12; ++t) E = max(E, exponent_of(dg[t]));
    long long s_ax = 0, s_far = 0, s_dg = 0;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
        s_ax += to_fixed(ax[t], E);
        s_far += to_fixed(far[t], E);
    }
#pragma unroll
    for (int t = 0; t < 12; ++t) s_dg += to_fixed(dg[t], E);
    const int c = (i == 1) + (i == n - 1) + (j == 1) + (j == n - 1) + (k == 1) + (k == n - 1);
    const long long acc = (long long)(42 + sigma * c) * to_fixed(ctr, E) - 12 * s_ax + s_far + 2 * s_dg;
    return fx_result(acc, E, E == 0x7FF);
}

// ---------------------------------------------------------------------------
// Bi-CG iterations of a small grid in one cooperative launch.  On grids of a
// few tens of thousands of unknowns every kernel of an iteration lasts a few
// microseconds and launch gaps dominate; here all CTAs stay resident and run
// the three phases of an iteration (operator pair + sigma, x/r/r* update +
// (r*, r), (r, r), direction update) separated by grid barriers.  Every CTA
// adds the per-CTA partial sums itself, in CTA order, so all CTAs derive the
// same alpha, beta and stopping decision.  The barrier spins a bounded
// number of times; if it gives up, every CTA leaves and the state reports a
// timeout.
struct BicgVectors {
    double* x;
    double* r;
    double* rs;
    double* p;
    double* ps;
    double* q;
    double* qs;
};

// Sum of component c of the per-CTA partials, in CTA order (every CTA).
__device__ __forceinline__ double all_partials(const double* partials, int c, double* sh) {
    const int G = flat_grid();
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    double v = 0.0;
    for (int b = tid; b < G; b += nthreads) v += __ldcg(&partials[c * G + b]);
    v = block_sum(v, sh);
    __shared__ double bc;
    if (thread0()) bc = v;
    __syncthreads();
    v = bc;
    __syncthreads();
    return v;
}

// kElide: the shadow-elided mode (not the paper's Alg. 2 as printed): r*,
// p*, A^T p* are not stored because they equal r, p, A p bit for bit (the
// integer operator is symmetric and r*_0 = r_0); v.rs, v.ps, v.ps2, v.qs are
// unused and the iterates are the same bits as with kElide = false.
// Three phases per iteration: operator pair with sigma; x, r, r* update
// with (r*, r) and (r, r); direction update.
template <bool kPointwise, bool kElide>
__global__ void __launch_bounds__(FX_NT, 2)
bicg_persistent_kernel(BicgVectors v, size_t len, int n, int sigma, int gx, int gy, int slabs, int kz_per,
                       int iters, double* partials, BicgState* st, GridBarrier gb) {
    __shared__ double sh[32];
    const unsigned int G = gridDim.x;
    const int units = gx * gy * slabs;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nthreads = blockDim.x * blockDim.y;
    extern __shared__ __align__(128) unsigned char persistent_stage_smem[];
    double rho = st->rho, rr = st->rr, alpha = st->alpha, beta = st->beta, sigma_s = st->sigma;
    int iter = st->iter, status = st->status, done = st->done;
    const int max_iter = st->max_iter;
    const double stop = st->tol * st->bnorm;
    bool ok = true;
    for (int it = 0; it < iters && !done && ok; ++it) {
        // phase A: q = A p, qs = A^T ps, sigma = (ps, q); per node on the
        // smallest grids, by z-marching tiles otherwise
        double dot = 0.0;
        if (kPointwise) {
            const int m = n - 1, np = n + 1;
            const long long pts = (long long)m * m * m;
            for (long long t = (long long)blockIdx.x * nthreads + tid; t < pts; t += (long long)G * nthreads) {
                const int i = (int)(t % m) + 1, j = (int)((t / m) % m) + 1, k = (int)(t / ((long long)m * m)) + 1;
                const size_t o = ((size_t)k * np + j) * np + i;
                const double qv = fx_point(v.p, n, sigma, i, j, k);
                v.q[o] = qv;
                if (kElide) {
                    dot += v.p[o] * qv;
                } else {
                    v.qs[o] = fx_point(v.ps, n, sigma, i, j, k);
                    dot += v.ps[o] * qv;
                }
            }
        } else {
            for (int u = blockIdx.x; u < units; u += G) {
                const int bx = u % gx, by = (u / gx) % gy, bz = u / (gx * gy);
                const int kz0 = 1 + bz * kz_per;
                const int kz1 = min(kz0 + kz_per, n);
                // the copy-ahead march (same sums as fx_march<2, true>); the
                // CTA's previous unit is done with the shared buffers
                __syncthreads();
                double dd = 0.0;
                if (pp_march<kElide, kPairCvt>(v.p, v.ps, v.q, v.qs, n, sigma, bx, by, kz0, kz1,
                                               persistent_stage_smem, &dd)) {
                    dot += dd;
                } else if constexpr (!kElide) {
                    __syncthreads();
                    dot += pair_two_field(v.p, v.ps, v.q, v.qs, n, sigma, bx, by, kz0, kz1);
                }
            }
        }
        dot = block_sum(dot, sh);
        if (thread0()) partials[blockIdx.x] = dot;
        if (!(ok = grid_sync(gb, G))) break;
        sigma_s = all_partials(partials, 0, sh);
        if (!(rho != 0.0 && isfinite(rho)) || !(sigma_s != 0.0 && isfinite(sigma_s))) {
            status = kBreakdown;
            done = 1;
            break;
        }
        alpha = rho / sigma_s;
        // phase B: x += alpha p; r -= alpha q; r* -= alpha q*; (r*, r), (r, r)
        // (entries t, t + S of this thread loaded together,
        // then updated and summed in index order)
        double vr = 0.0, vrr = 0.0;
        const double* const pcur = v.p;
        bool twin = true;   // as in bicg_update_kernel: vr == vrr so far
        const size_t S = (size_t)G * nthreads;
        constexpr int kB = kPointwise ? 1 : 2;   // entries per thread loaded together
        for (size_t t0 = (size_t)blockIdx.x * nthreads + tid; t0 < len; t0 += kB * S) {
            double xv[kB], pv[kB], rv[kB], qv[kB], rsv[kB], qsv[kB];
#pragma unroll
            for (int k = 0; k < kB; ++k) {
                const size_t t = t0 + k * S;
                if (t < len) {
                    xv[k] = v.x[t];
                    pv[k] = pcur[t];
                    rv[k] = v.r[t];
                    qv[k] = v.q[t];
                    if (!kElide) {
                        rsv[k] = v.rs[t];
                        qsv[k] = v.qs[t];
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < kB; ++k) {
                const size_t t = t0 + k * S;
                if (t >= len) break;
                v.x[t] = xv[k] + alpha * pv[k];
                const double rn = rv[k] - alpha * qv[k];
                v.r[t] = rn;
                if (kElide) {
                    vrr += rn * rn;
                    continue;
                }
                if (__double_as_longlong(rsv[k]) == __double_as_longlong(rv[k]) &&
                    __double_as_longlong(qsv[k]) == __double_as_longlong(qv[k])) {
                    v.rs[t] = rn;
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
                    const double rsn = rsv[k] - alpha * qsv[k];
                    v.rs[t] = rsn;
                    vr += rsn * rn;
                    vrr += rn * rn;
                }
            }
        }
        if (twin) vr = vrr;
        vr = block_sum(vr, sh);
        vrr = block_sum(vrr, sh);
        if (thread0()) {
            partials[G + blockIdx.x] = vr;
            partials[2 * G + blockIdx.x] = vrr;
        }
        if (!(ok = grid_sync(gb, G))) break;
        const double rho_new = all_partials(partials, 1, sh);
        rr = all_partials(partials, 2, sh);
        beta = rho_new / rho;
        rho = rho_new;
        ++iter;
        if (sqrt(rr) <= stop) {
            status = kConverged;
            done = 1;
            break;
        }
        if (iter >= max_iter) {
            status = kCapped;
            done = 1;
            break;
        }
        {
            // phase C: p = r + beta p; p* = r* + beta p*
            for (size_t t0 = (size_t)blockIdx.x * nthreads + tid; t0 < len; t0 += kB * S) {
                double rv[kB], pv[kB], rsv[kB], psv[kB];
#pragma unroll
                for (int k = 0; k < kB; ++k) {
                    const size_t t = t0 + k * S;
                    if (t < len) {
                        rv[k] = v.r[t];
                        pv[k] = v.p[t];
                        if (!kElide) {
                            rsv[k] = v.rs[t];
                            psv[k] = v.ps[t];
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < kB; ++k) {
                    const size_t t = t0 + k * S;
                    if (t >= len) break;
                    v.p[t] = rv[k] + beta * pv[k];
                    if (!kElide) v.ps[t] = rsv[k] + beta * psv[k];
                }
            }
            if (!(ok = grid_sync(gb, G))) break;
        }
    }
    if (blockIdx.x == 0 && thread0()) {
        if (!ok) {
            status = kTimeout;
            done = 1;
        }
        st->rho = rho;
        st->rr = rr;
        st->alpha = alpha;
        st->beta = beta;
        st->sigma = sigma_s;
        st->iter = iter;
        st->status = status;
        st->done = done;
    }
}

__global__ void zero_boundary_kernel(double* __restrict__ y, int n) {
    // one thread per node of the six faces (faces overlap at edges: harmless)
    const int np = n + 1;
    const size_t per_face = (size_t)np * np;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < 6 * per_face;
         t += (size_t)gridDim.x * blockDim.x) {
        const int face = (int)(t / per_face);
        const size_t r = t - face * per_face;
        const int a = (int)(r % np), bb = (int)(r / np);
        const int fixed = (face & 1) ? n : 0;
        int i, j, k;
        if (face < 2) { i = fixed; j = a; k = bb; }
        else if (face < 4) { i = a; j = fixed; k = bb; }
        else { i = a; j = bb; k = fixed; }
        y[((size_t)k * np + j) * np + i] = 0.0;
    }
}

}  // namespace

namespace {

struct StencilGrid {
    dim3 grid, block;
    int kz_per_cta;
    size_t smem = 0;   // dynamic shared memory per CTA
};

// Column tiles x z-slabs.  The slab count is chosen so that the CTAs fill
// whole waves of the GPU's resident slots (SMs x CTAs per SM) while each
// slab stays long enough that its 4 extra halo planes cost little.
StencilGrid stencil_grid(int n, int tx, int rows, int per_sm) {
    const int m = n - 1;  // interior extent
    StencilGrid g;
    const int gx = (m + tx - 1) / tx, gy = (m + rows - 1) / rows;
    const int tiles = gx * gy;
    const int slots = device_sms() * (per_sm > 0 ? per_sm : 1);
    int best = 1;
    double best_eff = -1.0;
    for (int slabs = 1; slabs <= 64; ++slabs) {
        const int planes = (m + slabs - 1) / slabs;
        if (slabs > 1 && planes < 8) break;
        const long long ctas = (long long)tiles * slabs;
        if (slabs > 1 && ctas > 4096) break;   // keeps the fused reductions' partials small
        const long long waves = (ctas + slots - 1) / slots;
        const double eff = (double)ctas / (double)(waves * slots) * planes / (planes + 4.0);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = slabs;
        }
    }
    g.kz_per_cta = (m + best - 1) / best;
    const int slabs = (m + g.kz_per_cta - 1) / g.kz_per_cta;
    g.grid = dim3(gx, gy, slabs);
    return g;
}

// Resident CTAs per SM of a kernel on the current device (cached per
// kernel and device; opts the kernel in to `smem` bytes of dynamic shared
// memory there first).  Function attributes belong to each device's
// context, so the staged launches call this before every launch.
template <typename K>
int resident_per_sm(K kernel, int threads, size_t smem = 0) {
    return kernel_occupancy((const void*)kernel, threads, smem);
}

template <typename K>
void opt_in_smem(K kernel, size_t smem) {
    (void)kernel_occupancy((const void*)kernel, FX_NT, smem);
}

// The single-field operator launch (A u, b - A u).
StencilGrid fx_grid(int n) {
    const int occ1 = resident_per_sm(stencil_fx_kernel, FX_NT);
    StencilGrid g = stencil_grid(n, FX_TX, FX_OY, occ1);
    g.block = dim3(FX_TX, FX_TY, 1);
    return g;
}

// The copy-ahead operator launch (both modes run on this grid, so that
// sigma adds the same per-CTA partial sums).
StencilGrid pair_grid(int n) {
    const int occ = resident_per_sm(stencil_pair_kernel<false>, PP_NT, pp_smem_bytes<2>());
    StencilGrid g = stencil_grid(n, PP_TX, PP_OY, occ);
    g.block = dim3(PP_TX, PP_TY, 1);
    g.smem = pp_smem_bytes<2>();
    return g;
}

// The fused schedule's launches (both modes on this grid: the same sigma
// partial sums); the first iteration of a call (no previous directions) runs
// stencil_pair_kernel on the same grid.
StencilGrid pair_dir_grid(int n) {
    const int occ = resident_per_sm(stencil_pair_dir_kernel<false>, PP_NT, pp_smem_bytes<4>());
    StencilGrid g = stencil_grid(n, PP_TX, PP_OY, occ);
    g.block = dim3(PP_TX, PP_TY, 1);
    g.smem = pp_smem_bytes<4>();
    return g;
}

StencilGrid f64_grid(int n) {
    const int occ = resident_per_sm(stencil_f64_kernel<false>, TX * TY);
    StencilGrid g = stencil_grid(n, TX, TY, occ);
    g.block = dim3(TX, TY, 1);
    return g;
}

}  // namespace

int stencil_cta_count(int n) {
    unsigned most = 0;
    const StencilGrid g1 = fx_grid(n);
    most = max(most, g1.grid.x * g1.grid.y * g1.grid.z);
    const StencilGrid g = pair_grid(n);
    most = max(most, g.grid.x * g.grid.y * g.grid.z);
    const StencilGrid gd = pair_dir_grid(n);
    most = max(most, gd.grid.x * gd.grid.y * gd.grid.z);
    return (int)most;
}

cudaError_t launch_stencil(const double* u, double* y, const double* b, int n, int bc_kind,
                           bool transpose, const int* skip, cudaStream_t s, int variant) {
    if (variant == kStencilFp64) {
        const StencilGrid g = f64_grid(n);
        const double sigma = bc_kind == 1 ? 1.0 : -1.0;
        if (transpose)
            stencil_f64_kernel<true><<<g.grid, g.block, 0, s>>>(u, y, b, n, sigma, g.kz_per_cta, skip);
        else
            stencil_f64_kernel<false><<<g.grid, g.block, 0, s>>>(u, y, b, n, sigma, g.kz_per_cta, skip);
    } else {
        // A^T u == A u bit for bit in integer arithmetic (see above)
        (void)transpose;
        const StencilGrid g = fx_grid(n);
        FxFields fl{{u, nullptr}, {y, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}, 0.0};
        stencil_fx_kernel<<<g.grid, g.block, 0, s>>>(fl, b, n, bc_kind == 1 ? 1 : -1, g.kz_per_cta, skip);
    }
    return cudaGetLastError();
}

constexpr int kPointwiseMaxN = 32;   // per-node operator on grids up to 32^3

// dynamic shared memory of the z-march variant: the copy-ahead march's
// stages and tiles
size_t persistent_smem(bool pointwise) { return pointwise ? 0 : pp_smem_bytes<2>(); }

int persistent_grid(int n, int* gx, int* gy, int* slabs, int* kz_per) {
    // the elided variants run on the grids of the full ones (same partial
    // sums)
    const int occ_pt = min(2, resident_per_sm(bicg_persistent_kernel<true, false>, FX_NT));
    const int sms = device_sms();
    const int m = n - 1;
    *gx = (m + FX_TX - 1) / FX_TX;
    *gy = (m + FX_OY - 1) / FX_OY;
    *kz_per = m < 8 ? m : (n <= 64 ? 4 : 8);
    *slabs = (m + *kz_per - 1) / *kz_per;
    if (n > kPointwiseMaxN) {
        // z-march: one CTA per SM, and the shortest slabs (at least two
        // planes) that still give every CTA at most one unit per phase.
        // Measured on 48^3 / 64^3: 22.2 / 27.9 us per iteration, against
        // 31.5 / 34.4 with two CTAs per SM and 4-plane slabs (longer waits
        // at the grid barriers, units the CTAs take in two rounds).
        const int G = sms;
        for (int k = 2; k <= 8; ++k) {
            *kz_per = k;
            *slabs = (m + k - 1) / k;
            if ((*gx) * (*gy) * (*slabs) <= G) break;
        }
        return G;
    }
    // one CTA per ~256 interior nodes, at most every resident slot: fewer
    // CTAs keep the grid barriers short on small grids
    const long long pts = (long long)m * m * m;
    long long want = (pts + 255) / 256;
    if (want < 8) want = 8;
    if (want > (long long)sms * occ_pt) want = (long long)sms * occ_pt;
    return (int)want;
}

bool persistent_pointwise(int n) { return n <= kPointwiseMaxN; }

cudaError_t launch_bicg_persistent(double* x, double* r, double* rs, double* p, double* ps, double* q, double* qs,
                                   int n, int bc_kind, int iters, double* partials, BicgState* st,
                                   unsigned int* barrier_words, cudaStream_t s, bool elide) {
    const bool pw = persistent_pointwise(n);
    int gx, gy, slabs, kz_per;
    const int G = persistent_grid(n, &gx, &gy, &slabs, &kz_per);
    cudaError_t e = cudaMemsetAsync(barrier_words, 0, 3 * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    BicgVectors v{x, r, rs, p, ps, q, qs};
    size_t len = node_count(n);
    int sigma = bc_kind == 1 ? 1 : -1;
    GridBarrier gb{barrier_words, barrier_words + 1, (int*)(barrier_words + 2), kBarrierSpinLimit};
    void* args[] = {&v, &len, &n, &sigma, &gx, &gy, &slabs, &kz_per, &iters, &partials, &st, &gb};
    const void* fn;
    if (pw) {
        fn = elide ? (const void*)bicg_persistent_kernel<true, true> : (const void*)bicg_persistent_kernel<true, false>;
    } else {
        opt_in_smem(bicg_persistent_kernel<false, true>, pp_smem_bytes<2>());
        opt_in_smem(bicg_persistent_kernel<false, false>, pp_smem_bytes<2>());
        fn = elide ? (const void*)bicg_persistent_kernel<false, true> : (const void*)bicg_persistent_kernel<false, false>;
    }
    return cudaLaunchCooperativeKernel(fn, dim3(G), dim3(FX_TX, FX_TY, 1), args, persistent_smem(pw), s);
}

cudaError_t launch_bicg_stencil_pair_dir(const double* r, const double* rs, const double* p_prev,
                                         const double* ps_prev, double* p, double* ps, double* q, double* qs, int n,
                                         int bc_kind, double* partials, BicgState* st, cudaStream_t s) {
    const int sg = bc_kind == 1 ? 1 : -1;
    const StencilGrid g = pair_dir_grid(n);
    opt_in_smem(stencil_pair_dir_kernel<false>, g.smem);
    stencil_pair_dir_kernel<false><<<g.grid, g.block, g.smem, s>>>(r, rs, p_prev, ps_prev, p, ps, q, qs, n, sg,
                                                                   g.kz_per_cta, partials, st);
    return cudaGetLastError();
}

cudaError_t launch_bicg_stencil_pair(const double* p, double* q, const double* ps, double* qs, int n,
                                     int bc_kind, double* partials, BicgState* st, cudaStream_t s, bool staged) {
    const int sg = bc_kind == 1 ? 1 : -1;
    if (staged) {   // the fused schedule's first iteration: its grid
        const StencilGrid g = pair_dir_grid(n);
        const size_t smem = pp_smem_bytes<2>();
        opt_in_smem(stencil_pair_kernel<false>, smem);
        stencil_pair_kernel<false><<<g.grid, g.block, smem, s>>>(p, ps, q, qs, n, sg, g.kz_per_cta, partials, st);
    } else {
        const StencilGrid g = pair_grid(n);
        opt_in_smem(stencil_pair_kernel<false>, g.smem);
        stencil_pair_kernel<false><<<g.grid, g.block, g.smem, s>>>(p, ps, q, qs, n, sg, g.kz_per_cta, partials, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_cg_stencil(const double* p, double* q, int n, int bc_kind, double* partials, BicgState* st,
                              cudaStream_t s, bool staged) {
    const int sg = bc_kind == 1 ? 1 : -1;
    if (staged) {   // the fused schedule's first iteration: its grid
        const StencilGrid g = pair_dir_grid(n);
        const size_t smem = pp_smem_bytes<1>();
        opt_in_smem(stencil_pair_kernel<true>, smem);
        stencil_pair_kernel<true><<<g.grid, g.block, smem, s>>>(p, nullptr, q, nullptr, n, sg, g.kz_per_cta, partials,
                                                               st);
    } else {
        const StencilGrid g = pair_grid(n);
        const size_t smem = pp_smem_bytes<1>();
        opt_in_smem(stencil_pair_kernel<true>, smem);
        stencil_pair_kernel<true><<<g.grid, g.block, smem, s>>>(p, nullptr, q, nullptr, n, sg, g.kz_per_cta, partials,
                                                               st);
    }
    return cudaGetLastError();
}

cudaError_t launch_cg_stencil_dir(const double* r, const double* p_prev, double* p, double* q, int n, int bc_kind,
                                  double* partials, BicgState* st, cudaStream_t s) {
    const int sg = bc_kind == 1 ? 1 : -1;
    const StencilGrid g = pair_dir_grid(n);
    const size_t smem = pp_smem_bytes<2>();
    opt_in_smem(stencil_pair_dir_kernel<true>, smem);
    stencil_pair_dir_kernel<true><<<g.grid, g.block, smem, s>>>(r, nullptr, p_prev, nullptr, p, nullptr, q, nullptr,
                                                                n, sg, g.kz_per_cta, partials, st);
    return cudaGetLastError();
}

cudaError_t launch_zero_boundary(double* y, int n, cudaStream_t s) {
    const size_t total = 6 * (size_t)(n + 1) * (n + 1);
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    zero_boundary_kernel<<<blocks, 256, 0, s>>>(y, n);
    return cudaGetLastError();
}

}  // namespace excmg
