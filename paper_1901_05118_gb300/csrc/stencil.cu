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
#include "excmg_internal.cuh"
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

// ---------------------------------------------------------------------------
// Exact-integer variant.  GB300 issues FP64 arithmetic at a small fraction of
// its integer rate, while the 25 weights are small integers (|w| summing to
// 144).  Each input plane of the CTA is mapped to 64-bit integers on one
// power-of-two scale: a double with biased exponent e and 53-bit significand
// m becomes m >> (E - e), E being the largest exponent the CTA has met so
// far; all sums are then exact integer additions (144 * 2^53 < 2^61), and
// only the final value is rounded once back to double.  The result differs
// from the exact weighted sum by less than 144 units of 2^(E-1075) plus the
// final rounding, i.e. at most about 3.2e-14 of the largest input magnitude
// the CTA reads (FP64 summation of the 25 terms carries errors of the same
// order).  When E grows, the running
// accumulators are shifted to the new scale.  A plane holding a non-finite
// value turns the CTA's remaining outputs into NaN.
__device__ __forceinline__ long long to_fixed(double v, int E) {
    const unsigned hi = (unsigned)__double2hiint(v);
    const unsigned lo = (unsigned)__double2loint(v);
    const int e = (int)((hi >> 20) & 0x7FFu);
    unsigned mh = hi & 0xFFFFFu;
    int ee = 1;
    if (e) { mh |= 0x100000u; ee = e; }
    unsigned long long m = ((unsigned long long)mh << 32) | lo;
    const int d = E - ee;
    m = d < 64 ? (m >> d) : 0ull;
    const long long r = (long long)m;
    return ((int)hi < 0) ? -r : r;
}

// Y * 2^(E - 1075), rounded to nearest even; valid for 53 <= E <= 2037 and
// |Y| < 2^62.
__device__ __forceinline__ double from_fixed(long long Y, int E) {
    if (Y == 0) return 0.0;
    const unsigned long long sgn = Y < 0 ? (1ull << 63) : 0ull;
    unsigned long long a = Y < 0 ? (unsigned long long)(-Y) : (unsigned long long)Y;
    const int lz = __clzll((long long)a);
    a <<= lz;
    unsigned long long mant = a >> 11;
    const unsigned rem = (unsigned)(a & 0x7FFull);
    if (rem > 0x400u || (rem == 0x400u && (mant & 1ull))) mant += 1ull;
    const unsigned long long bits = sgn + ((unsigned long long)(E + 11 - lz - 1) << 52) + mant;
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ int exponent_of(double v) {
    return (int)(((unsigned)__double2hiint(v) >> 20) & 0x7FFu);
}

// Register-blocked integer kernel.  A CTA of FX_TX x FX_TY threads owns
// FX_TX x (FX_TY * FX_RY) output columns; each thread produces FX_RY = 2
// vertically adjacent columns, which share 9 of their 18 shared-memory reads.
// NF fields are marched together through the same z-planes (NF = 2 applies A
// to p and A^T to p* in one pass for Bi-CG); field f has its own running
// scale exponent E[f].  Each thread's halo-load slots are the same on every
// plane, so their offsets are computed once.
//
// The transposed operator gathers over the mirrored tap set; every tap d of
// eq. (method1) has a partner -d of equal weight and integer sums do not
// depend on order, so A^T u and A u come out bit for bit equal here.
//
// With kDot the kernel also forms the Bi-CG scalar sigma = (p*, A p) of
// Alg. 2 (field 1's input against field 0's output) and, in the last CTA,
// alpha = rho / sigma.
constexpr int FX_TX = 32;
constexpr int FX_TY = 8;
constexpr int FX_RY = 2;
constexpr int FX_OY = FX_TY * FX_RY;                 // output rows per CTA
constexpr int FX_HX = FX_TX + 4;
constexpr int FX_HY = FX_OY + 4;
constexpr int FX_NT = FX_TX * FX_TY;
constexpr int FX_SLOTS = (FX_HX * FX_HY + FX_NT - 1) / FX_NT;

struct FxFields {
    const double* in[2];
    double* out[2];
};

__device__ __forceinline__ double fx_result(long long acc, int E, bool poisoned) {
    if (poisoned) return __longlong_as_double(0x7FF8000000000000ll);
    if (E >= 53 && E <= 2037) return from_fixed(acc, E);
    return ldexp((double)acc, E - 1075);
}

template <int NF, bool kDot>
__global__ void __launch_bounds__(FX_NT)
stencil_fx_kernel(FxFields fl, const double* __restrict__ b, int n, int sigma, int kz_per_cta,
                  const int* __restrict__ skip, double* partials, BicgState* st) {
    if (skip != nullptr && *skip) return;
    __shared__ long long tile[NF][FX_HY * FX_HX];
    __shared__ int wmax[NF][FX_NT / 32];
    const int np = n + 1;
    const size_t plane = (size_t)np * np;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * FX_TX + tx;
    const int lane = tid & 31;
    const int i0 = 1 + blockIdx.x * FX_TX, j0 = 1 + blockIdx.y * FX_OY;
    const int kz0 = 1 + blockIdx.z * kz_per_cta;
    const int kz1 = min(kz0 + kz_per_cta, n);

    // halo-load slots of this thread: in-plane offset (-1: outside the
    // interior, reads as zero) and shared-memory index (-1: no slot)
    int soff[FX_SLOTS], sidx[FX_SLOTS];
#pragma unroll
    for (int r = 0; r < FX_SLOTS; ++r) {
        const int e = tid + r * FX_NT;
        soff[r] = -1;
        sidx[r] = -1;
        if (e < FX_HX * FX_HY) {
            const int ly = e / FX_HX, lx = e - ly * FX_HX;
            const int gi = i0 - 2 + lx, gj = j0 - 2 + ly;
            sidx[r] = e;
            if (gi >= 1 && gi <= n - 1 && gj >= 1 && gj <= n - 1) soff[r] = gj * np + gi;
        }
    }
    const int i = i0 + tx, ja = j0 + ty * FX_RY;
    const bool act0 = (i <= n - 1) && (ja <= n - 1);
    const bool act1 = (i <= n - 1) && (ja + 1 <= n - 1);
    const int cx = (i == 1) + (i == n - 1);
    const int c0 = cx + (ja == 1) + (ja == n - 1);
    const int c1 = cx + (ja + 1 == 1) + (ja + 1 == n - 1);
    const int ry = ty * FX_RY + 2, rx = tx + 2;   // tile coordinates of the first output

    long long acc[NF][FX_RY][5];
    int E[NF];
    bool poisoned[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
#pragma unroll
        for (int q = 0; q < FX_RY; ++q)
#pragma unroll
            for (int k = 0; k < 5; ++k) acc[f][q][k] = 0;
        E[f] = 1;
        poisoned[f] = false;
    }
    double dot = 0.0;

    for (int zin = kz0 - 2; zin <= kz1 + 1; ++zin) {
        const bool zok = (zin >= 1) && (zin <= n - 1);
        const size_t zbase = zok ? (size_t)zin * plane : 0;
        double v[NF][FX_SLOTS];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            int emax = 0;
#pragma unroll
            for (int r = 0; r < FX_SLOTS; ++r) {
                v[f][r] = (zok && soff[r] >= 0) ? fl.in[f][zbase + soff[r]] : 0.0;
                emax = max(emax, exponent_of(v[f][r]));
            }
            emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)emax);
            if (lane == 0) wmax[f][tid >> 5] = emax;
        }
        __syncthreads();   // also: every thread is done reading the previous tiles
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const int ep = (int)__reduce_max_sync(0xffffffffu, (unsigned)wmax[f][lane & (FX_NT / 32 - 1)]);
            if (ep == 0x7FF) poisoned[f] = true;
            if (ep > E[f]) {
                const int d = ep - E[f];
#pragma unroll
                for (int q = 0; q < FX_RY; ++q)
#pragma unroll
                    for (int k = 0; k < 5; ++k) acc[f][q][k] = d >= 63 ? 0 : (acc[f][q][k] >> d);
                E[f] = ep;
            }
#pragma unroll
            for (int r = 0; r < FX_SLOTS; ++r)
                if (sidx[r] >= 0) tile[f][sidx[r]] = to_fixed(v[f][r], E[f]);
        }
        __syncthreads();
        const int cz = (zin == 1) + (zin == n - 1);
        const int zo = zin - 2;
        const bool zstore = zo >= kz0 && zo < kz1;
        const size_t o0 = ((size_t)zo * np + ja) * np + i;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const long long* T = tile[f];
            auto at = [&](int yy, int xx) { return T[yy * FX_HX + xx]; };
            // column x: rows ry-2 .. ry+3; columns x-1, x+1: rows ry-1 .. ry+2;
            // columns x-2, x+2: rows ry, ry+1
            const long long cm2 = at(ry - 2, rx), cm1 = at(ry - 1, rx), c_0 = at(ry, rx),
                            c_1 = at(ry + 1, rx), c_2 = at(ry + 2, rx), c_3 = at(ry + 3, rx);
            const long long lm1 = at(ry - 1, rx - 1), l_0 = at(ry, rx - 1), l_1 = at(ry + 1, rx - 1),
                            l_2 = at(ry + 2, rx - 1);
            const long long rm1 = at(ry - 1, rx + 1), r_0 = at(ry, rx + 1), r_1 = at(ry + 1, rx + 1),
                            r_2 = at(ry + 2, rx + 1);
            const long long ll0 = at(ry, rx - 2), ll1 = at(ry + 1, rx - 2), rr0 = at(ry, rx + 2),
                            rr1 = at(ry + 1, rx + 2);
            {   // output row ja
                const long long n4 = l_0 + r_0 + cm1 + c_1;
                const long long f4 = ll0 + rr0 + cm2 + c_2;
                const long long d4 = lm1 + l_1 + rm1 + r_1;
                const long long p0 = (long long)(42 + sigma * (c0 + cz)) * c_0 - 12 * n4 + f4 + 2 * d4;
                const long long p1 = 2 * n4 - 12 * c_0;
                acc[f][0][0] += c_0;
                acc[f][0][1] += p1;
                acc[f][0][2] += p0;
                acc[f][0][3] += p1;
                acc[f][0][4] += c_0;
            }
            {   // output row ja + 1
                const long long n4 = l_1 + r_1 + c_0 + c_2;
                const long long f4 = ll1 + rr1 + cm1 + c_3;
                const long long d4 = l_0 + l_2 + r_0 + r_2;
                const long long p0 = (long long)(42 + sigma * (c1 + cz)) * c_1 - 12 * n4 + f4 + 2 * d4;
                const long long p1 = 2 * n4 - 12 * c_1;
                acc[f][1][0] += c_1;
                acc[f][1][1] += p1;
                acc[f][1][2] += p0;
                acc[f][1][3] += p1;
                acc[f][1][4] += c_1;
            }
            if (zstore) {
                if (act0) {
                    double val = fx_result(acc[f][0][0], E[f], poisoned[f]);
                    if (NF == 1 && b != nullptr) val = b[o0] - val;
                    fl.out[f][o0] = val;
                    if (kDot && f == 0) dot += __ldg(&fl.in[1][o0]) * val;
                }
                if (act1) {
                    double val = fx_result(acc[f][1][0], E[f], poisoned[f]);
                    if (NF == 1 && b != nullptr) val = b[o0 + np] - val;
                    fl.out[f][o0 + np] = val;
                    if (kDot && f == 0) dot += __ldg(&fl.in[1][o0 + np]) * val;
                }
            }
#pragma unroll
            for (int q = 0; q < FX_RY; ++q) {
                acc[f][q][0] = acc[f][q][1];
                acc[f][q][1] = acc[f][q][2];
                acc[f][q][2] = acc[f][q][3];
                acc[f][q][3] = acc[f][q][4];
                acc[f][q][4] = 0;
            }
        }
    }
    if (kDot) {
        __shared__ double sh[32];
        __shared__ bool am_last;
        double sdot = block_sum(dot, sh);
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
};

// Column tiles x z-slabs.  The slab count is chosen so that the CTAs fill
// whole waves of the GPU's resident slots (152 SMs x CTAs per SM) while each
// slab stays long enough that its 4 extra halo planes cost little.
StencilGrid stencil_grid(int n, int tx, int rows, int per_sm) {
    const int m = n - 1;  // interior extent
    StencilGrid g;
    const int gx = (m + tx - 1) / tx, gy = (m + rows - 1) / rows;
    const int tiles = gx * gy;
    const int slots = 152 * (per_sm > 0 ? per_sm : 1);
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

template <typename K>
int resident_per_sm(K kernel, int threads) {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        v = 1;
    }
    return v > 0 ? v : 1;
}

StencilGrid fx_grid(int n, int nf) {
    static int occ1 = 0, occ2 = 0;
    if (nf == 1) {
        if (!occ1) occ1 = resident_per_sm(stencil_fx_kernel<1, false>, FX_NT);
        StencilGrid g = stencil_grid(n, FX_TX, FX_OY, occ1);
        g.block = dim3(FX_TX, FX_TY, 1);
        return g;
    }
    if (!occ2) occ2 = resident_per_sm(stencil_fx_kernel<2, true>, FX_NT);
    StencilGrid g = stencil_grid(n, FX_TX, FX_OY, occ2);
    g.block = dim3(FX_TX, FX_TY, 1);
    return g;
}

StencilGrid f64_grid(int n) {
    static int occ = 0;
    if (!occ) occ = resident_per_sm(stencil_f64_kernel<false>, TX * TY);
    StencilGrid g = stencil_grid(n, TX, TY, occ);
    g.block = dim3(TX, TY, 1);
    return g;
}

}  // namespace

int stencil_cta_count(int n) {
    const StencilGrid g = fx_grid(n, 2);
    return (int)(g.grid.x * g.grid.y * g.grid.z);
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
        const StencilGrid g = fx_grid(n, 1);
        FxFields fl{{u, nullptr}, {y, nullptr}};
        stencil_fx_kernel<1, false><<<g.grid, g.block, 0, s>>>(fl, b, n, bc_kind == 1 ? 1 : -1, g.kz_per_cta,
                                                               skip, nullptr, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_bicg_stencil_pair(const double* p, double* q, const double* ps, double* qs, int n,
                                     int bc_kind, double* partials, BicgState* st, cudaStream_t s) {
    const StencilGrid g = fx_grid(n, 2);
    FxFields fl{{p, ps}, {q, qs}};
    stencil_fx_kernel<2, true><<<g.grid, g.block, 0, s>>>(fl, nullptr, n, bc_kind == 1 ? 1 : -1, g.kz_per_cta,
                                                          &st->done, partials, st);
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
