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

template <bool kTranspose>
__global__ void __launch_bounds__(TX * TY)
stencil_fx_kernel(const double* __restrict__ u, double* __restrict__ y, const double* __restrict__ b,
                  int n, int sigma, int kz_per_cta, const int* __restrict__ skip) {
    if (skip != nullptr && *skip) return;
    __shared__ long long tile[HY][HX];
    __shared__ int wmax[TX * TY / 32];
    constexpr int kPerThread = (HX * HY + TX * TY - 1) / (TX * TY);
    const int np = n + 1;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int i0 = 1 + blockIdx.x * TX, j0 = 1 + blockIdx.y * TY;
    const int kz0 = 1 + blockIdx.z * kz_per_cta;
    const int kz1 = min(kz0 + kz_per_cta, n);
    const int i = i0 + tx, j = j0 + ty;
    const bool active = (i <= n - 1) && (j <= n - 1);
    const int cxy = (i == 1) + (i == n - 1) + (j == 1) + (j == n - 1);
    const int sg = kTranspose ? -1 : 1;

    long long acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0, acc4 = 0;
    int E = 1;            // running scale exponent (1: nothing non-zero met yet)
    bool poisoned = false;
    for (int zin = kz0 - 2; zin <= kz1 + 1; ++zin) {
        const bool zok = (zin >= 1) && (zin <= n - 1);
        double v[kPerThread];
        int emax = 0;
#pragma unroll
        for (int r = 0; r < kPerThread; ++r) {
            const int e = tid + r * TX * TY;
            v[r] = 0.0;
            if (e < HX * HY) {
                const int ly = e / HX, lx = e - ly * HX;
                const int gi = i0 - 2 + lx, gj = j0 - 2 + ly;
                if (zok && gi >= 1 && gi <= n - 1 && gj >= 1 && gj <= n - 1)
                    v[r] = u[((size_t)zin * np + gj) * np + gi];
            }
            emax = max(emax, exponent_of(v[r]));
        }
        emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)emax);
        if ((tid & 31) == 0) wmax[tid >> 5] = emax;
        __syncthreads();   // also: every thread is done reading the previous tile
        int ep = wmax[0];
#pragma unroll
        for (int w = 1; w < TX * TY / 32; ++w) ep = max(ep, wmax[w]);
        if (ep == 0x7FF) poisoned = true;
        if (ep > E) {
            const int d = ep - E;
            if (d >= 63) {
                acc0 = acc1 = acc2 = acc3 = acc4 = 0;
            } else {
                acc0 >>= d; acc1 >>= d; acc2 >>= d; acc3 >>= d; acc4 >>= d;
            }
            E = ep;
        }
#pragma unroll
        for (int r = 0; r < kPerThread; ++r) {
            const int e = tid + r * TX * TY;
            if (e < HX * HY) {
                const int ly = e / HX, lx = e - ly * HX;
                tile[ly][lx] = to_fixed(v[r], E);
            }
        }
        __syncthreads();
        const int cy = ty + 2, cx = tx + 2;
        const long long a = tile[cy][cx];
        const long long n4 = tile[cy][cx - sg] + tile[cy][cx + sg] + tile[cy - sg][cx] + tile[cy + sg][cx];
        const long long f4 = tile[cy][cx - 2 * sg] + tile[cy][cx + 2 * sg] + tile[cy - 2 * sg][cx] +
                             tile[cy + 2 * sg][cx];
        const long long d4 = tile[cy - sg][cx - sg] + tile[cy - sg][cx + sg] + tile[cy + sg][cx - sg] +
                             tile[cy + sg][cx + sg];
        const int cz = (zin == 1) + (zin == n - 1);
        const long long centre = 42 + sigma * (cxy + cz);
        const long long p0 = centre * a - 12 * n4 + f4 + 2 * d4;
        const long long p1 = 2 * n4 - 12 * a;
        acc0 += a;
        acc1 += p1;
        acc2 += p0;
        acc3 += p1;
        acc4 += a;
        const int zo = zin - 2;
        if (active && zo >= kz0 && zo < kz1) {
            const size_t o = ((size_t)zo * np + j) * np + i;
            double val;
            if (poisoned)
                val = __longlong_as_double(0x7FF8000000000000ll);
            else if (E >= 53 && E <= 2037)
                val = from_fixed(acc0, E);
            else
                val = ldexp((double)acc0, E - 1075);
            y[o] = b ? (b[o] - val) : val;
        }
        acc0 = acc1;
        acc1 = acc2;
        acc2 = acc3;
        acc3 = acc4;
        acc4 = 0;
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

cudaError_t launch_stencil(const double* u, double* y, const double* b, int n, int bc_kind,
                           bool transpose, const int* skip, cudaStream_t s, int variant) {
    const int m = n - 1;  // interior extent
    dim3 block(TX, TY, 1);
    const int gx = (m + TX - 1) / TX, gy = (m + TY - 1) / TY;
    const int tiles = gx * gy;
    // enough CTAs to fill the GPU: split z into slabs when there are few columns
    const int target = 152 * 6;
    int slabs = (target + tiles - 1) / tiles;
    const int max_slabs = (m + 3) / 4;
    if (slabs > max_slabs) slabs = max_slabs;
    if (slabs < 1) slabs = 1;
    const int kz_per_cta = (m + slabs - 1) / slabs;
    slabs = (m + kz_per_cta - 1) / kz_per_cta;
    dim3 grid(gx, gy, slabs);
    if (variant == kStencilFp64) {
        const double sigma = bc_kind == 1 ? 1.0 : -1.0;
        if (transpose)
            stencil_f64_kernel<true><<<grid, block, 0, s>>>(u, y, b, n, sigma, kz_per_cta, skip);
        else
            stencil_f64_kernel<false><<<grid, block, 0, s>>>(u, y, b, n, sigma, kz_per_cta, skip);
    } else {
        const int sigma = bc_kind == 1 ? 1 : -1;
        if (transpose)
            stencil_fx_kernel<true><<<grid, block, 0, s>>>(u, y, b, n, sigma, kz_per_cta, skip);
        else
            stencil_fx_kernel<false><<<grid, block, 0, s>>>(u, y, b, n, sigma, kz_per_cta, skip);
    }
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
