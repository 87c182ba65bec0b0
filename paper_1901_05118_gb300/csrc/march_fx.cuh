// The integer ("exact") evaluation of the 25-point operator of eq. (method1)
// with the reflections of eqs. (reflection2) / (reflection4): conversions
// between doubles and 64-bit fixed point, and the register-blocked z-march
// of one tile of output columns.  Shared by the operator kernels, the
// cooperative small-grid Bi-CG and the batch engine.
#pragma once

#include <cuda_runtime.h>

#include "excmg_internal.cuh"

namespace excmg {
namespace {

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
    // direction update fused into the march (kDir): the inputs in[] are the
    // previous directions p, p*, and each loaded value becomes
    // r + beta p (r* + beta p* for field 1); nodes the CTA owns are written
    // to pn[] (a second buffer: neighbours still read the old directions)
    const double* dr[2];
    double* pn[2];
    double beta;
};

// Rare cases (a non-finite input, or a scale outside the normal range of the
// fast conversion) leave the hot path through a call, so that the compiler
// does not evaluate them -- on GB300's slow FP64 pipe -- for every output.
__device__ __noinline__ double fx_result_slow(long long acc, int E, bool poisoned) {
    if (poisoned) return __longlong_as_double(0x7FF8000000000000ll);
    return ldexp((double)acc, E - 1075);
}

__device__ __forceinline__ double fx_result(long long acc, int E, bool poisoned) {
    if (!poisoned && E >= 53 && E <= 2037) return from_fixed(acc, E);
    return fx_result_slow(acc, E, poisoned);
}

// One CTA's z-march over the output columns of tile (bx, by) and the output
// planes [kz0, kz1).  Returns this thread's share of (field 1 in, field 0
// out) when kDot.  Called uniformly by all threads of the CTA.
template <int NF, bool kDot, bool kDir = false>
__device__ __forceinline__ double fx_march(const FxFields& fl, const double* __restrict__ b, int n, int sigma,
                                           int bx, int by, int kz0, int kz1) {
    __shared__ long long tile[NF][FX_HY * FX_HX];
    __shared__ int wmax[NF][FX_NT / 32];
    const int np = n + 1;
    const size_t plane = (size_t)np * np;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * FX_TX + tx;
    const int lane = tid & 31;
    const int i0 = 1 + bx * FX_TX, j0 = 1 + by * FX_OY;

    // halo-load slots of this thread: in-plane offset (-1: outside the
    // interior, reads as zero) and shared-memory index (-1: no slot)
    int soff[FX_SLOTS], sidx[FX_SLOTS];
    bool own[FX_SLOTS];   // the slot is one of this CTA's output columns
#pragma unroll
    for (int r = 0; r < FX_SLOTS; ++r) {
        const int e = tid + r * FX_NT;
        soff[r] = -1;
        sidx[r] = -1;
        own[r] = false;
        if (e < FX_HX * FX_HY) {
            const int ly = e / FX_HX, lx = e - ly * FX_HX;
            const int gi = i0 - 2 + lx, gj = j0 - 2 + ly;
            sidx[r] = e;
            if (gi >= 1 && gi <= n - 1 && gj >= 1 && gj <= n - 1) soff[r] = gj * np + gi;
            own[r] = soff[r] >= 0 && lx >= 2 && lx < 2 + FX_TX && ly >= 2 && ly < 2 + FX_OY;
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
    // NF = 2: while the two fields' planes have been equal bit for bit (with
    // r*_0 = r_0 in Bi-CG, always), field 1's accumulators would equal field
    // 0's; they are then not kept separately (exact integer sums, so no bit
    // of the result changes)
    bool shared1 = NF == 2;

    for (int zin = kz0 - 2; zin <= kz1 + 1; ++zin) {
        const bool zok = (zin >= 1) && (zin <= n - 1);
        const size_t zbase = zok ? (size_t)zin * plane : 0;
        double v[NF][FX_SLOTS];
        bool same = true;
        if (kDir) {
            // p = r + beta p, p* = r* + beta p* on every loaded node; where
            // r*, p* equal r, p bit for bit, p* takes p's bits
            const bool zown = zin >= kz0 && zin < kz1;
#pragma unroll
            for (int r = 0; r < FX_SLOTS; ++r) {
                double pv = 0.0, psv = 0.0;
                if (zok && soff[r] >= 0) {
                    const size_t o = zbase + soff[r];
                    const double rv = fl.dr[0][o];
                    const double po = fl.in[0][o];
                    pv = rv + fl.beta * po;
                    if (NF == 2) {
                        const double rsv = fl.dr[NF - 1][o];
                        const double pso = fl.in[NF - 1][o];
                        if (__double_as_longlong(rsv) == __double_as_longlong(rv) &&
                            __double_as_longlong(pso) == __double_as_longlong(po))
                            psv = pv;
                        else
                            psv = rsv + fl.beta * pso;
                    }
                    if (zown && own[r]) {
                        fl.pn[0][o] = pv;
                        if (NF == 2) fl.pn[NF - 1][o] = psv;
                    }
                }
                v[0][r] = pv;
                if (NF == 2) v[NF - 1][r] = psv;
            }
        } else {
#pragma unroll
            for (int f = 0; f < NF; ++f)
#pragma unroll
                for (int r = 0; r < FX_SLOTS; ++r)
                    v[f][r] = (zok && soff[r] >= 0) ? fl.in[f][zbase + soff[r]] : 0.0;
        }
        if (NF == 2) {
#pragma unroll
            for (int r = 0; r < FX_SLOTS; ++r)
                same = same && (__double_as_longlong(v[0][r]) == __double_as_longlong(v[NF - 1][r]));
        }
        // a warp whose two fields agree bit for bit has one exponent maximum
        const bool warp_same = NF == 2 && __all_sync(0xffffffffu, same);
        int emax0 = 0;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            int emax = 0;
            if (f > 0 && warp_same) {
                emax = emax0;
            } else {
#pragma unroll
                for (int r = 0; r < FX_SLOTS; ++r) emax = max(emax, exponent_of(v[f][r]));
                emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)emax);
            }
            if (f == 0) emax0 = emax;
            if (lane == 0) wmax[f][tid >> 5] = emax;
        }
        // also: every thread is done reading the previous tiles
        const bool plane_same = NF == 2 ? (__syncthreads_and(same) != 0) : (__syncthreads(), false);
        if (NF == 2 && shared1 && !plane_same) {
            // first plane on which the fields differ: from here on field 1
            // keeps accumulators of its own, starting from field 0's
#pragma unroll
            for (int q = 0; q < FX_RY; ++q)
#pragma unroll
                for (int k = 0; k < 5; ++k) acc[NF - 1][q][k] = acc[0][q][k];
            shared1 = false;
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            if (f > 0 && shared1) {   // the same plane: the same scale
                E[f] = E[0];
                poisoned[f] = poisoned[0];
                continue;
            }
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
        }
        // Twin fields: when this plane of field 1 equals field 0's bit for bit
        // and both are on the same scale, field 1's integer contributions are
        // field 0's, so they are computed once (the sums are exact, so this
        // changes no bit of the result).  With r*_0 = r_0 the Bi-CG shadow
        // vector p* always equals p.
        const bool twin = NF == 2 && plane_same && E[0] == E[NF - 1] && poisoned[0] == poisoned[NF - 1];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            if (f > 0 && twin) continue;
#pragma unroll
            for (int r = 0; r < FX_SLOTS; ++r)
                if (sidx[r] >= 0) tile[f][sidx[r]] = to_fixed(v[f][r], E[f]);
        }
        __syncthreads();
        const int cz = (zin == 1) + (zin == n - 1);
        const int zo = zin - 2;
        const bool zstore = zo >= kz0 && zo < kz1;
        const size_t o0 = ((size_t)zo * np + ja) * np + i;
        long long ca[FX_RY], p0a[FX_RY], p1a[FX_RY];   // field 0's contributions of this plane
        double val0[FX_RY] = {0.0, 0.0};
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            if (f > 0 && shared1) {
                // field 1 has been field 0 bit for bit on every plane so far:
                // its exact sums, hence its outputs, are field 0's
                if (zstore) {
#pragma unroll
                    for (int q = 0; q < FX_RY; ++q)
                        if (q == 0 ? act0 : act1) fl.out[f][o0 + (size_t)q * np] = val0[q];
                }
                continue;
            }
            long long cc[FX_RY], p0[FX_RY], p1[FX_RY];
            if (f > 0 && twin) {
#pragma unroll
                for (int q = 0; q < FX_RY; ++q) {
                    cc[q] = ca[q];
                    p0[q] = p0a[q];
                    p1[q] = p1a[q];
                }
            } else {
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
                    cc[0] = c_0;
                    p0[0] = (long long)(42 + sigma * (c0 + cz)) * c_0 - 12 * n4 + f4 + 2 * d4;
                    p1[0] = 2 * n4 - 12 * c_0;
                }
                {   // output row ja + 1
                    const long long n4 = l_1 + r_1 + c_0 + c_2;
                    const long long f4 = ll1 + rr1 + cm1 + c_3;
                    const long long d4 = l_0 + l_2 + r_0 + r_2;
                    cc[1] = c_1;
                    p0[1] = (long long)(42 + sigma * (c1 + cz)) * c_1 - 12 * n4 + f4 + 2 * d4;
                    p1[1] = 2 * n4 - 12 * c_1;
                }
                if (f == 0) {
#pragma unroll
                    for (int q = 0; q < FX_RY; ++q) {
                        ca[q] = cc[q];
                        p0a[q] = p0[q];
                        p1a[q] = p1[q];
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < FX_RY; ++q) {
                acc[f][q][0] += cc[q];
                acc[f][q][1] += p1[q];
                acc[f][q][2] += p0[q];
                acc[f][q][3] += p1[q];
                acc[f][q][4] += cc[q];
            }
            if (zstore) {
#pragma unroll
                for (int q = 0; q < FX_RY; ++q) {
                    if (!(q == 0 ? act0 : act1)) continue;
                    const size_t o = o0 + (size_t)q * np;
                    double val;
                    if (f > 0 && acc[f][q][0] == acc[0][q][0] && E[f] == E[0] && poisoned[f] == poisoned[0])
                        val = val0[q];          // same exact sum on the same scale
                    else
                        val = fx_result(acc[f][q][0], E[f], poisoned[f]);
                    if (f == 0) val0[q] = val;
                    if (NF == 1 && b != nullptr) val = b[o] - val;
                    fl.out[f][o] = val;
                    if (kDot && f == 0)
                        // sigma = (p*, A p) (with one field: (p, A p)); with
                        // kDir p*'s new value was written by this CTA two
                        // planes ago
                        dot += (kDir ? __ldcg(&fl.pn[NF - 1][o]) : __ldg(&fl.in[NF - 1][o])) * val;
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
    return dot;
}

}  // namespace
}  // namespace excmg
