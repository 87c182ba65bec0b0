// The operator launch of Bi-CG (Alg. 2): q = A p and q* = A^T p* of eq.
// (method1) with the reflections of eqs. (reflection2) / (reflection4), with
// sigma = (p*, q), in the integer arithmetic of march_fx.cuh (each input
// plane of a CTA on one power-of-two scale, taps summed exactly, one
// rounding per output).  Same results, bit for bit, as fx_march<2, true>:
// the same scale sequence, the same integer sums, the same per-thread order
// of the sigma terms.  What differs is how the work is fed:
//
//  * Loads are staged ahead by per-thread asynchronous copies (cp.async, 8
//    bytes each) of the thread's own halo slots into a ring of four shared
//    memory stages, three planes ahead of the plane being converted.  Each
//    thread reads back only the slots it copied itself, so completing a stage
//    needs no CTA barrier: cp.async.wait_group orders the thread's own copies.
//  * A thread's slots are its own two output columns (x = i, rows j, j+1)
//    plus at most one element of the 2-node ring around the CTA's 32 x 16
//    columns, so its centre values also feed sigma without another load.
//  * One CTA barrier per plane: the exponent maximum of plane t+1 is
//    published (per warp) before the barrier that also publishes the
//    fixed-point tile of plane t, so the scale of every plane is known one
//    plane ahead.  Tiles alternate between two buffers.
//  * The march runs on p alone and checks, slot by slot, that p* equals p
//    bit for bit (with r*_0 = r_0 it always does: A^T p* is then A p bit for
//    bit, and q* is written from q).  A CTA that meets a differing slot
//    returns `false` and the caller runs the general two-field march.
//  * Multiplications by the small weights are 64 x 32-bit products (two
//    integer multiply-adds) and sums of mirrored taps are shared between the
//    two output rows (the diagonal taps of a row are the horizontal axis
//    taps of the rows above and below).
#pragma once

#include <cuda_runtime.h>

#include "march_fx.cuh"

namespace excmg {
namespace {

constexpr int PP_TX = 32;                       // threads along x
constexpr int PP_TY = 8;                        // threads along y
constexpr int PP_OY = 2 * PP_TY;                // output rows per CTA (2 per thread)
constexpr int PP_HX = PP_TX + 4;                // halo width (36)
constexpr int PP_HY = PP_OY + 4;                // halo height (20)
constexpr int PP_HALO = PP_HX * PP_HY;          // 720 nodes per plane
constexpr int PP_NT = PP_TX * PP_TY;            // 256 threads
constexpr int PP_RING = PP_HALO - PP_TX * PP_OY;   // 208 ring nodes
constexpr int PP_STAGES = 4;                    // copy stages
constexpr int PP_AHEAD = PP_STAGES - 1;         // planes copied ahead of the one converted

static_assert(PP_TX == FX_TX && PP_OY == FX_OY, "same tiles as fx_march (same sigma partials)");

// copy stages: four (three planes ahead), three when four arrays are copied
// per slot (the fused direction update), so that two CTAs fit on an SM
__host__ __device__ constexpr int pp_stages(int nf) { return nf > 2 ? 3 : PP_STAGES; }

// dynamic shared memory: copy stages (NF arrays copied per slot) + two
// fixed-point tiles
template <int NF>
__host__ __device__ constexpr size_t pp_smem_bytes() {
    return (size_t)pp_stages(NF) * NF * PP_HALO * sizeof(double) + (size_t)2 * PP_HALO * sizeof(long long);
}

// Halo index (ly * PP_HX + lx) of slot s of thread tid: slots 0, 1 are the
// thread's output columns; slot 2 (threads below PP_RING) one ring node --
// the two rows above and below the CTA's columns, then the two columns left
// and right of them, four nodes per row.
__device__ __forceinline__ int pp_slot(int tid, int s) {
    const int tx = tid & (PP_TX - 1), ty = tid / PP_TX;
    if (s < 2) return (2 * ty + 2 + s) * PP_HX + tx + 2;
    if (tid < 4 * PP_HX) {
        const int row = tid / PP_HX, lx = tid - row * PP_HX;
        const int ly = row < 2 ? row : PP_HY - 4 + row;
        return ly * PP_HX + lx;
    }
    const int k = tid - 4 * PP_HX;
    const int c = k & 3;
    return (2 + (k >> 2)) * PP_HX + (c < 2 ? c : PP_HX - 4 + c);
}

// 32-bit shared-memory address of a generic pointer into shared memory
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ double lds_f64(unsigned a) {
    double v;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ long long lds_s64(unsigned a) {
    long long v;
    asm volatile("ld.shared.s64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
}
// ld.shared.s64 at a + OFF (OFF a non-negative constant folded into the
// instruction's immediate offset)
template <int OFF>
__device__ __forceinline__ long long lds_s64_at(unsigned a) {
    long long v;
    asm volatile("ld.shared.s64 %0, [%1+%2];" : "=l"(v) : "r"(a), "n"(OFF));
    return v;
}
__device__ __forceinline__ void sts_s64(unsigned a, long long v) {
    asm volatile("st.shared.s64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
__device__ __forceinline__ void cp_async8_u32(unsigned dst, const void* src, unsigned src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
// x >> k for 0 <= k, 0 once k >= 32 (PTX clamps the shift amount)
__device__ __forceinline__ unsigned shr_clamp(unsigned x, unsigned k) {
    unsigned r;
    asm("shr.b32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(k));
    return r;
}

// to_fixed (march_fx.cuh) with the biased exponent e of v already at hand
// and the 64-bit shift written as clamped 32-bit shifts: the same value,
// m >> (E - max(e, 1)) with the sign of v, 0 once the shift reaches 64.
__device__ __forceinline__ long long to_fixed_e(double v, unsigned e, int E) {
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    const unsigned mh = (hi & 0xFFFFFu) | (e != 0u ? 0x100000u : 0u);
    const unsigned d = (unsigned)(E - (int)max(e, 1u));
    const unsigned rlo = shr_clamp(__funnelshift_rc(lo, mh, d), (unsigned)max((int)d - 32, 0));
    const unsigned rhi = shr_clamp(mh, d);
    const unsigned sg = (unsigned)((int)hi >> 31);   // 0 or all ones
    const unsigned long long m = ((unsigned long long)(rhi ^ sg) << 32) | (rlo ^ sg);
    return (long long)(m - (unsigned long long)(long long)(int)sg);
}

// a * w for a 64-bit integer a and a small positive weight w (|a w| < 2^63):
// one 32 x 32 -> 64 product of the low word and one multiply-add of the high
// word, instead of a general 64-bit multiplication
__device__ __forceinline__ long long mul_w(long long a, unsigned w) {
    const unsigned long long lo = (unsigned long long)(unsigned)a * w;
    const unsigned hi = (unsigned)((unsigned long long)a >> 32) * w + (unsigned)(lo >> 32);
    return (long long)(((unsigned long long)hi << 32) | (unsigned)lo);
}

// Y * 2^(E - 1075) rounded to nearest even, by the hardware conversion of Y
// to double (the same rounding of Y to 53 bits as from_fixed) and an exact
// power-of-two scaling of the exponent field; valid for 53 <= E <= 2036.
__device__ __forceinline__ double fx_result_cvt(long long acc, int E, bool poisoned) {
    if (!poisoned && E >= 53 && E <= 2036) {
        const double d = (double)acc;
        const long long bits = __double_as_longlong(d) + ((long long)(E - 1075) << 52);
        return acc == 0 ? 0.0 : __longlong_as_double(bits);
    }
    return fx_result_slow(acc, E, poisoned);
}

// One CTA's march over output planes [kz0, kz1) of column tile (bx, by).
// Returns false (uniformly) if some slot of p* differs from p; otherwise
// writes q (and q* = q unless kElide) and adds this thread's share of
// sigma = (p*, q) to *dot.  kElide: p* is not read and q* not written (the
// shadow-elided mode; the same sums in the same order).  kCvt: round the
// outputs through the hardware integer-to-double conversion.  Shared memory
// is addressed through 32-bit shared-window addresses.
//
// kDir (the fused schedule): p and ps hold the previous directions p_{k-1},
// p*_{k-1}; every loaded node first becomes p_k = r_k + beta p_{k-1} (r, rs
// give r_k, r*_k; p*_k likewise, and the twin check asks r* = r and
// p*_{k-1} = p_{k-1}); the nodes the CTA owns are written to pn (and psn),
// which must not alias p, ps (neighbouring CTAs still read the old values).
struct PairDir {
    const double* r = nullptr;
    const double* rs = nullptr;
    double* pn = nullptr;
    double* psn = nullptr;
    double beta = 0.0;
};

template <bool kElide, bool kCvt, bool kDir = false>
__device__ __forceinline__ bool pp_march(const double* __restrict__ p, const double* __restrict__ ps,
                                         double* __restrict__ q, double* __restrict__ qs, int n, int sigma, int bx,
                                         int by, int kz0, int kz1, unsigned char* smem, double* dot,
                                         const PairDir& dir = PairDir{}) {
    // arrays copied per slot: p (or p_{k-1}) [, r] [, p* (or p*_{k-1}) [, r*]]
    constexpr int NF = (kElide ? 1 : 2) * (kDir ? 2 : 1);
    constexpr int kShadow = kDir ? 2 : 1;   // index of the first shadow array
    constexpr int S = pp_stages(NF);        // copy stages
    constexpr int AHEAD = S - 1;            // planes copied ahead of the one converted
    constexpr unsigned kField = PP_HALO * 8u;          // bytes of one field of a stage
    constexpr unsigned kStage = NF * kField;           // bytes of one stage
    constexpr unsigned kTile = PP_HALO * 8u;           // bytes of one fixed-point tile
    __shared__ int wmax[2][PP_NT / 32];
    const unsigned raw = smem_u32(smem);
    const unsigned tiles = raw + S * kStage;
    const int np = n + 1;
    const unsigned plane = (unsigned)np * (unsigned)np;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * PP_TX + tx;
    const int lane = tid & 31, warp = tid >> 5;
    const int i0 = 1 + bx * PP_TX, j0 = 1 + by * PP_OY;
    const bool ring = tid < PP_RING;

    // slots: byte offset in a stage / tile, in-plane node index, whether the
    // node is an unknown (else it reads as zero)
    unsigned so[3], sidx[3];
    bool sin[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const int e = (s < 2 || ring) ? pp_slot(tid, s) : 0;
        const int ly = e / PP_HX, lx = e - ly * PP_HX;
        const int gi = i0 - 2 + lx, gj = j0 - 2 + ly;
        so[s] = 8u * (unsigned)e;
        sin[s] = (s < 2 || ring) && gi >= 1 && gi <= n - 1 && gj >= 1 && gj <= n - 1;
        sidx[s] = sin[s] ? (unsigned)(gj * np + gi) : 0u;
    }
    const int i = i0 + tx, ja = j0 + 2 * ty;
    const bool act0 = (i <= n - 1) && (ja <= n - 1);
    const bool act1 = (i <= n - 1) && (ja + 1 <= n - 1);
    const int cx = (i == 1) + (i == n - 1);
    const int c0 = cx + (ja == 1) + (ja == n - 1);
    const int c1 = cx + (ja + 1 == 1) + (ja + 1 == n - 1);
    // byte offset in a tile of the top-left corner (row ry - 2, column
    // rx - 2) of this thread's 5 x 6 stencil window
    const unsigned tc = 8u * (unsigned)((2 * ty) * PP_HX + tx);
    const int T = kz1 - kz0 + 4;   // input planes kz0 - 2 .. kz1 + 1

    // copy plane t (all of this thread's slots) into its stage; nodes
    // outside the interior are zero-filled; always one commit group
    auto issue = [&](int t) {
        if (t < T) {
            const int zin = kz0 - 2 + t;
            const bool zok = zin >= 1 && zin <= n - 1;
            const unsigned zb = zok ? (unsigned)zin * plane : 0u;
            const unsigned st = raw + ((unsigned)t % (unsigned)S) * kStage;
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                if (s < 2 || ring) {
                    const bool ld = zok && sin[s];
                    const unsigned gidx = ld ? zb + sidx[s] : 0u;
                    const unsigned nb = ld ? 8u : 0u;
                    cp_async8_u32(st + so[s], p + gidx, nb);
                    if (kDir) cp_async8_u32(st + kField + so[s], dir.r + gidx, nb);
                    if (!kElide) cp_async8_u32(st + kShadow * kField + so[s], ps + gidx, nb);
                    if (!kElide && kDir) cp_async8_u32(st + (kShadow + 1) * kField + so[s], dir.rs + gidx, nb);
                }
            }
        }
        cp_async_commit();
    };
    // read back plane t's slots (its copies complete) and their exponents,
    // publish the warp's exponent maximum; false if p* differs from p
    auto scan = [&](int t, double (&v)[3], unsigned (&ev)[3]) -> bool {
        const unsigned st = raw + ((unsigned)t % (unsigned)S) * kStage;
        unsigned diff = 0u, emax = 0u;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            v[s] = 0.0;
            ev[s] = 0u;
            if (s < 2 || ring) {
                const double po = lds_f64(st + so[s]);
                if (!kElide) {
                    const double w = lds_f64(st + kShadow * kField + so[s]);
                    diff |= ((unsigned)__double2loint(po) ^ (unsigned)__double2loint(w)) |
                            ((unsigned)__double2hiint(po) ^ (unsigned)__double2hiint(w));
                }
                if (kDir) {
                    const double rv = lds_f64(st + kField + so[s]);
                    if (!kElide) {
                        const double w = lds_f64(st + (kShadow + 1) * kField + so[s]);
                        diff |= ((unsigned)__double2loint(rv) ^ (unsigned)__double2loint(w)) |
                                ((unsigned)__double2hiint(rv) ^ (unsigned)__double2hiint(w));
                    }
                    v[s] = rv + dir.beta * po;   // p_k = r_k + beta p_{k-1}
                } else {
                    v[s] = po;
                }
                ev[s] = ((unsigned)__double2hiint(v[s]) >> 20) & 0x7FFu;
                emax = max(emax, ev[s]);
            }
        }
        emax = __reduce_max_sync(0xffffffffu, emax);
        if (lane == 0) wmax[t & 1][warp] = (int)emax;
        return diff == 0u;
    };
    auto plane_max = [&](int t) { return (int)__reduce_max_sync(0xffffffffu, (unsigned)wmax[t & 1][lane & 7]); };

#pragma unroll
    for (int t = 0; t < AHEAD; ++t) issue(t);
    cp_async_wait<AHEAD - 1>();
    double cur[3];
    unsigned ecur[3];
    bool same = scan(0, cur, ecur);
    if (!__syncthreads_and(same)) {
        cp_async_wait_all();
        return false;
    }
    int E = max(1, plane_max(0));
    bool poisoned = E == 0x7FF;

    long long acc[2][5];
#pragma unroll
    for (int qq = 0; qq < 2; ++qq)
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[qq][k] = 0;
    double pc1[2] = {0.0, 0.0}, pc2[2] = {0.0, 0.0};   // centre p of the last two planes
    double d = 0.0;

    for (int t = 0; t < T; ++t) {
        issue(t + AHEAD);
        cp_async_wait<AHEAD - 1>();   // planes up to t + 1 have landed
        double nxt[3] = {0.0, 0.0, 0.0};
        unsigned enx[3] = {0u, 0u, 0u};
        same = t + 1 < T ? scan(t + 1, nxt, enx) : true;
        // plane t on scale E into its tile
        const unsigned tl = tiles + (unsigned)(t & 1) * kTile;
#pragma unroll
        for (int s = 0; s < 3; ++s)
            if (s < 2 || ring) sts_s64(tl + so[s], to_fixed_e(cur[s], ecur[s], E));
        if (kDir) {   // the new directions of the nodes this CTA owns
            const int zt = kz0 - 2 + t;
            if (zt >= kz0 && zt < kz1) {
                const unsigned zb = (unsigned)zt * plane;
#pragma unroll
                for (int s = 0; s < 2; ++s)
                    if (s == 0 ? act0 : act1) {
                        dir.pn[zb + sidx[s]] = cur[s];
                        if (!kElide) dir.psn[zb + sidx[s]] = cur[s];
                    }
            }
        }
        // every tile of plane t written, every exponent of plane t + 1
        // published, every read of the tile of plane t - 2 done
        if (!__syncthreads_and(same)) {
            cp_async_wait_all();
            return false;
        }
        const int ep = t + 1 < T ? plane_max(t + 1) : 0;

        const int zin = kz0 - 2 + t;
        const int cz = (zin == 1) + (zin == n - 1);
        const unsigned b0 = tl + tc;
#define PP_AT(dy, dx) lds_s64_at<8 * (((dy) + 2) * PP_HX + (dx) + 2)>(b0)
        const long long cm2 = PP_AT(-2, 0), cm1 = PP_AT(-1, 0), cc0 = PP_AT(0, 0), cc1 = PP_AT(1, 0),
                        cc2 = PP_AT(2, 0), cc3 = PP_AT(3, 0);
        // x-neighbour sums at distance 1 (rows -1 .. 2) and 2 (rows 0, 1)
        const long long h1m = PP_AT(-1, -1) + PP_AT(-1, 1);
        const long long h10 = PP_AT(0, -1) + PP_AT(0, 1);
        const long long h11 = PP_AT(1, -1) + PP_AT(1, 1);
        const long long h12 = PP_AT(2, -1) + PP_AT(2, 1);
        const long long h20 = PP_AT(0, -2) + PP_AT(0, 2);
        const long long h21 = PP_AT(1, -2) + PP_AT(1, 2);
#undef PP_AT
        long long P0[2], P1[2], C[2];
        {   // output row ja: same plane (42 + sigma c) u - 12 (4 axis) + (4 at 2) + 2 (4 diagonals);
            // planes +-1: 2 (4 axis) - 12 u; planes +-2: u
            const long long n4 = h10 + cm1 + cc1;
            const long long f4 = h20 + cm2 + cc2;
            const long long d4 = h1m + h11;
            P0[0] = mul_w(cc0, (unsigned)(42 + sigma * (c0 + cz))) - mul_w(n4, 12u) + f4 + d4 + d4;
            P1[0] = n4 + n4 - mul_w(cc0, 12u);
            C[0] = cc0;
        }
        {   // output row ja + 1
            const long long n4 = h11 + cc0 + cc2;
            const long long f4 = h21 + cm1 + cc3;
            const long long d4 = h10 + h12;
            P0[1] = mul_w(cc1, (unsigned)(42 + sigma * (c1 + cz))) - mul_w(n4, 12u) + f4 + d4 + d4;
            P1[1] = n4 + n4 - mul_w(cc1, 12u);
            C[1] = cc1;
        }
        const int zo = zin - 2;
        const bool zstore = zo >= kz0 && zo < kz1;
        const unsigned orow = ((unsigned)zo * (unsigned)np + (unsigned)ja) * (unsigned)np + (unsigned)i;
#pragma unroll
        for (int qq = 0; qq < 2; ++qq) {
            acc[qq][0] += C[qq];
            acc[qq][1] += P1[qq];
            acc[qq][2] += P0[qq];
            acc[qq][3] += P1[qq];
            acc[qq][4] = C[qq];
            if (zstore && (qq == 0 ? act0 : act1)) {
                const unsigned o = orow + (unsigned)qq * (unsigned)np;
                const double val = kCvt ? fx_result_cvt(acc[qq][0], E, poisoned) : fx_result(acc[qq][0], E, poisoned);
                q[o] = val;
                if (!kElide) qs[o] = val;
                // sigma = (p*, A p): p* = p here, the centre value of plane zo
                d += pc2[qq] * val;
            }
            acc[qq][0] = acc[qq][1];
            acc[qq][1] = acc[qq][2];
            acc[qq][2] = acc[qq][3];
            acc[qq][3] = acc[qq][4];
            pc2[qq] = pc1[qq];
            pc1[qq] = cur[qq];
        }
        // scale of plane t + 1: a larger exponent shifts the accumulators
        if (ep == 0x7FF) poisoned = true;
        if (ep > E) {
            const int dd = ep - E;
#pragma unroll
            for (int qq = 0; qq < 2; ++qq)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[qq][k] = dd >= 63 ? 0 : (acc[qq][k] >> dd);
            E = ep;
        }
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            cur[s] = nxt[s];
            ecur[s] = enx[s];
        }
    }
    cp_async_wait_all();
    *dot = d;
    return true;
}

}  // namespace
}  // namespace excmg
