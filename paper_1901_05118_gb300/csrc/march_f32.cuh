// FP32 z-march of the 25-point operator (eq. (method1) + reflections) over
// one tile of output columns, shared by the FP32 correction solver and the
// batched engine.  A CTA of S_TX x S_TY threads owns S_TX x (S_TY * S_RY)
// columns (two outputs per thread in y) and the output planes [kz0, kz1).
// NF = 2 with kDot applies A to both fields and returns this thread's share
// of (field 1 in, field 0 out); A^T is applied with the same code because
// A_h is symmetric.  Called uniformly by every thread of the CTA.
#pragma once

#include <cuda_runtime.h>

namespace excmg {

constexpr int S_TX = 32;
constexpr int S_TY = 8;
constexpr int S_RY = 2;
constexpr int S_OY = S_TY * S_RY;
constexpr int S_HX = S_TX + 4;
constexpr int S_HY = S_OY + 4;
constexpr int S_NT = S_TX * S_TY;
constexpr int S_SLOTS = (S_HX * S_HY + S_NT - 1) / S_NT;

template <int NF, bool kDot>
__device__ __forceinline__ float f32_march(const float* __restrict__ in0, const float* __restrict__ in1,
                                           float* __restrict__ out0, float* __restrict__ out1, int n, float sigma,
                                           int bx, int by, int kz0, int kz1) {
    __shared__ float tile[NF][S_HY * S_HX];
    const int np = n + 1;
    const size_t plane = (size_t)np * np;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * S_TX + tx;
    const int i0 = 1 + bx * S_TX, j0 = 1 + by * S_OY;
    const float* in[2] = {in0, in1};
    float* out[2] = {out0, out1};
    int soff[S_SLOTS], sidx[S_SLOTS];
#pragma unroll
    for (int r = 0; r < S_SLOTS; ++r) {
        const int e = tid + r * S_NT;
        soff[r] = -1;
        sidx[r] = -1;
        if (e < S_HX * S_HY) {
            const int ly = e / S_HX, lx = e - ly * S_HX;
            const int gi = i0 - 2 + lx, gj = j0 - 2 + ly;
            sidx[r] = e;
            if (gi >= 1 && gi <= n - 1 && gj >= 1 && gj <= n - 1) soff[r] = gj * np + gi;
        }
    }
    const int i = i0 + tx, ja = j0 + ty * S_RY;
    const bool act0 = (i <= n - 1) && (ja <= n - 1);
    const bool act1 = (i <= n - 1) && (ja + 1 <= n - 1);
    const int cx = (i == 1) + (i == n - 1);
    const int c0 = cx + (ja == 1) + (ja == n - 1);
    const int c1 = cx + (ja + 1 == 1) + (ja + 1 == n - 1);
    const int ry = ty * S_RY + 2, rx = tx + 2;

    float acc[NF][S_RY][5];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int q = 0; q < S_RY; ++q)
#pragma unroll
            for (int k = 0; k < 5; ++k) acc[f][q][k] = 0.f;
    float dot = 0.f;

    for (int zin = kz0 - 2; zin <= kz1 + 1; ++zin) {
        const bool zok = (zin >= 1) && (zin <= n - 1);
        const size_t zbase = zok ? (size_t)zin * plane : 0;
        float v[NF][S_SLOTS];
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int r = 0; r < S_SLOTS; ++r) v[f][r] = (zok && soff[r] >= 0) ? in[f][zbase + soff[r]] : 0.f;
        __syncthreads();   // every thread is done reading the previous tiles
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int r = 0; r < S_SLOTS; ++r)
                if (sidx[r] >= 0) tile[f][sidx[r]] = v[f][r];
        __syncthreads();
        const int cz = (zin == 1) + (zin == n - 1);
        const int zo = zin - 2;
        const bool zstore = zo >= kz0 && zo < kz1;
        const size_t o0 = ((size_t)zo * np + ja) * np + i;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const float* T = tile[f];
            auto at = [&](int yy, int xx) { return T[yy * S_HX + xx]; };
            const float cm2 = at(ry - 2, rx), cm1 = at(ry - 1, rx), c_0 = at(ry, rx), c_1 = at(ry + 1, rx),
                        c_2 = at(ry + 2, rx), c_3 = at(ry + 3, rx);
            const float lm1 = at(ry - 1, rx - 1), l_0 = at(ry, rx - 1), l_1 = at(ry + 1, rx - 1),
                        l_2 = at(ry + 2, rx - 1);
            const float rm1 = at(ry - 1, rx + 1), r_0 = at(ry, rx + 1), r_1 = at(ry + 1, rx + 1),
                        r_2 = at(ry + 2, rx + 1);
            const float ll0 = at(ry, rx - 2), ll1 = at(ry + 1, rx - 2), rr0 = at(ry, rx + 2), rr1 = at(ry + 1, rx + 2);
            {
                const float n4 = (l_0 + r_0) + (cm1 + c_1);
                const float f4 = (ll0 + rr0) + (cm2 + c_2);
                const float d4 = (lm1 + l_1) + (rm1 + r_1);
                const float p0 = (42.f + sigma * (float)(c0 + cz)) * c_0 - 12.f * n4 + f4 + 2.f * d4;
                const float p1 = 2.f * n4 - 12.f * c_0;
                acc[f][0][0] += c_0;
                acc[f][0][1] += p1;
                acc[f][0][2] += p0;
                acc[f][0][3] += p1;
                acc[f][0][4] += c_0;
            }
            {
                const float n4 = (l_1 + r_1) + (c_0 + c_2);
                const float f4 = (ll1 + rr1) + (cm1 + c_3);
                const float d4 = (l_0 + l_2) + (r_0 + r_2);
                const float p0 = (42.f + sigma * (float)(c1 + cz)) * c_1 - 12.f * n4 + f4 + 2.f * d4;
                const float p1 = 2.f * n4 - 12.f * c_1;
                acc[f][1][0] += c_1;
                acc[f][1][1] += p1;
                acc[f][1][2] += p0;
                acc[f][1][3] += p1;
                acc[f][1][4] += c_1;
            }
            if (zstore) {
                if (act0) {
                    out[f][o0] = acc[f][0][0];
                    if (kDot && f == 0) dot += __ldg(&in[1][o0]) * acc[f][0][0];
                }
                if (act1) {
                    out[f][o0 + np] = acc[f][1][0];
                    if (kDot && f == 0) dot += __ldg(&in[1][o0 + np]) * acc[f][1][0];
                }
            }
#pragma unroll
            for (int q = 0; q < S_RY; ++q) {
                acc[f][q][0] = acc[f][q][1];
                acc[f][q][1] = acc[f][q][2];
                acc[f][q][2] = acc[f][q][3];
                acc[f][q][3] = acc[f][q][4];
                acc[f][q][4] = 0.f;
            }
        }
    }
    return dot;
}

}  // namespace excmg
