// Right-hand side f_h of eq. (sec) and the boundary values of a level.
//
// Every interior node's row of eq. (method1) is h^4 f; the taps that land on
// boundary nodes carry known values g1 and move to the right-hand side, and
// the +-2 axis taps of nodes one step from a face reach a fictitious node
// whose value eq. (reflection2) / (reflection4) splits into a mirror unknown
// (folded into the operator's diagonal) and known data:
//   first kind:   u_ghost = u_mirror + 2h g2          (g2 = outward du/dn)
//   second kind:  u_ghost = -u_mirror + 2 g1 + h^2 g2  (g2 = d2u/dn2)
// The level's arrays are taken at every stride-th node of the given (finer)
// arrays, as the grids of Alg. 1 are nested.
#include "excmg_internal.cuh"

namespace excmg {
namespace {

struct Src {
    const double* g1;
    const double* g2;
    int np_src;   // n_src + 1
    int stride;
    __device__ __forceinline__ double node(int i, int j, int k) const {
        return g1[((size_t)(k * stride) * np_src + (size_t)(j * stride)) * np_src + (size_t)(i * stride)];
    }
    // face value at the boundary node (i,j,k) of face `face`
    __device__ __forceinline__ double face(int face, int i, int j, int k) const {
        const int axis = face >> 1;
        int a, b;
        if (axis == 0) { a = j; b = k; }
        else if (axis == 1) { a = i; b = k; }
        else { a = i; b = j; }
        return g2[(size_t)face * np_src * np_src + (size_t)(b * stride) * np_src + (size_t)(a * stride)];
    }
};

__device__ __forceinline__ bool on_boundary(int v, int n) { return v == 0 || v == n; }

__global__ void assemble_rhs_kernel(double* __restrict__ fh, int n, int bc_kind,
                                    const double* __restrict__ f, Src src) {
    const int np = n + 1;
    const size_t total = (size_t)np * np * np;
    const double h = 1.0 / (double)n;
    const double h4 = h * h * h * h;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % np);
        const int j = (int)((t / np) % np);
        const int k = (int)(t / ((size_t)np * np));
        if (i < 1 || i > n - 1 || j < 1 || j > n - 1 || k < 1 || k > n - 1) {
            fh[t] = 0.0;
            continue;
        }
        double rhs = h4 * f[((size_t)(k * src.stride) * src.np_src + (size_t)(j * src.stride)) * src.np_src +
                            (size_t)(i * src.stride)];
        if (i >= 3 && i <= n - 3 && j >= 3 && j <= n - 3 && k >= 3 && k <= n - 3) {
            fh[t] = rhs;
            continue;
        }
        const int p[3] = {i, j, k};
        double moved = 0.0;
        // axis taps: +-1 (weight -12) and +-2 (weight +1)
        for (int ax = 0; ax < 3; ++ax) {
            for (int s = -1; s <= 1; s += 2) {
                int q[3] = {p[0], p[1], p[2]};
                q[ax] = p[ax] + s;
                if (on_boundary(q[ax], n)) moved += -12.0 * src.node(q[0], q[1], q[2]);
                q[ax] = p[ax] + 2 * s;
                if (on_boundary(q[ax], n)) {
                    moved += src.node(q[0], q[1], q[2]);
                } else if (q[ax] < 0 || q[ax] > n) {
                    int bnode[3] = {p[0], p[1], p[2]};
                    bnode[ax] = s < 0 ? 0 : n;
                    const int face = 2 * ax + (s < 0 ? 0 : 1);
                    const double g2v = src.face(face, bnode[0], bnode[1], bnode[2]);
                    if (bc_kind == 1)
                        moved += 2.0 * h * g2v;
                    else
                        moved += 2.0 * src.node(bnode[0], bnode[1], bnode[2]) + h * h * g2v;
                }
            }
        }
        // in-plane diagonal taps (weight +2)
        for (int a = 0; a < 3; ++a)
            for (int b = a + 1; b < 3; ++b)
                for (int sa = -1; sa <= 1; sa += 2)
                    for (int sb = -1; sb <= 1; sb += 2) {
                        int q[3] = {p[0], p[1], p[2]};
                        q[a] += sa;
                        q[b] += sb;
                        if (on_boundary(q[0], n) || on_boundary(q[1], n) || on_boundary(q[2], n))
                            moved += 2.0 * src.node(q[0], q[1], q[2]);
                    }
        fh[t] = rhs - moved;
    }
}

__global__ void set_boundary_kernel(double* __restrict__ u, int n, Src src) {
    const int np = n + 1;
    const size_t per_face = (size_t)np * np;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < 6 * per_face;
         t += (size_t)gridDim.x * blockDim.x) {
        const int face = (int)(t / per_face);
        const size_t r = t - face * per_face;
        const int a = (int)(r % np), b = (int)(r / np);
        const int fixed = (face & 1) ? n : 0;
        int i, j, k;
        if (face < 2) { i = fixed; j = a; k = b; }
        else if (face < 4) { i = a; j = fixed; k = b; }
        else { i = a; j = b; k = fixed; }
        u[((size_t)k * np + j) * np + i] = src.node(i, j, k);
    }
}

int grid_for(size_t work) {
    size_t b = (work + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

cudaError_t launch_assemble_rhs(double* fh, int n, int bc_kind, const double* f, const double* g1,
                                const double* g2, int stride, cudaStream_t s) {
    Src src{g1, g2, n * stride + 1, stride};
    assemble_rhs_kernel<<<grid_for(node_count(n)), 256, 0, s>>>(fh, n, bc_kind, f, src);
    return cudaGetLastError();
}

cudaError_t launch_set_boundary(double* u, int n, const double* g1, int stride, cudaStream_t s) {
    Src src{g1, nullptr, n * stride + 1, stride};
    set_boundary_kernel<<<grid_for(face_count(n)), 256, 0, s>>>(u, n, src);
    return cudaGetLastError();
}

}  // namespace excmg
