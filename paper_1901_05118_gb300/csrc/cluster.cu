// Bi-CG iterations (Alg. 2, M = I) of the smallest Bi-CG grids -- N <= 32,
// at most 31^3 = 29 791 unknowns -- inside one thread-block cluster of 16
// CTAs, one per SM, with every work vector held in the CTAs' shared memory.
//
// CTA `rank` of the cluster owns the interior planes k = 1 + rank P ..
// rank P + P (P = ceil((N-1) / 16) <= 2) of x, r, r*, p, p*, q, q*.  The
// operator reads the taps of planes owned by other CTAs directly from their
// shared memory (distributed shared memory, `ld.shared::cluster`), the
// per-CTA partial sums of the inner products are read the same way, and the
// phases of an iteration are separated by hardware cluster barriers instead
// of the grid barriers of the cooperative kernel: no vector leaves the SMs
// between the load at the start of a launch and the write-back at its end.
//
// The operator is the per-node integer evaluation of eq. (method1) (each
// node's 25 taps on the scale of their largest exponent, summed exactly,
// rounded once), so A u and A^T u are the same bits.  When r* = r and p* = p
// on entry (Alg. 2 with r*_0 = r_0, as the solver runs it), the shadow
// sequence equals the primal one bit for bit and is computed once; a
// caller-chosen r*_0 runs the full two-sequence iteration.  Every CTA forms
// the cluster-wide sums in the same order, so all take the same alpha, beta
// and stopping decision.
#include <cuda_runtime.h>

#include <mutex>
#include <utility>
#include <vector>

#include "excmg_internal.cuh"
#include "march_fx.cuh"
#include "reduce.cuh"

namespace excmg {
namespace {

constexpr int kCC = 16;        // CTAs per cluster
constexpr int kCT = 512;      // threads per CTA
constexpr int kCMaxM = 31;     // largest N - 1
constexpr int kCVec = 7;       // x, r, r*, p, p*, q, q*
constexpr int kCMaxPlanes = (kCMaxM + kCC - 1) / kCC;   // planes per CTA
enum { VX = 0, VR, VRS, VP, VPS, VQ, VQS };

__device__ __forceinline__ unsigned cl_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ unsigned cl_map(unsigned addr, unsigned rank) {
    unsigned d;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(addr), "r"(rank));
    return d;
}

// (volatile: never merged with or moved across another load of the same
// address; the cluster barriers order it against the writes)
__device__ __forceinline__ double cl_ld(unsigned addr) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr));
    return v;
}

// all threads of all CTAs of the cluster; orders their shared-memory writes
// before the reads that follow
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

struct ClusterGeom {
    int m, P;          // interior points per axis, planes per CTA
    unsigned base;     // shared-memory address of the vectors
    // shared-memory offset (bytes) of vector v, local plane pl, node (i, j)
    __device__ __forceinline__ unsigned off(int v, int pl, int i, int j) const {
        return 8u * (unsigned)(((v * P + pl) * m + (j - 1)) * m + (i - 1));
    }
};

// Cluster addresses of node (1, 1) of planes k0 - 2 .. k0 + P + 1 of vector
// v (0 outside the interior), the planes a CTA owning k0 .. k0 + P - 1 reads.
__device__ __forceinline__ unsigned cl_plane_base(const ClusterGeom& g, int v, int kk) {
    if (kk < 1 || kk > g.m) return 0u;
    const int owner = (kk - 1) / g.P, pl = (kk - 1) - owner * g.P;
    return cl_map(g.base + g.off(v, pl, 1, 1), (unsigned)owner);
}

// The CTA's operator tile: planes k0 - 2 .. k0 + P + 1 of a vector (pbase:
// their cluster addresses, 0 outside the interior) as 64-bit integers on one
// power-of-two scale -- the largest exponent among them -- with a two-node
// zero border in x and y.  Returns the scale exponent (0x7FF: a value is
// not finite).  Border entries are zeroed by the caller once per launch.
__device__ __forceinline__ int cl_fill_tile(const unsigned* pbase, int P, int m, long long* tile, int* wred) {
    const int mm = m * m, tot = (P + 4) * mm, tid = threadIdx.x, tw = m + 4;
    int e = 0;
    for (int t = tid; t < tot; t += kCT) {
        const int d = t / mm, rem = t - d * mm;
        const unsigned b = pbase[d];
        e = max(e, b ? exponent_of(cl_ld(b + 8u * (unsigned)rem)) : 0);
    }
    e = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
    if ((tid & 31) == 0) wred[tid >> 5] = e;
    __syncthreads();
    const int E = max(1, (int)__reduce_max_sync(0xffffffffu, (unsigned)wred[tid & (kCT / 32 - 1)]));
    for (int t = tid; t < tot; t += kCT) {
        const int d = t / mm, rem = t - d * mm;
        const int jj = rem / m, ii = rem - jj * m;
        const unsigned b = pbase[d];
        tile[(d * tw + jj + 2) * tw + ii + 2] = b ? to_fixed(cl_ld(b + 8u * (unsigned)rem), E) : 0ll;
    }
    __syncthreads();
    return E;
}

// y at own node (i, j) of local plane pl = A u from the CTA's tile of u on
// scale E: the 25 taps of eq. (method1) summed exactly, rounded once.
__device__ __forceinline__ double cl_apply(const long long* tile, int m, int E, int sigma, int pl, int i, int j,
                                           int k) {
    const int tw = m + 4;
    auto at = [&](int d, int a, int b) { return tile[((pl + 2 + d) * tw + b + 1) * tw + a + 1]; };
    const long long c0 = at(0, i, j);
    const long long s_ax = at(0, i - 1, j) + at(0, i + 1, j) + at(0, i, j - 1) + at(0, i, j + 1) + at(-1, i, j) +
                           at(1, i, j);
    const long long s_far = at(0, i - 2, j) + at(0, i + 2, j) + at(0, i, j - 2) + at(0, i, j + 2) + at(-2, i, j) +
                            at(2, i, j);
    const long long s_dg = at(0, i - 1, j - 1) + at(0, i - 1, j + 1) + at(0, i + 1, j - 1) + at(0, i + 1, j + 1) +
                           at(-1, i - 1, j) + at(-1, i + 1, j) + at(-1, i, j - 1) + at(-1, i, j + 1) +
                           at(1, i - 1, j) + at(1, i + 1, j) + at(1, i, j - 1) + at(1, i, j + 1);
    const int c = (i == 1) + (i == m) + (j == 1) + (j == m) + (k == 1) + (k == m);
    const long long acc = (long long)(42 + sigma * c) * c0 - 12 * s_ax + s_far + 2 * s_dg;
    return fx_result(acc, E, E == 0x7FF);
}

// The cluster-wide sums of cnt (<= 4) per-thread values: each CTA's total
// (fixed tree) goes to its slot set `set`, a cluster barrier, then every CTA
// adds the 16 totals with the same shuffle tree and broadcasts them.
__device__ __forceinline__ void cl_reduce(double (&v)[4], int cnt, int set, double* red, double* sh, double* bc) {
    const int tid = threadIdx.x, lane = tid & 31;
    for (int c = 0; c < cnt; ++c) {
        const double s = block_sum(v[c], sh);
        if (tid == 0) red[set * 4 + c] = s;
    }
    cl_sync();
    if (tid < 32) {
        const unsigned a0 = (unsigned)__cvta_generic_to_shared(red + set * 4);
        for (int c = 0; c < cnt; ++c) {
            double t = lane < kCC ? cl_ld(cl_map(a0 + 8u * (unsigned)c, (unsigned)lane)) : 0.0;
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) bc[c] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (c < cnt) v[c] = bc[c];
    __syncthreads();
}

__global__ void __launch_bounds__(kCT, 1)
bicg_cluster_kernel(double* __restrict__ x, double* __restrict__ r, double* __restrict__ rs, double* __restrict__ p,
                    double* __restrict__ ps, int n, int sigma, int iters, BicgState* st) {
    extern __shared__ __align__(16) double csm[];
    __shared__ double sh[32];
    __shared__ double bc[4];
    __shared__ unsigned pbase[2][kCMaxPlanes + 4];   // p and p* planes k0 - 2 .. k0 + P + 1
    const int m = n - 1, P = (m + kCC - 1) / kCC, mm = m * m;
    const int rank = (int)cl_rank();
    const int k0 = 1 + rank * P;
    const int nown = max(0, min(k0 + P, m + 1) - k0) * mm;
    const int tid = threadIdx.x;
    const int np = n + 1;
    ClusterGeom g{m, P, (unsigned)__cvta_generic_to_shared(csm)};
    double* red = csm + kCVec * P * mm;
    long long* tile = reinterpret_cast<long long*>(red + 8);   // (P + 4) x (m + 4)^2
    __shared__ int wred[kCT / 32];
    const bool elide = rs == nullptr;
    auto sm = [&](int v, int t) -> double& { return csm[v * P * mm + t]; };
    auto gidx = [&](int t) {
        const int pl = t / mm, rem = t - pl * mm;
        const int j = rem / m + 1, i = rem - (j - 1) * m + 1;
        return ((size_t)(k0 + pl) * np + j) * np + i;
    };

    // the launch's start: the state, the own nodes of every vector, and
    // whether the shadow sequence is the primal one
    double rho = st->rho, rr = st->rr, alpha = st->alpha, beta = st->beta, sigma_s = st->sigma;
    int iter = st->iter, status = st->status, done = st->done;
    const int max_iter = st->max_iter;
    const double stop = st->tol * st->bnorm;
    double diff = 0.0;
    for (int t = tid; t < nown; t += kCT) {
        const size_t o = gidx(t);
        sm(VX, t) = x[o];
        sm(VR, t) = r[o];
        sm(VP, t) = p[o];
        if (!elide) {
            sm(VRS, t) = rs[o];
            sm(VPS, t) = ps[o];
            if (__double_as_longlong(rs[o]) != __double_as_longlong(r[o]) ||
                __double_as_longlong(ps[o]) != __double_as_longlong(p[o]))
                diff = 1.0;
        }
    }
    if (tid < P + 4) {
        pbase[0][tid] = cl_plane_base(g, VP, k0 - 2 + tid);
        pbase[1][tid] = cl_plane_base(g, VPS, k0 - 2 + tid);
    }
    for (int t = tid; t < (P + 4) * (m + 4) * (m + 4); t += kCT) tile[t] = 0ll;   // the zero border
    double tw[4] = {diff, 0.0, 0.0, 0.0};
    cl_reduce(tw, 1, 1, red, sh, bc);   // also: every CTA's vectors are loaded
    const bool twin = elide || tw[0] == 0.0;

    for (int it = 0; it < iters && !done; ++it) {
        // phase A: q = A p, q* = A^T p* (= A p* here), sigma = (p*, q)
        double a[4] = {0.0, 0.0, 0.0, 0.0};
        const int Ep = cl_fill_tile(pbase[0], P, m, tile, wred);
        for (int t = tid; t < nown; t += kCT) {
            const int pl = t / mm, rem = t - pl * mm;
            const int j = rem / m + 1, i = rem - (j - 1) * m + 1;
            sm(VQ, t) = cl_apply(tile, m, Ep, sigma, pl, i, j, k0 + pl);
        }
        if (!twin) {
            __syncthreads();   // every read of p's tile is done
            const int Es = cl_fill_tile(pbase[1], P, m, tile, wred);
            for (int t = tid; t < nown; t += kCT) {
                const int pl = t / mm, rem = t - pl * mm;
                const int j = rem / m + 1, i = rem - (j - 1) * m + 1;
                sm(VQS, t) = cl_apply(tile, m, Es, sigma, pl, i, j, k0 + pl);
            }
        }
        for (int t = tid; t < nown; t += kCT) a[0] += sm(twin ? VP : VPS, t) * sm(VQ, t);
        cl_reduce(a, 1, 0, red, sh, bc);
        sigma_s = a[0];
        if (!(rho != 0.0 && isfinite(rho)) || !(sigma_s != 0.0 && isfinite(sigma_s))) {
            status = kBreakdown;
            done = 1;
            break;
        }
        alpha = rho / sigma_s;
        // phase B: x += alpha p; r -= alpha q; r* -= alpha q*; (r*, r), (r, r)
        double b[4] = {0.0, 0.0, 0.0, 0.0};
        for (int t = tid; t < nown; t += kCT) {
            sm(VX, t) = sm(VX, t) + alpha * sm(VP, t);
            const double rn = sm(VR, t) - alpha * sm(VQ, t);
            sm(VR, t) = rn;
            b[1] += rn * rn;
            if (!twin) {
                const double rsn = sm(VRS, t) - alpha * sm(VQS, t);
                sm(VRS, t) = rsn;
                b[0] += rsn * rn;
            }
        }
        if (twin) b[0] = b[1];
        cl_reduce(b, 2, 1, red, sh, bc);
        const double rho_new = b[0];
        rr = b[1];
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
        // phase C: p = r + beta p; p* = r* + beta p*
        for (int t = tid; t < nown; t += kCT) {
            sm(VP, t) = sm(VR, t) + beta * sm(VP, t);
            if (!twin) sm(VPS, t) = sm(VRS, t) + beta * sm(VPS, t);
        }
        cl_sync();   // every p is final before the next operator phase reads it
    }

    // the launch's end: the own nodes back to global memory, the state
    for (int t = tid; t < nown; t += kCT) {
        const size_t o = gidx(t);
        x[o] = sm(VX, t);
        r[o] = sm(VR, t);
        p[o] = sm(VP, t);
        if (!elide) {
            rs[o] = twin ? sm(VR, t) : sm(VRS, t);
            ps[o] = twin ? sm(VP, t) : sm(VPS, t);
        }
    }
    if (rank == 0 && tid == 0) {
        st->rho = rho;
        st->rr = rr;
        st->alpha = alpha;
        st->beta = beta;
        st->sigma = sigma_s;
        st->iter = iter;
        st->status = status;
        st->done = done;
    }
    cl_sync();   // no CTA leaves while another may still read its shared memory
}

size_t cluster_smem(int n) {
    const int m = n - 1, P = (m + kCC - 1) / kCC;
    return (size_t)(kCVec * P * m * m + 8 + (P + 4) * (m + 4) * (m + 4)) * sizeof(double);
}

std::mutex g_cluster_mu;
std::vector<std::pair<int, int>> g_cluster_ok;   // (device, usable)

// Whether this device can keep one 16-CTA cluster of the kernel resident
// (queried once per device; the kernel is opted in to the non-portable
// cluster size and the largest shared memory it uses).
bool cluster_ready() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    std::lock_guard<std::mutex> lock(g_cluster_mu);
    for (auto& d : g_cluster_ok)
        if (d.first == dev) return d.second != 0;
    const size_t smem = cluster_smem(kCMaxM + 1);
    bool ok = cudaFuncSetAttribute(bicg_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                  cudaSuccess &&
              cudaFuncSetAttribute(bicg_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                  cudaSuccess;
    if (ok) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kCC, 1, 1);
        cfg.blockDim = dim3(kCT, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kCC;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        ok = cudaOccupancyMaxActiveClusters(&clusters, (const void*)bicg_cluster_kernel, &cfg) == cudaSuccess &&
             clusters >= 1;
    }
    if (!ok) cudaGetLastError();
    g_cluster_ok.push_back({dev, ok ? 1 : 0});
    return ok;
}

}  // namespace

bool cluster_bicg_usable(int n) { return n >= 4 && n - 1 <= kCMaxM && cluster_ready(); }

cudaError_t launch_bicg_cluster(double* x, double* r, double* rs, double* p, double* ps, int n, int bc_kind, int iters,
                                BicgState* st, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCC, 1, 1);
    cfg.blockDim = dim3(kCT, 1, 1);
    cfg.dynamicSmemBytes = cluster_smem(n);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kCC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int sigma = bc_kind == 1 ? 1 : -1;
    return cudaLaunchKernelEx(&cfg, bicg_cluster_kernel, x, r, rs, p, ps, n, sigma, iters, st);
}

}  // namespace excmg
