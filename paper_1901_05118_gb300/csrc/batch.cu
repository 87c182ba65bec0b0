// Many independent EXCMG solves on one GPU at once.
//
// Each instance keeps its whole level hierarchy (Alg. 1) and its Bi-CG (FP64)
// or refinement (FP64 around FP32 correction solves) state resident on the
// device and moves through a small state machine: direct solves of the two
// coarsest grids, then per Bi-CG level EXP_finite + right-hand side, FP64
// true residual, Bi-CG call (or FP32 correction solve and FP64 update),
// until the level's tolerance (or the stagnation rule) is met, and finally
// EXP_true.  The Bi-CG iterations (Alg. 2, M = I, r*_0 = r_0) of the
// instances waiting for them run per level group -- instances of one
// precision at one grid size -- each group on its own stream:
//  * grids up to 64^3 and FP32 correction solves: one cooperative launch for
//    all members; CTAs take operator tiles and vector chunks from every
//    member, members advance in lock step one iteration per grid-barrier
//    round, and each member's scalars are formed by the CTA that completes
//    its last tile / chunk;
//  * FP64 grids above 64^3 (launched mode): per member and round the single
//    solver's fused operator and update kernels with the member's own state.
// Instances can be submitted at any time (the engine admits them against
// its device-memory budget) and leave as soon as they are done, so the
// batch continuously refills: the same engine serves the fixed batch and
// the request stream.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <thread>
#include <vector>

#include "excmg_internal.cuh"
#include "grid_sync.cuh"
#include "march_f32.cuh"
#include "march_fx.cuh"
#include "march_pair.cuh"
#include "reduce.cuh"

namespace excmg {
namespace {

constexpr int kChunk = 8192;          // vector entries per chunk of the batched kernel
constexpr int kLd = 2;                // vector entries per thread loaded together
constexpr int kBatchMaxInst = 1024;

template <typename T>
struct BatchInst {     // device table entry, one per instance in the Bi-CG phase
    int n;
    int sigma;
    int gx, gy, kz_per, nunits, unit_begin;
    int nchunks, chunk_begin;
    int slot;          // index into the state array
    long long len;
    T *x, *r, *rs, *p, *ps, *q, *qs;
    T *p2, *ps2;       // FP64: second direction pair (p_k in p for even k, in p2 for odd k)
};

// One tile's operator pair (A p, A p* -- A is symmetric) and this thread's
// share of (p*, A p): FP32 arithmetic for the correction solves; for FP64
// solves the integer evaluation by the copy-ahead march (p* equals p bit for
// bit: every call starts from r*_0 = p_0 = p*_0 = r_0), with the general
// two-field march where a tile holds p* != p.  Called uniformly by the CTA.
__device__ __forceinline__ float march_pair(const BatchInst<float>& in, int bx, int by, int kz0, int kz1,
                                            unsigned char*) {
    return f32_march<2, true>(in.p, in.ps, in.q, in.qs, in.n, (float)in.sigma, bx, by, kz0, kz1);
}
__device__ __forceinline__ double march_pair(const BatchInst<double>& in, int bx, int by, int kz0, int kz1,
                                             unsigned char* smem) {
    __syncthreads();   // the CTA's previous unit is done with the shared buffers
    double d = 0.0;
    if (pp_march<false, true>(in.p, in.ps, in.q, in.qs, in.n, in.sigma, bx, by, kz0, kz1, smem, &d)) return d;
    __syncthreads();
    const FxFields fl{{in.p, in.ps}, {in.q, in.qs}, {nullptr, nullptr}, {nullptr, nullptr}, 0.0};
    return fx_march<2, true>(fl, nullptr, in.n, in.sigma, bx, by, kz0, kz1);
}

// FP64, iteration k >= 1 of a Bi-CG call: p_k = r_k + beta p_{k-1} (and p*_k)
// formed on every loaded node from the pair holding p_{k-1}, the CTA's own
// nodes written to the other pair, then the operator pair on p_k.
__device__ __forceinline__ double march_pair_dir(const BatchInst<double>& in, int k, double beta, int bx, int by,
                                                 int kz0, int kz1, unsigned char* smem) {
    const bool odd = k & 1;
    const double* pp = odd ? in.p : in.p2;
    const double* psp = odd ? in.ps : in.ps2;
    double* pn = odd ? in.p2 : in.p;
    double* psn = odd ? in.ps2 : in.ps;
    __syncthreads();   // the CTA's previous unit is done with the shared buffers
    double d = 0.0;
    const PairDir dir{in.r, in.rs, pn, psn, beta};
    if (pp_march<false, true, true>(pp, psp, in.q, in.qs, in.n, in.sigma, bx, by, kz0, kz1, smem, &d, dir))
        return d;
    __syncthreads();
    const FxFields fl{{pp, psp}, {in.q, in.qs}, {in.r, in.rs}, {pn, psn}, beta};
    return fx_march<2, true, true>(fl, nullptr, in.n, in.sigma, bx, by, kz0, kz1);
}

// dynamic shared memory of the batched kernel: the copy-ahead march's stages
// and tiles for FP64 instances, none for the FP32 march
template <typename T>
constexpr size_t batch_smem() {
    return sizeof(T) == sizeof(double) ? pp_smem_bytes<4>() : 0;
}

struct BatchState {    // device, one per slot
    double rho, rr, alpha, beta, sigma, tol;
    int iter, max_iter, done, status;
    unsigned int ticket_a, ticket_b;
    // set in phase A at a breakdown: the instance leaves the launch's count
    // of running instances in phase B, so that the count changes in phase B
    // only and every CTA reads the same value after its barrier
    int exit_pending, pad;
};

// Instance owning global index g, given each instance's first index.
__device__ __forceinline__ int owner(const int* begin, int ninst, int g) {
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// True in every thread of the CTA that took the last ticket of `ticket`.
__device__ __forceinline__ bool take_last(unsigned int* ticket, unsigned int total, bool* flag) {
    if (thread0()) {
        __threadfence();
        *flag = atomicAdd(ticket, 1u) == total - 1u;
    }
    __syncthreads();
    const bool last = *flag;
    __syncthreads();
    return last;
}

__device__ __forceinline__ double sum_range(const double* v, int begin, int count, int stride, double* sh) {
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nt = blockDim.x * blockDim.y;
    double s = 0.0;
    for (int k = tid; k < count; k += nt) s += __ldcg(&v[(size_t)(begin + k) * stride]);
    return block_sum(s, sh);
}

template <typename T>
__global__ void __launch_bounds__(S_NT, 2)
batch_bicg_kernel(const BatchInst<T>* __restrict__ inst, const int* __restrict__ unit_begin,
                    const int* __restrict__ chunk_begin, int ninst, int total_units, int total_chunks,
                    double* unit_part, double* chunk_part, BatchState* states, int iters, int* active,
                    GridBarrier gb, int* rounds) {
    __shared__ double sh[32];
    __shared__ T shf[32];
    __shared__ bool flag;
    extern __shared__ __align__(128) unsigned char batch_smem_buf[];
    // FP64 groups fold the direction update into the operator phase (two
    // grid barriers per round); FP32 groups keep a separate phase C
    constexpr bool kFused = sizeof(T) == sizeof(double);
    const unsigned int G = gridDim.x;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nt = blockDim.x * blockDim.y;
    bool ok = true;
    int rounds_done = 0;
    for (int it = 0; it < iters && ok; ++it) {
        ++rounds_done;
        // phase A: q = A p, q* = A p*, per-tile (p*, q); the CTA finishing an
        // instance's last tile forms sigma and alpha
        for (int u = blockIdx.x; u < total_units; u += G) {
            const int i = owner(unit_begin, ninst, u);
            const BatchInst<T>& in = inst[i];
            BatchState& st = states[in.slot];
            if (*(volatile int*)&st.done) continue;
            const int loc = u - in.unit_begin;
            const int bx = loc % in.gx, by = (loc / in.gx) % in.gy, bz = loc / (in.gx * in.gy);
            const int kz0 = 1 + bz * in.kz_per;
            T d;
            if constexpr (kFused) {
                // the state's iteration count is this call's k until phase B
                // of this round completes
                const int k = st.iter;
                d = k == 0 ? march_pair(in, bx, by, kz0, min(kz0 + in.kz_per, in.n), batch_smem_buf)
                           : march_pair_dir(in, k, st.beta, bx, by, kz0, min(kz0 + in.kz_per, in.n),
                                            batch_smem_buf);
            } else {
                d = march_pair(in, bx, by, kz0, min(kz0 + in.kz_per, in.n), batch_smem_buf);
            }
            const double ds = (double)block_sum(d, shf);
            if (thread0()) unit_part[u] = ds;
            if (take_last(&st.ticket_a, (unsigned)in.nunits, &flag)) {
                const double sg = sum_range(unit_part, in.unit_begin, in.nunits, 1, sh);
                if (thread0()) {
                    st.sigma = sg;
                    if (!(st.rho != 0.0 && isfinite(st.rho)) || !(sg != 0.0 && isfinite(sg))) {
                        st.status = kBreakdown;
                        st.done = 1;
                        st.exit_pending = 1;
                    } else {
                        st.alpha = st.rho / sg;
                    }
                    st.ticket_a = 0;
                }
            }
        }
        if (!(ok = grid_sync(gb, G))) break;
        // phase B: x += alpha p; r -= alpha q; r* -= alpha q*; per-chunk
        // (r*, r), (r, r); the CTA finishing the last chunk forms beta and
        // tests convergence
        for (int c = blockIdx.x; c < total_chunks; c += G) {
            const int i = owner(chunk_begin, ninst, c);
            const BatchInst<T>& in = inst[i];
            BatchState& st = states[in.slot];
            if (*(volatile int*)&st.done) {
                // an instance that broke down in phase A of this round: its
                // chunks update nothing, the CTA taking the last one takes
                // it out of the running count
                if (*(volatile int*)&st.exit_pending && take_last(&st.ticket_b, (unsigned)in.nchunks, &flag) &&
                    thread0()) {
                    st.exit_pending = 0;
                    st.ticket_b = 0;
                    atomicSub(active, 1);
                }
                continue;
            }
            const T alpha = (T)st.alpha;
            const T* const pk = (kFused && (st.iter & 1)) ? in.p2 : in.p;   // p_k
            const long long t0 = (long long)(c - in.chunk_begin) * kChunk;
            const long long t1 = min(t0 + kChunk, in.len);
            T vr = 0, vrr = 0;
            // kLd entries per thread loaded together, then updated and summed
            // in index order
            for (long long tb = t0 + tid; tb < t1; tb += (long long)kLd * nt) {
                T xv[kLd], pv[kLd], rv[kLd], qv[kLd], rsv[kLd], qsv[kLd];
#pragma unroll
                for (int k = 0; k < kLd; ++k) {
                    const long long t = tb + (long long)k * nt;
                    if (t < t1) {
                        xv[k] = in.x[t];
                        pv[k] = pk[t];
                        rv[k] = in.r[t];
                        qv[k] = in.q[t];
                        rsv[k] = in.rs[t];
                        qsv[k] = in.qs[t];
                    }
                }
#pragma unroll
                for (int k = 0; k < kLd; ++k) {
                    const long long t = tb + (long long)k * nt;
                    if (t >= t1) break;
                    in.x[t] = xv[k] + alpha * pv[k];
                    const T rn = rv[k] - alpha * qv[k];
                    const T rsn = rsv[k] - alpha * qsv[k];
                    in.r[t] = rn;
                    in.rs[t] = rsn;
                    vr += rsn * rn;
                    vrr += rn * rn;
                }
            }
            const double a = (double)block_sum(vr, shf);
            const double b = (double)block_sum(vrr, shf);
            if (thread0()) {
                chunk_part[2 * (size_t)c] = a;
                chunk_part[2 * (size_t)c + 1] = b;
            }
            if (take_last(&st.ticket_b, (unsigned)in.nchunks, &flag)) {
                const double rho_new = sum_range(chunk_part, in.chunk_begin, in.nchunks, 2, sh);
                const double rr = sum_range(chunk_part + 1, in.chunk_begin, in.nchunks, 2, sh);
                if (thread0()) {
                    st.beta = rho_new / st.rho;
                    st.rho = rho_new;
                    st.rr = rr;
                    st.iter += 1;
                    if (sqrt(rr) <= st.tol) {
                        st.status = kConverged;
                        st.done = 1;
                        atomicSub(active, 1);
                    } else if (st.iter >= st.max_iter) {
                        st.status = kCapped;
                        st.done = 1;
                        atomicSub(active, 1);
                    }
                    st.ticket_b = 0;
                }
            }
        }
        if (!(ok = grid_sync(gb, G))) break;
        // the counter changes only in phase B: between this barrier and the
        // next phase B every CTA reads the same value
        if (*(volatile int*)active <= 0) break;
        if constexpr (!kFused) {
            // phase C: p = r + beta p; p* = r* + beta p*
            for (int c = blockIdx.x; c < total_chunks; c += G) {
                const int i = owner(chunk_begin, ninst, c);
                const BatchInst<T>& in = inst[i];
                const BatchState& st = states[in.slot];
                if (*(volatile const int*)&st.done) continue;
                const T beta = (T)st.beta;
                const long long t0 = (long long)(c - in.chunk_begin) * kChunk;
                const long long t1 = min(t0 + kChunk, in.len);
                for (long long tb = t0 + tid; tb < t1; tb += (long long)kLd * nt) {
                    T rv[kLd], pv[kLd], rsv[kLd], psv[kLd];
#pragma unroll
                    for (int k = 0; k < kLd; ++k) {
                        const long long t = tb + (long long)k * nt;
                        if (t < t1) {
                            rv[k] = in.r[t];
                            pv[k] = in.p[t];
                            rsv[k] = in.rs[t];
                            psv[k] = in.ps[t];
                        }
                    }
#pragma unroll
                    for (int k = 0; k < kLd; ++k) {
                        const long long t = tb + (long long)k * nt;
                        if (t >= t1) break;
                        in.p[t] = rv[k] + beta * pv[k];
                        in.ps[t] = rsv[k] + beta * psv[k];
                    }
                }
            }
            if (!(ok = grid_sync(gb, G))) break;
        }
    }
    if (blockIdx.x == 0 && thread0()) {
        if (!ok) *active = -1;   // barrier gave up
        *rounds = rounds_done;
    }
}

// r32 = r / s, e = 0, r*_0 = p_0 = p*_0 = r_0 and rho_0 = (r_0, r_0) of one
// instance's correction solve; the state is initialised by the last CTA.
__global__ void __launch_bounds__(kVecThreads)
batch_init32_kernel(const double* __restrict__ r64, double inv_s, float* __restrict__ r32, float* __restrict__ e,
                    float* __restrict__ rs, float* __restrict__ p, float* __restrict__ ps, size_t len,
                    double* partials, unsigned int* ticket, BatchState* st, double tol, int max_iter) {
    __shared__ float shf[32];
    __shared__ double sh[32];
    __shared__ bool am_last;
    float v = 0.f;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len; t += (size_t)gridDim.x * blockDim.x) {
        const float rv = (float)(r64[t] * inv_s);
        r32[t] = rv;
        e[t] = 0.f;
        rs[t] = rv;
        p[t] = rv;
        ps[t] = rv;
        v += rv * rv;
    }
    const double s = (double)block_sum(v, shf);
    if (publish_partials(&s, 1, partials, ticket, &am_last)) {
        const double tot = gather_partials(partials, 0, sh);
        if (thread0()) {
            st->rho = tot;
            st->rr = tot;
            st->alpha = st->beta = st->sigma = 0.0;
            st->tol = tol * sqrt(tot);
            st->iter = 0;
            st->max_iter = max_iter;
            const bool conv = sqrt(tot) <= st->tol;
            st->done = conv ? 1 : 0;
            st->status = conv ? kConverged : kRunning;
            st->ticket_a = st->ticket_b = 0;
            *ticket = 0;
        }
    }
}

__global__ void __launch_bounds__(kVecThreads)
batch_correct_kernel(double* __restrict__ u, const float* __restrict__ e, size_t len, double s) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len; t += (size_t)gridDim.x * blockDim.x)
        u[t] = u[t] + s * (double)e[t];
}

// The cooperative grid: every SM of the current device, at most two CTAs each.
template <typename T>
int batch_resident_ctas() {
    const int occ = min(2, kernel_occupancy((const void*)batch_bicg_kernel<T>, S_NT, batch_smem<T>()));
    return device_sms() * occ;
}

}  // namespace
}  // namespace excmg

using namespace excmg;

// ------------------------------------------------------------------ host side
namespace {

enum Phase { kSetup = 0, kResidual = 1, kInner = 2, kFinal = 3, kDone = 4, kFailed = 5 };

struct Instance {
    int id = -1;
    int n = 0, nc = 0, bc = 1, nl = 0, L = 0;
    int prec = EXCMG_PRECISION_MIXED;
    const double* f = nullptr;
    const double* g1 = nullptr;
    const double* g2 = nullptr;
    double* u_out = nullptr;
    double tol = 1e-8, inner_tol = 1e-4;
    int tol_mode = EXCMG_TOL_UNIFORM;
    int max_iter = 100000, max_total = 1000000;
    // device buffers (one allocation)
    void* block = nullptr;
    size_t bytes = 0;
    std::vector<double*> u;    // per level
    double *fh = nullptr, *res = nullptr, *W = nullptr;
    // FP64 Bi-CG vectors (r is `res`)
    double *rs64 = nullptr, *p64 = nullptr, *ps64 = nullptr, *q64 = nullptr, *qs64 = nullptr;
    double *p2_64 = nullptr, *ps2_64 = nullptr;   // second direction pair
    // launched mode (FP64 levels above 64^3): iterations of the current
    // Bi-CG call enqueued so far, and which direction pair holds p_k
    long long launched_k = 0;
    bool dir_in_p2 = false;
    // FP32 correction solve vectors
    float *r32 = nullptr, *e = nullptr, *r = nullptr, *rs = nullptr, *p = nullptr, *ps = nullptr, *q = nullptr,
          *qs = nullptr;
    // device state slot (fixed for the instance's life) and whether a group
    // launch holding it is running
    int slot = -1;
    bool in_flight = false;
    // progress
    Phase phase = kSetup;
    int level = 0;
    int iters = 0, outer = 0, bad = 0, stag = 0;
    int call_iter = 0;         // iterations of the current Bi-CG call taken back so far
    double fnorm = 0.0, rel = 0.0, prev = 0.0, scale = 0.0;
    int status = EXCMG_OK;
    excmg_stats stats{};
    double t_submit = 0.0, t_done = 0.0;
};

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

size_t instance_bytes(int n, int nc, int prec) {
    size_t b = 0;
    for (int m = nc; m <= n; m *= 2) b += align256(node_count(m) * sizeof(double));   // u per level
    b += 2 * align256(node_count(n) * sizeof(double));                                   // fh, res
    b += align256(node_count(n / 2) * sizeof(double));                                   // W
    if (prec == EXCMG_PRECISION_FP64)
        b += 7 * align256(node_count(n) * sizeof(double));                   // r*, p, p*, q, q*, p2, p*2
    else
        b += 8 * align256(node_count(n) * sizeof(float));                                // r32, e, 6 vectors
    return b;
}

}  // namespace

struct excmg_batch {
    excmg_ctx* ctx = nullptr;
    size_t budget = 0, bytes = 0;
    int max_instances = 0;
    int next_id = 0;
    std::vector<Instance*> live;
    std::vector<Instance*> finished;
    // per-slot Bi-CG states of the cooperative launches (device, pinned host)
    BatchState* d_states = nullptr;
    BatchState* h_states = nullptr;
    double* d_norms = nullptr;   // per-slot norms
    double* h_norms = nullptr;
    int inner_chunk = 256;       // iterations per cooperative launch
    int launched_rounds = 16;    // iterations per launched-mode group launch
    std::string last_error;
    long long launches = 0;
    excmg_batch_profile prof{};
    // launched mode: a Bi-CG state and a partial-sum array per slot, and a
    // pinned host copy of the states
    BicgState* d_bstate = nullptr;
    BicgState* h_bstate = nullptr;
    double* d_bpart = nullptr;
    std::vector<int> free_slots;
    // One cooperative launch per level group (instances of one precision at
    // one grid size), each on its own stream with its own tables, partial
    // sums, barrier and counters, harvested as soon as it completes.
    struct Group {
        cudaStream_t stream = nullptr;
        cudaEvent_t start = nullptr, done = nullptr;
        bool busy = false;
        bool launched = false;   // launched mode: per-member kernels, no grid barrier
        int prec = 0, n = 0, ctas = 0, cand = -1;
        std::vector<Instance*> members;
        void* d_inst = nullptr;        // BatchInst<T>[max_instances]
        int *d_unit_begin = nullptr, *d_chunk_begin = nullptr, *d_active = nullptr, *d_rounds = nullptr;
        int *h_active = nullptr, *h_rounds = nullptr;
        unsigned int* d_barrier = nullptr;
        double *d_unit_part = nullptr, *d_chunk_part = nullptr;
        size_t unit_cap = 0, chunk_cap = 0;
    };
    std::vector<Group> groups;
    cudaEvent_t host_ready = nullptr;   // the context stream's state uploads
    // Grid-size tuner (its table is the context's, shared by its batches).
    // Candidate c gives each instance ceil(W / kTuneItems[c]) CTAs, W being
    // its operator tiles or vector chunks, whichever are more.  Candidates
    // are tried from the most CTAs down, and trying stops once a round takes
    // more than twice the best round time seen.  The choice: the fewest
    // CTA-milliseconds per instance round among the candidates within 1.25x
    // of the best round time.  The grid size changes no result bit (every
    // partial sum belongs to a tile or chunk, not to a CTA).
};

namespace {

void bnote(excmg_batch* b, long long k) {
    b->launches += k;
    note_launches(k);
}

int bfail(excmg_batch* b, int st, const std::string& m) {
    b->last_error = m;
    return st;
}

int bcuda(excmg_batch* b, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return EXCMG_OK;
    cudaGetLastError();
    return bfail(b, EXCMG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void free_instance(excmg_batch* b, Instance* in) {
    if (in->block) {
        cudaFree(in->block);
        b->bytes -= in->bytes;
        in->block = nullptr;
    }
}

// Level l's eps (Alg. 1's tolerance schedule).
double level_eps(const Instance* in, int l) {
    const int i = l - 1;
    return in->tol_mode == EXCMG_TOL_PAPER ? in->tol * std::pow(10.0, (double)(i - in->L)) : in->tol;
}

// ||a||_2 over the level for every instance listed, one sync.
int norms(excmg_batch* b, const std::vector<std::pair<Instance*, const double*>>& work) {
    excmg_ctx* ctx = b->ctx;
    for (size_t k = 0; k < work.size(); ++k) {
        Instance* in = work[k].first;
        const int N = in->nc << in->level;
        cudaError_t e = launch_dot(work[k].second, work[k].second, node_count(N), ctx->partials, ctx->ticket,
                                   b->d_norms + k, ctx->stream);
        bnote(b, 1);
        if (e != cudaSuccess) return bcuda(b, e, "batch norm");
    }
    if (work.empty()) return EXCMG_OK;
    cudaError_t e = cudaMemcpyAsync(b->h_norms, b->d_norms, work.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return bcuda(b, e, "batch norm read");
}

// Set up level `in->level`: right-hand side, initial guess, and for the two
// coarsest levels the direct solve.
int setup_level(excmg_batch* b, Instance* in) {
    excmg_ctx* ctx = b->ctx;
    const int l = in->level, N = in->nc << l, stride = in->n / N;
    double* u = in->u[l];
    cudaError_t e = launch_assemble_rhs(in->fh, N, in->bc, in->f, in->g1, in->g2, stride, ctx->stream);
    if (e == cudaSuccess && l >= 2) e = launch_exp_finite(u, in->u[l - 1], in->u[l - 2], in->W, N, ctx->stream);
    if (e == cudaSuccess) e = launch_set_boundary(u, N, in->g1, stride, ctx->stream);
    // the operator writes interior entries only and the buffers of A p, A p*
    // are shared by all levels: clear them in this level's layout, or the
    // previous level's values would sit on this level's boundary nodes and
    // enter r, the inner products and u through the vector updates
    if (e == cudaSuccess && l >= 2) {
        const size_t len = node_count(N);
        if (in->prec == EXCMG_PRECISION_FP64) {
            // (the second direction pair as well: the operator phase writes
            // its interior entries only)
            double* const zero[] = {in->q64, in->qs64, in->p2_64, in->ps2_64};
            for (double* z : zero)
                if (e == cudaSuccess) e = cudaMemsetAsync(z, 0, len * sizeof(double), ctx->stream);
        } else {
            e = cudaMemsetAsync(in->q, 0, len * sizeof(float), ctx->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(in->qs, 0, len * sizeof(float), ctx->stream);
        }
    }
    bnote(b, l >= 2 ? 4 : 2);
    if (e != cudaSuccess) return bcuda(b, e, "level setup");
    if (l <= 1) {
        const int st = dsolve_run(ctx, N, in->bc, in->fh, u);
        bnote(b, 1);
        if (st) return bfail(b, st, ctx->last_error);
    }
    return EXCMG_OK;
}

int finish(excmg_batch* b, Instance* in) {
    excmg_ctx* ctx = b->ctx;
    const int lf = in->nl - 1;
    cudaError_t e = launch_exp_true(in->u_out, in->u[lf], in->u[lf - 1], in->n, ctx->stream);
    bnote(b, 1);
    return bcuda(b, e, "EXP_true");
}

bool grow(excmg_batch* b, double** buf, size_t* cap, size_t need) {
    if (need <= *cap) return true;
    cudaFree(*buf);
    *cap = need * 2;
    if (cudaMalloc(buf, *cap * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        *cap = 0;
        *buf = nullptr;
        return false;
    }
    return true;
}

// Tile / chunk geometry of one instance's current level.
template <typename T>
BatchInst<T> geometry(Instance* in, int slot, int* units, int* chunks) {
    const int N = in->nc << in->level, m = N - 1;
    BatchInst<T> t{};
    t.n = N;
    t.sigma = in->bc == 1 ? 1 : -1;
    t.gx = (m + S_TX - 1) / S_TX;
    t.gy = (m + S_OY - 1) / S_OY;
    t.kz_per = m < 8 ? m : (N >= 128 ? 16 : 8);   // longer slabs: less halo per output plane
    t.nunits = t.gx * t.gy * ((m + t.kz_per - 1) / t.kz_per);
    t.unit_begin = *units;
    t.len = (long long)node_count(N);
    t.nchunks = (int)((t.len + kChunk - 1) / kChunk);
    t.chunk_begin = *chunks;
    t.slot = slot;
    *units += t.nunits;
    *chunks += t.nchunks;
    return t;
}

// ------------------------------------------------------------ level groups
constexpr int kTuneCands = 5;
constexpr int kTuneItems[kTuneCands] = {1, 2, 4, 8, 16};   // tiles or chunks per CTA

// CTAs per instance of candidate c for an instance with W work items.
int tune_cpi(int W, int c) { return (W + kTuneItems[c] - 1) / kTuneItems[c]; }

int capacity_of(int prec) {
    return prec == EXCMG_PRECISION_FP64 ? batch_resident_ctas<double>() : batch_resident_ctas<float>();
}

// The group record's stream, events and fixed tables (made once).
int group_init(excmg_batch* b, excmg_batch::Group& g) {
    if (g.stream) return EXCMG_OK;
    const size_t mi = (size_t)b->max_instances;
    bool ok = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreate(&g.start) == cudaSuccess && cudaEventCreate(&g.done) == cudaSuccess &&
              cudaMalloc(&g.d_inst, mi * sizeof(BatchInst<double>)) == cudaSuccess &&
              cudaMalloc(&g.d_unit_begin, mi * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&g.d_chunk_begin, mi * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&g.d_active, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&g.d_rounds, sizeof(int)) == cudaSuccess &&
              cudaMallocHost(&g.h_active, 2 * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&g.d_barrier, 4 * sizeof(unsigned int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return bfail(b, EXCMG_ERR_OOM, "batch group buffers");
    }
    g.h_rounds = g.h_active + 1;
    return EXCMG_OK;
}

void group_free(excmg_batch::Group& g) {
    if (g.stream) cudaStreamSynchronize(g.stream);
    cudaFree(g.d_inst);
    cudaFree(g.d_unit_begin);
    cudaFree(g.d_chunk_begin);
    cudaFree(g.d_active);
    cudaFree(g.d_rounds);
    cudaFreeHost(g.h_active);
    cudaFree(g.d_barrier);
    cudaFree(g.d_unit_part);
    cudaFree(g.d_chunk_part);
    if (g.start) cudaEventDestroy(g.start);
    if (g.done) cudaEventDestroy(g.done);
    if (g.stream) cudaStreamDestroy(g.stream);
    g = excmg_batch::Group{};
}

// One cooperative launch of up to b->inner_chunk Bi-CG iterations for the
// instances `list` (one precision, one grid size) on group record g, with
// `ctas` CTAs, after the context stream's state uploads.
template <typename T>
int launch_group(excmg_batch* b, excmg_batch::Group& g, const std::vector<Instance*>& list, int ctas, int cand) {
    int st = group_init(b, g);
    if (st) return st;
    std::vector<BatchInst<T>> tab;
    std::vector<int> ub, cb;
    int units = 0, chunks = 0;
    for (Instance* in : list) {
        BatchInst<T> t = geometry<T>(in, in->slot, &units, &chunks);
        if (sizeof(T) == sizeof(double)) {
            t.x = (T*)in->u[in->level];
            t.r = (T*)in->res;
            t.rs = (T*)in->rs64;
            t.p = (T*)in->p64;
            t.ps = (T*)in->ps64;
            t.q = (T*)in->q64;
            t.qs = (T*)in->qs64;
            t.p2 = (T*)in->p2_64;
            t.ps2 = (T*)in->ps2_64;
        } else {
            t.x = (T*)in->e;
            t.r = (T*)in->r;
            t.rs = (T*)in->rs;
            t.p = (T*)in->p;
            t.ps = (T*)in->ps;
            t.q = (T*)in->q;
            t.qs = (T*)in->qs;
        }
        ub.push_back(t.unit_begin);
        cb.push_back(t.chunk_begin);
        tab.push_back(t);
    }
    // the tables are pageable host vectors: each cudaMemcpyAsync below has
    // staged them by the time it returns
    if (!grow(b, &g.d_unit_part, &g.unit_cap, (size_t)units) ||
        !grow(b, &g.d_chunk_part, &g.chunk_cap, 2 * (size_t)chunks))
        return bfail(b, EXCMG_ERR_OOM, "batch partials");
    cudaStream_t s = g.stream;
    *g.h_active = (int)tab.size();
    cudaError_t e = cudaStreamWaitEvent(s, b->host_ready, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g.d_inst, tab.data(), tab.size() * sizeof(BatchInst<T>), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g.d_unit_begin, ub.data(), ub.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g.d_chunk_begin, cb.data(), cb.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g.d_active, g.h_active, sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g.d_barrier, 0, 4 * sizeof(unsigned int), s);
    if (e != cudaSuccess) return bcuda(b, e, "batch table upload");
    int iters = b->inner_chunk;
    int ninst = (int)tab.size();
    const BatchInst<T>* di = (const BatchInst<T>*)g.d_inst;
    const int* d_ub = g.d_unit_begin;
    const int* d_cb = g.d_chunk_begin;
    double* up = g.d_unit_part;
    double* cp = g.d_chunk_part;
    BatchState* sts = b->d_states;
    int* act = g.d_active;
    int* rounds = g.d_rounds;
    GridBarrier gb{g.d_barrier, g.d_barrier + 1, (int*)(g.d_barrier + 2), kBarrierSpinLimit};
    void* args[] = {(void*)&di,    (void*)&d_ub,  (void*)&d_cb, (void*)&ninst, (void*)&units, (void*)&chunks,
                    (void*)&up,    (void*)&cp,    (void*)&sts,  (void*)&iters, (void*)&act,   (void*)&gb,
                    (void*)&rounds};
    e = cudaEventRecord(g.start, s);
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel((const void*)batch_bicg_kernel<T>, dim3(ctas), dim3(S_TX, S_TY, 1), args,
                                        batch_smem<T>(), s);
    bnote(b, 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g.h_active, g.d_active, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g.h_rounds, g.d_rounds, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(g.done, s);
    if (e != cudaSuccess) return bcuda(b, e, "batched Bi-CG launch");
    g.busy = true;
    g.prec = sizeof(T) == sizeof(double) ? EXCMG_PRECISION_FP64 : EXCMG_PRECISION_MIXED;
    g.n = list.empty() ? 0 : (list[0]->nc << list[0]->level);
    g.ctas = ctas;
    g.cand = cand;
    g.members = list;
    for (Instance* in : list) in->in_flight = true;
    return EXCMG_OK;
}

// FP64 levels above the cooperative kernel's range run in launched mode:
// per member and iteration the single solver's two kernels (the operator
// launch with the direction update folded in, then the update), with the
// member's own state and partial sums, so that a large level moves its
// bytes as fast as in a single solve.
bool launched_level(const Instance* in) {
    return in->prec == EXCMG_PRECISION_FP64 && (in->nc << in->level) > kPersistentMaxN;
}

int launch_group_launched(excmg_batch* b, excmg_batch::Group& g, const std::vector<Instance*>& list) {
    int st = group_init(b, g);
    if (st) return st;
    cudaStream_t s = g.stream;
    const int K = b->launched_rounds;
    long long nl = 0;
    cudaError_t e = cudaStreamWaitEvent(s, b->host_ready, 0);
    if (e == cudaSuccess) e = cudaEventRecord(g.start, s);
    for (int k = 0; k < K && e == cudaSuccess; ++k) {
        for (Instance* in : list) {
            if (e != cudaSuccess) break;
            const int N = in->nc << in->level;
            BicgState* bs = b->d_bstate + in->slot;
            double* part = b->d_bpart + (size_t)in->slot * kMaxPartials;
            double* pc = in->dir_in_p2 ? in->p2_64 : in->p64;
            double* psc = in->dir_in_p2 ? in->ps2_64 : in->ps64;
            if (in->launched_k == 0) {
                // p_0 = r_0: the operator pair on the fused schedule's grid
                e = launch_bicg_stencil_pair(pc, in->q64, psc, in->qs64, N, in->bc, part, bs, s, true);
            } else {
                double* pn = in->dir_in_p2 ? in->p64 : in->p2_64;
                double* psn = in->dir_in_p2 ? in->ps64 : in->ps2_64;
                e = launch_bicg_stencil_pair_dir(in->res, in->rs64, pc, psc, pn, psn, in->q64, in->qs64, N, in->bc,
                                                 part, bs, s);
                in->dir_in_p2 = !in->dir_in_p2;
                pc = pn;
            }
            if (e == cudaSuccess)
                e = launch_bicg_update(in->u[in->level], pc, in->res, in->q64, in->rs64, in->qs64, node_count(N), part,
                                       bs, s);
            ++in->launched_k;
            nl += 2;
        }
    }
    bnote(b, nl);
    for (Instance* in : list)
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->h_bstate + in->slot, b->d_bstate + in->slot, sizeof(BicgState),
                                cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(g.done, s);
    if (e != cudaSuccess) return bcuda(b, e, "launched batch group");
    *g.h_active = 0;
    *g.h_rounds = K;
    g.busy = true;
    g.launched = true;
    g.prec = EXCMG_PRECISION_FP64;
    g.n = list[0]->nc << list[0]->level;
    g.ctas = 0;
    g.cand = -1;
    g.members = list;
    for (Instance* in : list) in->in_flight = true;
    return EXCMG_OK;
}

excmg_ctx::BatchTune& tune_of(excmg_batch* b, int prec, int n) {
    auto& table = b->ctx->batch_tune;
    auto it = table.find({prec, n});
    if (it == table.end()) {
        excmg_ctx::BatchTune t;
        for (int k = 0; k < 8; ++k) t.ms[k] = t.cta_ms[k] = -1.0;
        t.settled = false;
        it = table.emplace(std::make_pair(prec, n), t).first;
    }
    return it->second;
}

// A completed group launch: its members' states come back, the tuner learns
// the launch's cost, and every member whose Bi-CG call ended goes back to the
// true-residual test of Alg. 1 (mixed: after u += ||r|| e).
int harvest(excmg_batch* b, excmg_batch::Group& g) {
    excmg_ctx* ctx = b->ctx;
    cudaError_t e = cudaSuccess;
    if (!g.launched)
        for (Instance* in : g.members)
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(b->h_states + in->slot, b->d_states + in->slot, sizeof(BatchState),
                                    cudaMemcpyDeviceToHost, g.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g.stream);
    if (e != cudaSuccess) return bcuda(b, e, "batch state read");
    if (g.launched) {
        // the members' states came back in the single solver's layout
        for (Instance* in : g.members) {
            const BicgState& bs = b->h_bstate[in->slot];
            BatchState& hs = b->h_states[in->slot];
            hs.done = bs.done;
            hs.status = bs.status;
            hs.iter = bs.iter;
            hs.rr = bs.rr;
            hs.rho = bs.rho;
        }
        g.launched = false;
    }
    g.busy = false;
    for (Instance* in : g.members) in->in_flight = false;
    if (*g.h_active < 0) return bfail(b, EXCMG_ERR_TIMEOUT, "grid barrier of the batched Bi-CG gave up");
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, g.start, g.done) != cudaSuccess) {
        cudaGetLastError();
        ms = -1.f;
    }
    b->prof.group_launches += 1;
    b->prof.rounds += *g.h_rounds;
    b->prof.member_rounds += (long long)*g.h_rounds * (long long)g.members.size();
    if (ms >= 0.f) b->prof.group_ms += ms;
    for (Instance* in : g.members) {
        const BatchState& hs = b->h_states[in->slot];
        b->prof.member_iters += hs.iter - in->call_iter;
        in->call_iter = hs.iter;
    }
    if (g.cand >= 0 && *g.h_rounds > 0) {
        if (ms >= 0.f) {
            excmg_ctx::BatchTune& t = tune_of(b, g.prec, g.n);
            const double per_round = (double)ms / (double)*g.h_rounds;
            const double c = per_round * g.ctas / (double)g.members.size();
            if (t.ms[g.cand] < 0.0 || per_round < t.ms[g.cand]) {
                t.ms[g.cand] = per_round;
                t.cta_ms[g.cand] = c;
            }
            double best = -1.0;
            bool all = true;
            for (int k = 0; k < kTuneCands; ++k) {
                if (t.ms[k] < 0.0) all = false;
                else if (best < 0.0 || t.ms[k] < best) best = t.ms[k];
            }
            if (all || per_round > 2.0 * best) t.settled = true;
        }
    }
    for (Instance* in : g.members) {
        if (in->phase != kInner) continue;
        const BatchState& hs = b->h_states[in->slot];
        if (!hs.done) continue;   // the launch's iteration chunk ended first
        if (hs.status == kBreakdown) {
            in->phase = kFailed;
            in->status = EXCMG_ERR_BREAKDOWN;
            continue;
        }
        in->iters += hs.iter;
        ++in->outer;
        if (in->prec == EXCMG_PRECISION_MIXED) {
            const int N = in->nc << in->level;
            batch_correct_kernel<<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(in->u[in->level], in->e, node_count(N),
                                                                              in->scale);
            bnote(b, 1);
            if ((e = cudaGetLastError()) != cudaSuccess) return bcuda(b, e, "batch correction");
        }
        in->phase = kResidual;
    }
    g.members.clear();
    return EXCMG_OK;
}

// CTAs for a group of m instances of grid size n with W work items each:
// the tuner's next candidate while it is still trying, else its choice; *cand
// the candidate index.
int group_ctas(excmg_batch* b, int prec, int n, int W, int m, int* cand) {
    excmg_ctx::BatchTune& t = tune_of(b, prec, n);
    int pick = -1;
    if (!t.settled) {
        for (int k = 0; k < kTuneCands && pick < 0; ++k) {
            if (t.ms[k] >= 0.0) continue;
            if (k > 0 && t.ms[k - 1] >= 0.0 && tune_cpi(W, k) == tune_cpi(W, k - 1)) {
                // the same grid as the candidate before: nothing new to learn
                t.ms[k] = t.ms[k - 1];
                t.cta_ms[k] = t.cta_ms[k - 1];
                continue;
            }
            pick = k;
        }
        if (pick < 0) t.settled = true;
    }
    if (pick < 0) {
        double best = -1.0;
        for (int k = 0; k < kTuneCands; ++k)
            if (t.ms[k] >= 0.0 && (best < 0.0 || t.ms[k] < best)) best = t.ms[k];
        for (int k = 0; k < kTuneCands; ++k)
            if (t.ms[k] >= 0.0 && t.ms[k] <= 1.25 * best && (pick < 0 || t.cta_ms[k] < t.cta_ms[pick])) pick = k;
        if (pick < 0) pick = 0;
    }
    *cand = pick;
    return tune_cpi(W, pick) * m;
}

}  // namespace

extern "C" {

int excmg_batch_create(excmg_ctx* ctx, size_t hbm_budget_bytes, int max_instances, excmg_batch** out) {
    if (!ctx || !out || max_instances < 1 || max_instances > kBatchMaxInst) return EXCMG_ERR_ARG;
    *out = nullptr;
    excmg_batch* b = new (std::nothrow) excmg_batch();
    if (!b) return EXCMG_ERR_OOM;
    b->ctx = ctx;
    b->budget = hbm_budget_bytes;
    b->max_instances = max_instances;
    const size_t mi = (size_t)max_instances;
    bool ok = cudaMalloc(&b->d_states, mi * sizeof(BatchState)) == cudaSuccess &&
              cudaMallocHost(&b->h_states, mi * sizeof(BatchState)) == cudaSuccess &&
              cudaMalloc(&b->d_norms, mi * sizeof(double)) == cudaSuccess &&
              cudaMallocHost(&b->h_norms, mi * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&b->d_bstate, mi * sizeof(BicgState)) == cudaSuccess &&
              cudaMallocHost(&b->h_bstate, mi * sizeof(BicgState)) == cudaSuccess &&
              cudaMalloc(&b->d_bpart, mi * (size_t)kMaxPartials * sizeof(double)) == cudaSuccess &&
              cudaMemset(b->d_states, 0, mi * sizeof(BatchState)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        excmg_batch_destroy(b);
        return EXCMG_ERR_OOM;
    }
    memset(b->h_states, 0, mi * sizeof(BatchState));
    if (cudaEventCreateWithFlags(&b->host_ready, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        excmg_batch_destroy(b);
        return EXCMG_ERR_CUDA;
    }
    for (int k = max_instances - 1; k >= 0; --k) b->free_slots.push_back(k);
    *out = b;
    return EXCMG_OK;
}

int excmg_batch_destroy(excmg_batch* b) {
    if (!b) return EXCMG_ERR_ARG;
    if (b->ctx) {
        if (b->ctx->stream) cudaStreamSynchronize(b->ctx->stream);
        else cudaDeviceSynchronize();
    }
    for (auto& g : b->groups) group_free(g);
    if (b->host_ready) cudaEventDestroy(b->host_ready);
    for (Instance* in : b->live) {
        free_instance(b, in);
        delete in;
    }
    for (Instance* in : b->finished) {
        free_instance(b, in);
        delete in;
    }
    cudaFree(b->d_states);
    cudaFreeHost(b->h_states);
    cudaFree(b->d_norms);
    cudaFreeHost(b->h_norms);
    cudaFree(b->d_bstate);
    cudaFreeHost(b->h_bstate);
    cudaFree(b->d_bpart);
    delete b;
    return EXCMG_OK;
}

const char* excmg_batch_last_error(const excmg_batch* b) { return b ? b->last_error.c_str() : ""; }

size_t excmg_batch_bytes(const excmg_batch* b) { return b ? b->bytes : 0; }

size_t excmg_batch_instance_bytes(int n_finest, int n_coarsest, int precision) {
    if (n_coarsest < 4 || n_finest < n_coarsest) return 0;
    return instance_bytes(n_finest, n_coarsest, precision);
}

int excmg_batch_submit(excmg_batch* b, int n_finest, int n_coarsest, int bc_kind, const double* f, const double* g1,
                       const double* g2, const excmg_params* params, double* u_out, int* id_out) {
    if (!b || !f || !g1 || !g2 || !params || !u_out || !id_out) return EXCMG_ERR_ARG;
    if (bc_kind != 1 && bc_kind != 2) return bfail(b, EXCMG_ERR_ARG, "bc_kind must be 1 or 2");
    if (n_coarsest < 4 || 2 * n_coarsest > 16)
        return bfail(b, EXCMG_ERR_ARG, "n_coarsest must be 4..8 (DSOLVE grids up to 16 intervals)");
    int steps = 0, n = n_coarsest;
    while (n < n_finest) {
        n *= 2;
        ++steps;
    }
    if (n != n_finest || steps < 2) return bfail(b, EXCMG_ERR_ARG, "n_finest must be n_coarsest * 2^(L+1), L >= 1");
    // the per-slot partial sums hold one value per CTA of an operator launch
    if (stencil_cta_count(n_finest) > kMaxPartials)
        return bfail(b, EXCMG_ERR_ARG, "n_finest too large for the batch engine's per-instance partial sums");
    if (params->precision != EXCMG_PRECISION_FP64 && params->precision != EXCMG_PRECISION_MIXED)
        return bfail(b, EXCMG_ERR_ARG, "unknown precision");
    if (!(params->tol > 0.0) || params->max_iter < 1 || params->max_total < 1 ||
        (params->precision == EXCMG_PRECISION_MIXED && !(params->inner_tol > 0.0 && params->inner_tol < 1.0)))
        return bfail(b, EXCMG_ERR_ARG, "bad parameters");
    const int prec = params->precision;
    const size_t need = instance_bytes(n_finest, n_coarsest, prec);
    if (b->budget && need > b->budget)
        return bfail(b, EXCMG_ERR_TOO_LARGE, "the instance needs more device memory than the batch's whole budget");
    if (b->free_slots.empty()) return bfail(b, EXCMG_ERR_BUDGET, "all instance slots are busy");
    if (b->budget && b->bytes + need > b->budget)
        return bfail(b, EXCMG_ERR_BUDGET, "device-memory budget of the batch is full");
    Instance* in = new (std::nothrow) Instance();
    if (!in) return EXCMG_ERR_OOM;
    if (cudaMalloc(&in->block, need) != cudaSuccess) {
        cudaGetLastError();
        delete in;
        return bfail(b, EXCMG_ERR_OOM, "cudaMalloc of an instance failed");
    }
    // boundary entries of every work vector must read zero (the operator
    // writes interior entries only)
    if (cudaMemsetAsync(in->block, 0, need, b->ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(in->block);
        delete in;
        return bfail(b, EXCMG_ERR_CUDA, "clearing an instance failed");
    }
    in->bytes = need;
    b->bytes += need;
    in->id = b->next_id++;
    in->n = n_finest;
    in->nc = n_coarsest;
    in->bc = bc_kind;
    in->nl = steps + 1;
    in->L = in->nl - 2;
    in->prec = prec;
    in->f = f;
    in->g1 = g1;
    in->g2 = g2;
    in->u_out = u_out;
    in->tol = params->tol;
    in->inner_tol = params->inner_tol;
    in->tol_mode = params->tol_mode;
    in->max_iter = params->max_iter;
    in->max_total = params->max_total;
    char* c = (char*)in->block;
    auto take = [&](size_t bytes) {
        char* r = c;
        c += align256(bytes);
        return (void*)r;
    };
    for (int l = 0; l < in->nl; ++l) in->u.push_back((double*)take(node_count(n_coarsest << l) * sizeof(double)));
    const size_t n64 = node_count(n_finest) * sizeof(double), n32 = node_count(n_finest) * sizeof(float);
    in->fh = (double*)take(n64);
    in->res = (double*)take(n64);
    in->W = (double*)take(node_count(n_finest / 2) * sizeof(double));
    if (prec == EXCMG_PRECISION_FP64) {
        in->rs64 = (double*)take(n64);
        in->p64 = (double*)take(n64);
        in->ps64 = (double*)take(n64);
        in->q64 = (double*)take(n64);
        in->qs64 = (double*)take(n64);
        in->p2_64 = (double*)take(n64);
        in->ps2_64 = (double*)take(n64);
    } else {
        in->r32 = (float*)take(n32);
        in->e = (float*)take(n32);
        in->r = (float*)take(n32);
        in->rs = (float*)take(n32);
        in->p = (float*)take(n32);
        in->ps = (float*)take(n32);
        in->q = (float*)take(n32);
        in->qs = (float*)take(n32);
    }
    in->stats.levels = in->nl;
    in->t_submit = now_s();
    in->slot = b->free_slots.back();
    b->free_slots.pop_back();
    b->live.push_back(in);
    b->h_states[in->slot] = BatchState{};
    b->h_states[in->slot].done = 1;   // no Bi-CG call yet
    *id_out = in->id;
    return EXCMG_OK;
}

// Advance the live instances: take back every group launch that has
// completed, run the per-instance steps of every instance not on the GPU
// (level set-up, direct solves, FP64 true residuals and the decisions of
// Alg. 1 they drive), start one cooperative launch per level group of
// instances ready for Bi-CG iterations (instances of one precision at one
// grid size, each group on its own stream), then wait for at least one
// running group.  *n_live receives the number of instances still running.
int excmg_batch_step(excmg_batch* b, int* n_live) {
    if (!b) return EXCMG_ERR_ARG;
    const double t_enter = now_s();
    excmg_ctx* ctx = b->ctx;
    cudaStream_t s = ctx->stream;
    int st = EXCMG_OK;
    // 0. completed group launches
    for (auto& g : b->groups)
        if (g.busy && cudaEventQuery(g.done) == cudaSuccess)
            if ((st = harvest(b, g))) return st;
    cudaGetLastError();   // cudaErrorNotReady of the queries
    // 1. setup phases (the direct-solve levels run straight through)
    for (Instance* in : b->live) {
        if (in->in_flight) continue;
        while (in->phase == kSetup) {
            if ((st = setup_level(b, in))) {
                in->phase = kFailed;
                in->status = st;
                break;
            }
            if (in->level <= 1) {
                in->stats.n[in->level] = in->nc << in->level;
                ++in->level;
                continue;
            }
            in->phase = kResidual;
            in->iters = in->outer = in->bad = in->stag = 0;
            in->rel = in->prev = 0.0;
            in->fnorm = -1.0;   // formed with the first residual
        }
    }
    // 2. FP64 true residuals (Alg. 1's true-residual test) and the decisions they drive
    std::vector<Instance*> res;
    for (Instance* in : b->live)
        if (!in->in_flight && in->phase == kResidual) res.push_back(in);
    if (!res.empty()) {
        std::vector<std::pair<Instance*, const double*>> need_f;
        for (Instance* in : res)
            if (in->fnorm < 0.0) need_f.push_back({in, in->fh});
        if ((st = norms(b, need_f))) return st;
        for (size_t k = 0; k < need_f.size(); ++k) need_f[k].first->fnorm = std::sqrt(b->h_norms[k]);
        std::vector<std::pair<Instance*, const double*>> rw;
        for (Instance* in : res) {
            const int N = in->nc << in->level;
            cudaError_t e = cudaMemsetAsync(in->res, 0, node_count(N) * sizeof(double), s);
            if (e == cudaSuccess)
                e = launch_stencil(in->u[in->level], in->res, in->fh, N, in->bc, false, nullptr, s, kStencilExact);
            bnote(b, 1);
            if (e != cudaSuccess) return bcuda(b, e, "batch residual");
            rw.push_back({in, in->res});
        }
        if ((st = norms(b, rw))) return st;
        for (size_t k = 0; k < rw.size(); ++k) {
            Instance* in = rw[k].first;
            const double rn = std::sqrt(b->h_norms[k]);
            const int l = in->level, N = in->nc << l;
            in->prev = in->rel;
            in->rel = in->fnorm > 0.0 ? rn / in->fnorm : 0.0;
            if (!std::isfinite(in->rel)) {
                in->phase = kFailed;
                in->status = EXCMG_ERR_NAN;
                continue;
            }
            bool level_done = false;
            if (in->outer > 0) {
                // FP64: the rule of the single solver (two calls without halving
                // the residual); mixed: two steps that remove less than a tenth
                const double keep = in->prec == EXCMG_PRECISION_FP64 ? 0.5 : 0.9;
                if (in->rel > keep * in->prev) {
                    if (++in->bad >= 2) {
                        in->stag = 1;
                        level_done = true;
                    }
                } else {
                    in->bad = 0;
                }
            }
            if (in->rel <= level_eps(in, l) || in->iters >= in->max_total || rn == 0.0) level_done = true;
            if (level_done) {
                in->stats.n[l] = N;
                in->stats.iters[l] = in->iters;
                in->stats.calls[l] = in->outer;
                in->stats.stagnated[l] = in->stag;
                in->stats.relres[l] = in->rel;
                if (l + 1 < in->nl) {
                    ++in->level;
                    in->phase = kSetup;
                } else {
                    in->phase = kFinal;
                }
                continue;
            }
            const int slot = in->slot;
            int cap = in->max_total - in->iters;
            if (cap > in->max_iter) cap = in->max_iter;
            cudaError_t e = cudaSuccess;
            if (in->prec == EXCMG_PRECISION_FP64) {
                // a Bi-CG call of Alg. 1's WHILE loop: x = u, r_0 = the true
                // residual just formed, r*_0 = p_0 = p*_0 = r_0,
                // rho_0 = (r_0, r_0); stop at ||r|| <= eps ||f_h||
                const size_t bytes = node_count(N) * sizeof(double);
                e = cudaMemcpyAsync(in->rs64, in->res, bytes, cudaMemcpyDeviceToDevice, s);
                if (e == cudaSuccess) e = cudaMemcpyAsync(in->p64, in->res, bytes, cudaMemcpyDeviceToDevice, s);
                if (e == cudaSuccess) e = cudaMemcpyAsync(in->ps64, in->res, bytes, cudaMemcpyDeviceToDevice, s);
                BatchState& hs = b->h_states[slot];
                hs = BatchState{};
                hs.rho = b->h_norms[k];   // (r_0, r_0) exactly as summed
                hs.rr = b->h_norms[k];
                hs.tol = level_eps(in, l) * in->fnorm;
                hs.max_iter = cap;
                hs.done = 0;
                hs.status = kRunning;
                // h_states is pinned: the slot's state is not touched again
                // before its group launch has completed
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(b->d_states + slot, b->h_states + slot, sizeof(BatchState),
                                        cudaMemcpyHostToDevice, s);
                if (launched_level(in)) {
                    // the same call in the single solver's state layout
                    BicgState& bs = b->h_bstate[slot];
                    bs = BicgState{};
                    bs.rho = b->h_norms[k];
                    bs.rr = b->h_norms[k];
                    bs.bnorm = in->fnorm;
                    bs.tol = level_eps(in, l);
                    bs.max_iter = cap;
                    bs.status = kRunning;
                    in->launched_k = 0;
                    in->dir_in_p2 = false;
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(b->d_bstate + slot, b->h_bstate + slot, sizeof(BicgState),
                                            cudaMemcpyHostToDevice, s);
                }
            } else {
                // FP32 correction solve on A e = r / ||r||
                in->scale = rn;
                batch_init32_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(in->res, 1.0 / rn, in->r32, in->e, in->rs,
                                                                       in->p, in->ps, node_count(N), ctx->partials,
                                                                       ctx->ticket, b->d_states + slot,
                                                                       in->inner_tol, cap);
                bnote(b, 1);
                e = cudaGetLastError();
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(in->r, in->r32, node_count(N) * sizeof(float), cudaMemcpyDeviceToDevice, s);
            }
            if (e != cudaSuccess) return bcuda(b, e, "Bi-CG call setup");
            in->phase = kInner;
            in->call_iter = 0;
        }
    }
    // 3. one cooperative launch per level group of instances waiting for
    // Bi-CG iterations, largest groups first, within the device's
    // co-resident capacity (so that concurrent groups never wait on each
    // other's CTAs)
    std::map<std::pair<int, int>, std::vector<Instance*>> ready;
    for (Instance* in : b->live)
        if (!in->in_flight && in->phase == kInner) ready[{in->prec, in->nc << in->level}].push_back(in);
    if (!ready.empty()) {
        cudaError_t e = cudaEventRecord(b->host_ready, s);
        if (e != cudaSuccess) return bcuda(b, e, "batch event");
        std::vector<std::pair<long long, std::pair<int, int>>> order;
        for (auto& kv : ready)
            order.push_back({-(long long)kv.second.size() * node_count(kv.first.second), kv.first});
        std::sort(order.begin(), order.end());
        for (auto& o : order) {
            const auto key = o.second;
            std::vector<Instance*>& list = ready[key];
            auto free_group = [&]() -> excmg_batch::Group& {
                for (auto& g : b->groups)
                    if (!g.busy) return g;
                b->groups.emplace_back();
                return b->groups.back();
            };
            if (launched_level(list[0])) {
                if ((st = launch_group_launched(b, free_group(), list))) return st;
                continue;
            }
            int used = 0;
            for (auto& g : b->groups)
                if (g.busy && g.prec == key.first) used += g.ctas;
            // groups of the other precision run another kernel: count them too
            for (auto& g : b->groups)
                if (g.busy && g.prec != key.first) used += g.ctas;
            const int cap = capacity_of(key.first) - used;
            if (cap < 1) continue;
            int cand = -1, units = 0, chunks = 0;
            geometry<double>(list[0], 0, &units, &chunks);
            int ctas = group_ctas(b, key.first, key.second, units > chunks ? units : chunks, (int)list.size(), &cand);
            if (ctas > cap) {
                ctas = cap;
                cand = -1;   // not the candidate's shape: not a tuning sample
            }
            excmg_batch::Group* slot = &free_group();
            st = key.first == EXCMG_PRECISION_FP64 ? launch_group<double>(b, *slot, list, ctas, cand)
                                                   : launch_group<float>(b, *slot, list, ctas, cand);
            if (st) return st;
        }
    }
    // 4. finals (EXP_true)
    bool any_final = false;
    for (Instance* in : b->live)
        if (in->phase == kFinal) {
            if ((st = finish(b, in))) return st;
            any_final = true;
        }
    if (any_final) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return bcuda(b, e, "batch finals");
    }
    const double t = now_s();
    std::vector<Instance*> keep;
    for (Instance* in : b->live) {
        if (in->phase == kFinal || in->phase == kFailed) {
            if (in->phase == kFinal) in->phase = kDone;
            in->t_done = t;
            free_instance(b, in);
            b->free_slots.push_back(in->slot);
            b->finished.push_back(in);
        } else {
            keep.push_back(in);
        }
    }
    b->live = keep;
    // 5. wait for one running group (the next step takes it back) unless
    // some instance can move on without the GPU
    bool host_work = false;
    for (Instance* in : b->live)
        if (!in->in_flight && (in->phase == kSetup || in->phase == kResidual)) host_work = true;
    bool any_busy = false;
    for (auto& g : b->groups) any_busy = any_busy || g.busy;
    const double t_wait = now_s();
    b->prof.host_s += t_wait - t_enter;
    if (any_busy && !host_work) {
        for (;;) {
            bool one = false;
            for (auto& g : b->groups)
                if (g.busy && cudaEventQuery(g.done) == cudaSuccess) one = true;
            cudaGetLastError();
            if (one) break;
            std::this_thread::yield();
        }
    }
    b->prof.wait_s += now_s() - t_wait;
    if (n_live) *n_live = (int)b->live.size();
    return EXCMG_OK;
}

// Status of instance `id`: *done = 1 when finished (status in *status),
// stats (may be NULL) per level, *latency_s the time from submit to finish.
int excmg_batch_query(excmg_batch* b, int id, int* done, int* status, excmg_stats* stats, double* latency_s) {
    if (!b || !done) return EXCMG_ERR_ARG;
    for (Instance* in : b->finished)
        if (in->id == id) {
            *done = 1;
            if (status) *status = in->phase == kDone ? EXCMG_OK : in->status;
            if (stats) *stats = in->stats;
            if (latency_s) *latency_s = in->t_done - in->t_submit;
            return EXCMG_OK;
        }
    for (Instance* in : b->live)
        if (in->id == id) {
            *done = 0;
            if (status) *status = EXCMG_OK;
            return EXCMG_OK;
        }
    return bfail(b, EXCMG_ERR_ARG, "unknown instance id");
}

long long excmg_batch_launches(const excmg_batch* b) { return b ? b->launches : 0; }

int excmg_batch_get_profile(const excmg_batch* b, excmg_batch_profile* out) {
    if (!b || !out) return EXCMG_ERR_ARG;
    *out = b->prof;
    return EXCMG_OK;
}

}  // extern "C"
