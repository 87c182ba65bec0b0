// C ABI of the library (include/excmg.h): contexts, levels, the operator,
// Bi-CG, the two level transfers and the EXCMG cascade of Alg. 1.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include "excmg_internal.cuh"

using namespace excmg;

namespace excmg {

static std::atomic<long long> g_launches{0};
void note_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

namespace {
std::mutex g_dev_mu;
std::map<int, int> g_sms;
std::map<std::tuple<const void*, int, int, size_t>, int> g_occ;
}  // namespace

int device_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    std::lock_guard<std::mutex> lock(g_dev_mu);
    auto it = g_sms.find(dev);
    if (it != g_sms.end()) return it->second;
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
        cudaGetLastError();
        return 1;   // not cached: the next call asks again
    }
    g_sms[dev] = v;
    return v;
}

int kernel_occupancy(const void* kernel, int threads, size_t smem) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    const auto key = std::make_tuple(kernel, dev, threads, smem);
    std::lock_guard<std::mutex> lock(g_dev_mu);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) return it->second;
    // (static + dynamic shared memory above 48 KB needs the opt-in, so it is
    // made whenever dynamic shared memory is asked for)
    if (smem > 0 &&
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;   // not cached; the launch reports the error
    }
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    if (v < 1) v = 1;
    g_occ[key] = v;
    return v;
}

int ctx_fail(excmg_ctx* ctx, int status, const std::string& msg) {
    if (ctx) ctx->last_error = msg;
    return status;
}

int ctx_cuda(excmg_ctx* ctx, cudaError_t err, const char* what) {
    if (err == cudaSuccess) return EXCMG_OK;
    cudaGetLastError();
    return ctx_fail(ctx, EXCMG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(err));
}

cudaGraphExec_t ctx_chunk_graph(excmg_ctx* ctx, const std::vector<uintptr_t>& key) {
    auto it = ctx->chunk_graphs.find(key);
    return it == ctx->chunk_graphs.end() ? nullptr : it->second;
}

void ctx_store_chunk_graph(excmg_ctx* ctx, const std::vector<uintptr_t>& key, cudaGraphExec_t exec) {
    if (ctx->chunk_graphs.size() >= 64) {   // bounded: drop the old ones (buffers may have moved)
        cudaStreamSynchronize(ctx->stream);
        for (auto& kv : ctx->chunk_graphs) cudaGraphExecDestroy(kv.second);
        ctx->chunk_graphs.clear();
    }
    ctx->chunk_graphs[key] = exec;
}

cudaStream_t ctx_capture_stream(excmg_ctx* ctx) {
    if (!ctx->capture_stream && cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
        ctx->capture_stream = nullptr;
    return ctx->capture_stream;
}

// A named workspace buffer of at least `bytes`, grown on demand.
namespace {
// One warp copies `words` 8-byte words from device memory into mapped host
// memory (stores over the host link, visible to the host once the stream
// has been synchronised).
__global__ void read_back_kernel(const unsigned long long* __restrict__ src, unsigned long long* dst, int words) {
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}
}  // namespace

cudaError_t ctx_read_back(excmg_ctx* ctx, void* host_mirror, const void* dev_src, size_t bytes) {
    void* dst = nullptr;
    if (host_mirror == ctx->host_state) dst = ctx->host_state_dev;
    else if (host_mirror == ctx->host_scalar) dst = ctx->host_scalar_dev;
    if (!dst || bytes % 8 != 0) return cudaErrorInvalidValue;
    read_back_kernel<<<1, 32, 0, ctx->stream>>>((const unsigned long long*)dev_src, (unsigned long long*)dst,
                                                (int)(bytes / 8));
    note_launches(1);
    return cudaGetLastError();
}

double* ctx_buffer(excmg_ctx* ctx, const char* name, size_t bytes, int* status) {
    excmg_buffer& b = ctx->buffers[name];
    if (b.bytes >= bytes && b.ptr) return (double*)b.ptr;
    const size_t held = b.bytes;
    if (ctx->budget && ctx->bytes - held + bytes > ctx->budget) {
        *status = ctx_fail(ctx, EXCMG_ERR_BUDGET, std::string("HBM budget too small for buffer ") + name);
        return nullptr;
    }
    if (b.ptr) {
        cudaFree(b.ptr);
        ctx->bytes -= held;
        b.ptr = nullptr;
        b.bytes = 0;
    }
    if (cudaMalloc(&b.ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        b.ptr = nullptr;
        *status = ctx_fail(ctx, EXCMG_ERR_OOM, std::string("cudaMalloc failed for buffer ") + name);
        return nullptr;
    }
    b.bytes = bytes;
    ctx->bytes += bytes;
    return (double*)b.ptr;
}

}  // namespace excmg

namespace {

std::mutex g_default_mu;
excmg_ctx* g_default[64] = {};

excmg_ctx* default_ctx() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(g_default_mu);
    if (!g_default[dev]) {
        excmg_ctx* c = nullptr;
        if (excmg_ctx_create(nullptr, 0, &c) != EXCMG_OK) return nullptr;
        g_default[dev] = c;
    }
    return g_default[dev];
}

bool is_pow2_multiple(int fine, int coarse, int* steps) {
    if (coarse <= 0 || fine < coarse) return false;
    int s = 0, n = coarse;
    while (n < fine) {
        n *= 2;
        ++s;
    }
    *steps = s;
    return n == fine;
}

}  // namespace

extern "C" {

int excmg_ctx_create(void* cuda_stream, size_t hbm_budget_bytes, excmg_ctx** out) {
    if (!out) return EXCMG_ERR_ARG;
    *out = nullptr;
    excmg_ctx* c = new (std::nothrow) excmg_ctx();
    if (!c) return EXCMG_ERR_OOM;
    c->stream = (cudaStream_t)cuda_stream;
    c->budget = hbm_budget_bytes;
    cudaGetDevice(&c->device);
    bool ok = cudaMalloc(&c->partials, kMaxPartials * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&c->ticket, sizeof(unsigned int)) == cudaSuccess &&
              cudaMalloc(&c->scalar, 8 * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&c->state, sizeof(BicgState)) == cudaSuccess &&
              cudaMalloc(&c->barrier, 4 * sizeof(unsigned int)) == cudaSuccess &&
              cudaMemset(c->barrier, 0, 4 * sizeof(unsigned int)) == cudaSuccess &&
              cudaHostAlloc(&c->host_state, sizeof(BicgState), cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc(&c->host_scalar, 8 * sizeof(double), cudaHostAllocMapped) == cudaSuccess &&
              cudaHostGetDevicePointer((void**)&c->host_state_dev, c->host_state, 0) == cudaSuccess &&
              cudaHostGetDevicePointer((void**)&c->host_scalar_dev, c->host_scalar, 0) == cudaSuccess &&
              cudaMemset(c->ticket, 0, sizeof(unsigned int)) == cudaSuccess &&
              cudaMemset(c->state, 0, sizeof(BicgState)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        excmg_ctx_destroy(c);
        return EXCMG_ERR_OOM;
    }
    *out = c;
    return EXCMG_OK;
}

int excmg_ctx_destroy(excmg_ctx* c) {
    if (!c) return EXCMG_ERR_ARG;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    for (auto& kv : c->buffers)
        if (kv.second.ptr) cudaFree(kv.second.ptr);
    for (auto& kv : c->inverses)
        if (kv.second.ptr) cudaFree(kv.second.ptr);
    if (c->partials) cudaFree(c->partials);
    if (c->ticket) cudaFree(c->ticket);
    if (c->scalar) cudaFree(c->scalar);
    if (c->state) cudaFree(c->state);
    if (c->barrier) cudaFree(c->barrier);
    if (c->host_state) cudaFreeHost(c->host_state);
    if (c->host_scalar) cudaFreeHost(c->host_scalar);
    for (cudaEvent_t e : c->prof_events) cudaEventDestroy(e);
    for (auto& kv : c->chunk_graphs) cudaGraphExecDestroy(kv.second);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    delete c;
    return EXCMG_OK;
}

size_t excmg_ctx_bytes(const excmg_ctx* c) { return c ? c->bytes : 0; }

int excmg_ctx_set_stencil(excmg_ctx* c, int variant) {
    if (!c) c = default_ctx();
    if (!c) return EXCMG_ERR_CUDA;
    if (variant != EXCMG_STENCIL_EXACT && variant != EXCMG_STENCIL_FP64)
        return ctx_fail(c, EXCMG_ERR_ARG, "unknown stencil variant");
    c->stencil_variant = variant == EXCMG_STENCIL_EXACT ? kStencilExact : kStencilFp64;
    return EXCMG_OK;
}

int excmg_ctx_set_shadow_mode(excmg_ctx* c, int mode) {
    if (!c) c = default_ctx();
    if (!c) return EXCMG_ERR_CUDA;
    if (mode != EXCMG_SHADOW_FULL && mode != EXCMG_SHADOW_ELIDED)
        return ctx_fail(c, EXCMG_ERR_ARG, "unknown shadow mode");
    c->shadow_mode = mode;
    return EXCMG_OK;
}

int excmg_ctx_set_schedule(excmg_ctx* c, int schedule) {
    if (!c) c = default_ctx();
    if (!c) return EXCMG_ERR_CUDA;
    if (schedule != EXCMG_SCHEDULE_SEPARATE && schedule != EXCMG_SCHEDULE_FUSED)
        return ctx_fail(c, EXCMG_ERR_ARG, "unknown operator schedule");
    c->schedule = schedule;
    return EXCMG_OK;
}

int excmg_ctx_set_graphs(excmg_ctx* c, int enable) {
    if (!c) c = default_ctx();
    if (!c) return EXCMG_ERR_CUDA;
    c->graphs = enable != 0;
    return EXCMG_OK;
}

long long excmg_launch_count(void) { return g_launches.load(); }

int excmg_ctx_profile(excmg_ctx* c, int enable) {
    if (!c) return EXCMG_ERR_ARG;
    c->profile = enable != 0;
    c->prof.clear();
    return EXCMG_OK;
}

int excmg_ctx_profile_read(const excmg_ctx* c, int n, double* ms_total, long long* launches, double* bytes) {
    if (!c || !ms_total || !launches) return EXCMG_ERR_ARG;
    auto it = c->prof.find(n);
    const bool have = it != c->prof.end();
    *ms_total = have ? it->second.ms : 0.0;
    *launches = have ? it->second.launches : 0;
    if (bytes) *bytes = have ? it->second.bytes : 0.0;
    return EXCMG_OK;
}

const char* excmg_last_error(const excmg_ctx* c) {
    if (!c) c = default_ctx();
    return c ? c->last_error.c_str() : "no CUDA device";
}

int excmg_level_create(excmg_ctx* ctx, int n, int bc_kind, excmg_level** out) {
    if (!out) return EXCMG_ERR_ARG;
    *out = nullptr;
    if (!ctx) ctx = default_ctx();
    if (!ctx) return EXCMG_ERR_CUDA;
    if (n < 4) return ctx_fail(ctx, EXCMG_ERR_ARG, "a level needs N >= 4");
    if (bc_kind != 1 && bc_kind != 2) return ctx_fail(ctx, EXCMG_ERR_ARG, "bc_kind must be 1 or 2");
    excmg_level* l = new (std::nothrow) excmg_level{ctx, n, bc_kind};
    if (!l) return EXCMG_ERR_OOM;
    *out = l;
    return EXCMG_OK;
}

int excmg_level_destroy(excmg_level* l) {
    if (!l) return EXCMG_ERR_ARG;
    delete l;
    return EXCMG_OK;
}

int stencil_apply(const excmg_level* level, int transpose, const double* u, double* y) {
    if (!level || !u || !y) return EXCMG_ERR_ARG;
    excmg_ctx* ctx = level->ctx;
    if (u == y) return ctx_fail(ctx, EXCMG_ERR_ARG, "stencil_apply: u and y must not overlap");
    cudaError_t e = launch_stencil(u, y, nullptr, level->n, level->bc_kind, transpose != 0, nullptr,
                                   ctx->stream, ctx->stencil_variant);
    if (e == cudaSuccess) e = launch_zero_boundary(y, level->n, ctx->stream);
    note_launches(2);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return ctx_cuda(ctx, e, "stencil_apply");
}

int bicg_solve(const excmg_level* level, const double* b, double* x_inout, double tol, int max_iter,
               int* iters_out, double* relres_out) {
    if (!level || !b || !x_inout) return EXCMG_ERR_ARG;
    excmg_ctx* ctx = level->ctx;
    if (!(tol >= 0.0) || max_iter < 0) return ctx_fail(ctx, EXCMG_ERR_ARG, "bicg_solve: bad tol / max_iter");
    double bnorm = 0.0;
    int st = unknowns_norm(ctx, level->n, b, &bnorm);
    if (st) return st;
    return bicg_run(ctx, level->n, level->bc_kind, b, x_inout, tol, bnorm, max_iter, 16, iters_out,
                    relres_out);
}

int bicg_solve_ex(const excmg_level* level, const double* b, double* x_inout, const double* shadow_r0, double tol,
                  int max_iter, int* iters_out, double* relres_out) {
    if (!level || !b || !x_inout) return EXCMG_ERR_ARG;
    excmg_ctx* ctx = level->ctx;
    if (!(tol >= 0.0) || max_iter < 0) return ctx_fail(ctx, EXCMG_ERR_ARG, "bicg_solve_ex: bad tol / max_iter");
    double bnorm = 0.0;
    int st = unknowns_norm(ctx, level->n, b, &bnorm);
    if (st) return st;
    return bicg_run(ctx, level->n, level->bc_kind, b, x_inout, tol, bnorm, max_iter, 16, iters_out, relres_out,
                    shadow_r0);
}

int extrapolate_interpolate_ex(excmg_ctx* ctx, int n_fine, const double* u_2h, const double* u_4h,
                               const double* g1_fine, double* w_h) {
    if (!ctx) ctx = default_ctx();
    if (!ctx) return EXCMG_ERR_CUDA;
    if (n_fine < 8 || n_fine % 4 || !u_2h || !u_4h || !w_h)
        return ctx_fail(ctx, EXCMG_ERR_ARG, "extrapolate_interpolate: n_fine must be a multiple of 4, >= 8");
    int st = EXCMG_OK;
    double* W = ctx_buffer(ctx, "exp_W", node_count(n_fine / 2) * sizeof(double), &st);
    if (st) return st;
    cudaError_t e = launch_exp_finite(w_h, u_2h, u_4h, W, n_fine, ctx->stream);
    note_launches(2);
    // Alg. 1: the boundary nodes of the next level carry the Dirichlet data
    if (e == cudaSuccess && g1_fine) {
        e = launch_set_boundary(w_h, n_fine, g1_fine, 1, ctx->stream);
        note_launches(1);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return ctx_cuda(ctx, e, "extrapolate_interpolate");
}

int extrapolate_interpolate(int n_fine, const double* u_2h, const double* u_4h, const double* g1_fine,
                            double* w_h) {
    return extrapolate_interpolate_ex(nullptr, n_fine, u_2h, u_4h, g1_fine, w_h);
}

int midpoint_extrapolate_ex(excmg_ctx* ctx, int n_fine, const double* u_h, const double* u_2h,
                            double* u_tilde) {
    if (!ctx) ctx = default_ctx();
    if (!ctx) return EXCMG_ERR_CUDA;
    if (n_fine < 4 || n_fine % 2 || !u_h || !u_2h || !u_tilde)
        return ctx_fail(ctx, EXCMG_ERR_ARG, "midpoint_extrapolate: n_fine must be even, >= 4");
    cudaError_t e = launch_exp_true(u_tilde, u_h, u_2h, n_fine, ctx->stream);
    note_launches(1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return ctx_cuda(ctx, e, "midpoint_extrapolate");
}

int midpoint_extrapolate(int n_fine, const double* u_h, const double* u_2h, double* u_tilde) {
    return midpoint_extrapolate_ex(nullptr, n_fine, u_h, u_2h, u_tilde);
}

int excmg_assemble_rhs(const excmg_level* level, int n_src, const double* f, const double* g1,
                       const double* g2, double* fh) {
    if (!level || !f || !g1 || !g2 || !fh) return EXCMG_ERR_ARG;
    excmg_ctx* ctx = level->ctx;
    if (n_src < level->n || n_src % level->n)
        return ctx_fail(ctx, EXCMG_ERR_ARG, "excmg_assemble_rhs: n_src must be a multiple of N");
    cudaError_t e = launch_assemble_rhs(fh, level->n, level->bc_kind, f, g1, g2, n_src / level->n,
                                        ctx->stream);
    note_launches(1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return ctx_cuda(ctx, e, "excmg_assemble_rhs");
}

int excmg_dsolve(const excmg_level* level, const double* fh, double* u) {
    if (!level || !fh || !u) return EXCMG_ERR_ARG;
    excmg_ctx* ctx = level->ctx;
    int st = dsolve_run(ctx, level->n, level->bc_kind, fh, u);
    if (st) return st;
    return ctx_cuda(ctx, cudaStreamSynchronize(ctx->stream), "excmg_dsolve");
}

int excmg_solve_ex(excmg_ctx* ctx, int n_finest, int n_coarsest, int bc_kind, const double* f,
                   const double* g1, const double* g2, const excmg_params* params, double* u_h_out,
                   double* u_tilde_out, excmg_stats* stats) {
    if (!ctx) ctx = default_ctx();
    if (!ctx) return EXCMG_ERR_CUDA;
    int steps = 0;
    if (!f || !g1 || !g2 || !params) return ctx_fail(ctx, EXCMG_ERR_ARG, "excmg_solve: null argument");
    if (bc_kind != 1 && bc_kind != 2) return ctx_fail(ctx, EXCMG_ERR_ARG, "bc_kind must be 1 or 2");
    if (n_coarsest < 4 || 2 * n_coarsest > 16)
        return ctx_fail(ctx, EXCMG_ERR_ARG, "n_coarsest must be 4..8 (DSOLVE grids up to 16 intervals)");
    if (!is_pow2_multiple(n_finest, n_coarsest, &steps) || steps < 2)
        return ctx_fail(ctx, EXCMG_ERR_ARG, "n_finest must be n_coarsest * 2^(L+1) with L >= 1");
    if (!(params->tol > 0.0) || params->max_iter < 1 || params->max_total < 1)
        return ctx_fail(ctx, EXCMG_ERR_ARG, "excmg_solve: tol > 0, max_iter >= 1, max_total >= 1");
    if (params->precision != EXCMG_PRECISION_FP64 && params->precision != EXCMG_PRECISION_MIXED)
        return ctx_fail(ctx, EXCMG_ERR_ARG, "excmg_solve: unknown precision");
    if (params->precision == EXCMG_PRECISION_MIXED && !(params->inner_tol > 0.0 && params->inner_tol < 1.0))
        return ctx_fail(ctx, EXCMG_ERR_ARG, "excmg_solve: inner_tol must lie in (0, 1)");
    const int nl = steps + 1;   // levels 0 .. L+1
    if (nl > EXCMG_MAX_LEVELS) return ctx_fail(ctx, EXCMG_ERR_ARG, "too many levels");
    const int L = nl - 2;
    cudaStream_t s = ctx->stream;
    int st = EXCMG_OK;
    double* lvl[EXCMG_MAX_LEVELS] = {};
    for (int l = 0; l < nl; ++l) {
        char name[32];
        snprintf(name, sizeof name, "level_u%d", l);
        lvl[l] = ctx_buffer(ctx, name, node_count(n_coarsest << l) * sizeof(double), &st);
        if (st) return st;
    }
    double* fh = ctx_buffer(ctx, "level_fh", node_count(n_finest) * sizeof(double), &st);
    if (st) return st;
    double* W = ctx_buffer(ctx, "exp_W", node_count(n_finest / 2) * sizeof(double), &st);
    if (st) return st;
    if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->levels = nl;
    }
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    int result = EXCMG_OK;
    for (int l = 0; l < nl && result == EXCMG_OK; ++l) {
        const int N = n_coarsest << l;
        const int stride = n_finest / N;
        double* u = lvl[l];
        int iters = 0, calls = 0, stag = 0, bad = 0;
        double fnorm = 0.0, rn = 0.0, rel = 0.0;
        cudaEventRecord(ev0, s);
        cudaError_t e = launch_assemble_rhs(fh, N, bc_kind, f, g1, g2, stride, s);
        if (e == cudaSuccess && l >= 2) e = launch_exp_finite(u, lvl[l - 1], lvl[l - 2], W, N, s);
        // the FD solution carries the Dirichlet data on the boundary (Sec. 2)
        if (e == cudaSuccess) e = launch_set_boundary(u, N, g1, stride, s);
        note_launches(l >= 2 ? 4 : 2);
        if (e != cudaSuccess) { result = ctx_cuda(ctx, e, "level setup"); break; }
        if ((result = interior_norm(ctx, N, fh, &fnorm))) break;
        if (!std::isfinite(fnorm)) {
            result = ctx_fail(ctx, EXCMG_ERR_NAN, "right-hand side f_h is not finite");
            break;
        }
        if (l <= 1) {
            // Alg. 1's direct solves
            if ((result = dsolve_run(ctx, N, bc_kind, fh, u))) break;
            if ((result = true_residual_norm(ctx, N, bc_kind, fh, u, &rn))) break;
            rel = fnorm > 0.0 ? rn / fnorm : 0.0;
            if (!std::isfinite(rel)) {
                result = ctx_fail(ctx, EXCMG_ERR_NAN, "residual of the direct solve is not finite");
                break;
            }
        } else {
            const int i = l - 1;   // Alg. 1 loop counter 1..L
            const double eps = params->tol_mode == EXCMG_TOL_PAPER ? params->tol * std::pow(10.0, (double)(i - L))
                                                                   : params->tol;
            if (params->precision == EXCMG_PRECISION_MIXED) {
                result = mixed_level_solve(ctx, N, bc_kind, fh, u, fnorm, eps, params->inner_tol, params->max_iter,
                                           params->max_total, params->check_every, &iters, &calls, &stag, &rel);
                if (result) break;
                goto level_done;
            }
            if ((result = true_residual_norm(ctx, N, bc_kind, fh, u, &rn))) break;
            rel = fnorm > 0.0 ? rn / fnorm : 0.0;
            if (!std::isfinite(rel)) {
                result = ctx_fail(ctx, EXCMG_ERR_NAN, "residual of the initial guess is not finite");
                break;
            }
            // Alg. 1's WHILE loop
            while (rel > eps && iters < params->max_total) {
                int it = 0;
                double rr = 0.0;
                const double prev = rel;
                int cap = params->max_total - iters;
                if (cap > params->max_iter) cap = params->max_iter;
                const int bs = bicg_run(ctx, N, bc_kind, fh, u, eps, fnorm, cap, params->check_every, &it, &rr);
                iters += it;
                ++calls;
                if (bs != EXCMG_OK && bs != EXCMG_ERR_NOCONV) { result = bs; break; }
                if ((result = true_residual_norm(ctx, N, bc_kind, fh, u, &rn))) break;
                rel = rn / fnorm;
                if (!std::isfinite(rel)) { result = ctx_fail(ctx, EXCMG_ERR_NAN, "residual is not finite"); break; }
                if (rel > 0.5 * prev) {
                    if (++bad >= 2) { stag = 1; break; }
                } else {
                    bad = 0;
                }
            }
        }
    level_done:
        cudaEventRecord(ev1, s);
        cudaEventSynchronize(ev1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        if (stats) {
            stats->n[l] = N;
            stats->iters[l] = iters;
            stats->calls[l] = calls;
            stats->stagnated[l] = stag;
            stats->relres[l] = rel;
            stats->ms[l] = ms;
        }
    }
    if (result == EXCMG_OK) {
        const size_t bytes = node_count(n_finest) * sizeof(double);
        cudaError_t e = cudaSuccess;
        if (u_h_out) e = cudaMemcpyAsync(u_h_out, lvl[nl - 1], bytes, cudaMemcpyDeviceToDevice, s);
        // Alg. 1's final extrapolation
        if (e == cudaSuccess && u_tilde_out) {
            e = launch_exp_true(u_tilde_out, lvl[nl - 1], lvl[nl - 2], n_finest, s);
            note_launches(1);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        result = ctx_cuda(ctx, e, "excmg_solve output");
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    return result;
}

int excmg_solve(int n_finest, int n_coarsest, int bc_kind, const double* f, const double* g1,
                const double* g2, double tol, double* u_out) {
    excmg_params p;
    p.tol = tol;
    p.tol_mode = EXCMG_TOL_UNIFORM;
    p.max_iter = 100000;
    p.max_total = 1000000;
    p.check_every = 16;
    p.precision = EXCMG_PRECISION_FP64;
    p.inner_tol = 1e-4;
    if (!u_out) return EXCMG_ERR_ARG;
    return excmg_solve_ex(nullptr, n_finest, n_coarsest, bc_kind, f, g1, g2, &p, nullptr, u_out, nullptr);
}

}  // extern "C"
