// Host side of Bi-CG (Alg. 2, M = I, r*_0 = r_0): every iteration is a fixed
// sequence of kernels that read alpha, beta and the stopping flag from the
// device-resident BicgState, so iterations are enqueued in batches and the
// host only looks at the state between batches.
#include <cmath>
#include <utility>
#include <vector>

#include "excmg_internal.cuh"

namespace excmg {

int interior_norm(excmg_ctx* ctx, int n, const double* a, double* out) {
    const size_t len = node_count(n);
    cudaError_t e = launch_dot(a, a, len, ctx->partials, ctx->ticket, ctx->scalar, ctx->stream);
    note_launches(1);
    if (e == cudaSuccess)
        e = ctx_read_back(ctx, ctx->host_scalar, ctx->scalar, sizeof(double));
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "norm");
    *out = sqrt(*ctx->host_scalar);
    return EXCMG_OK;
}

// ||a||_2 over the unknowns only, for vectors from a caller (their boundary
// entries are not part of the system and may hold anything).
int unknowns_norm(excmg_ctx* ctx, int n, const double* a, double* out) {
    cudaError_t e = launch_interior_dot(a, n, ctx->partials, ctx->ticket, ctx->scalar, ctx->stream);
    note_launches(1);
    if (e == cudaSuccess)
        e = ctx_read_back(ctx, ctx->host_scalar, ctx->scalar, sizeof(double));
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "norm");
    *out = sqrt(*ctx->host_scalar);
    return EXCMG_OK;
}

// Norm of b - A x over the unknowns (boundary entries of the work vector are
// zero, so a flat norm over all nodes equals it).
int true_residual_norm(excmg_ctx* ctx, int n, int bc_kind, const double* b, const double* x,
                       double* out) {
    const size_t len = node_count(n);
    int st = EXCMG_OK;
    double* r = ctx_buffer(ctx, "res", len * sizeof(double), &st);
    if (st) return st;
    cudaError_t e = cudaMemsetAsync(r, 0, len * sizeof(double), ctx->stream);
    if (e == cudaSuccess) e = launch_stencil(x, r, b, n, bc_kind, false, nullptr, ctx->stream, ctx->stencil_variant);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "residual");
    note_launches(1);
    return interior_norm(ctx, n, r, out);
}

int bicg_run(excmg_ctx* ctx, int n, int bc_kind, const double* b, double* x, double tol,
             double bnorm, int max_iter, int check_every, int* iters_out, double* relres_out,
             const double* shadow) {
    const size_t len = node_count(n);
    const size_t bytes = len * sizeof(double);
    int st = EXCMG_OK;
    // shadow-elided mode (a labelled variant, not Alg. 2 as printed): with
    // r*_0 = r_0 and the integer operator the shadow vectors are the primal
    // ones bit for bit, so they are neither stored nor read
    const bool elide =
        ctx->shadow_mode == EXCMG_SHADOW_ELIDED && shadow == nullptr && ctx->stencil_variant == kStencilExact;
    double* r = ctx_buffer(ctx, "bicg_r", bytes, &st);
    double* rs = (st || elide) ? nullptr : ctx_buffer(ctx, "bicg_rs", bytes, &st);
    double* p = st ? nullptr : ctx_buffer(ctx, "bicg_p", bytes, &st);
    double* ps = (st || elide) ? nullptr : ctx_buffer(ctx, "bicg_ps", bytes, &st);
    double* q = st ? nullptr : ctx_buffer(ctx, "bicg_q", bytes, &st);
    double* qs = (st || elide) ? nullptr : ctx_buffer(ctx, "bicg_qs", bytes, &st);
    if (st) return st;
    // the integer operator has a fused two-field kernel; the FP64 one runs
    // as two applications and a separate inner product
    const bool fused = ctx->stencil_variant == kStencilExact && stencil_cta_count(n) <= kMaxPartials;
    // small grids run whole iterations in one cooperative launch
    const bool persistent = fused && n <= kPersistentMaxN;
    // the fused schedule (the default on the launched levels) folds
    // p = r + beta p into the operator step, which reads the previous
    // directions from one buffer pair and writes the new ones to the other
    // (neighbouring blocks still read the old values); the cooperative
    // kernel of the small grids keeps a separate direction-update phase
    const bool fuse = ctx->schedule == EXCMG_SCHEDULE_FUSED;
    const bool dir_fused = fused && fuse && !persistent;
    double* p2 = dir_fused ? ctx_buffer(ctx, "bicg_p2", bytes, &st) : nullptr;
    double* ps2 = (dir_fused && !elide && !st) ? ctx_buffer(ctx, "bicg_ps2", bytes, &st) : nullptr;
    if (st) return st;
    cudaStream_t s = ctx->stream;
    if (check_every < 1) check_every = 1;

    BicgState init{};
    init.bnorm = bnorm;
    init.tol = tol;
    init.max_iter = max_iter;
    *ctx->host_state = init;
    cudaError_t e = cudaMemcpyAsync(ctx->state, ctx->host_state, sizeof(BicgState), cudaMemcpyHostToDevice, s);
    // boundary entries of every work vector stay zero: the stencils write
    // interior entries only
    if (e == cudaSuccess) e = cudaMemsetAsync(r, 0, bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(q, 0, bytes, s);
    if (e == cudaSuccess && !elide) e = cudaMemsetAsync(qs, 0, bytes, s);
    // r_0 = b - A x_0; r*_0 = p_0 = p*_0 = r_0; rho_0
    if (e == cudaSuccess) e = launch_stencil(x, r, b, n, bc_kind, false, nullptr, s, ctx->stencil_variant);
    if (e == cudaSuccess)
        e = elide ? launch_cg_init(r, p, len, ctx->partials, ctx->state, s)
                  : launch_bicg_init(r, shadow, rs, p, ps, len, ctx->partials, ctx->state, s);
    // a caller's shadow may carry values on boundary nodes: the work vectors
    // keep zeros there
    if (e == cudaSuccess && shadow) e = launch_zero_boundary(rs, n, s);
    if (e == cudaSuccess && shadow) e = launch_zero_boundary(ps, n, s);
    if (e == cudaSuccess && dir_fused) e = launch_zero_boundary(p2, n, s);
    if (e == cudaSuccess && dir_fused && !elide) e = launch_zero_boundary(ps2, n, s);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "Bi-CG setup");
    note_launches(dir_fused ? (elide ? 1 : 2) : 0);

    const int* done = &ctx->state->done;
    if (persistent) {
        for (;;) {
            e = ctx_read_back(ctx, ctx->host_state, ctx->state, sizeof(BicgState));
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return ctx_cuda(ctx, e, "Bi-CG state read");
            if (ctx->host_state->done) break;
            int chunk = 256;
            const int left = max_iter - ctx->host_state->iter;
            if (chunk > left) chunk = left;
            e = launch_bicg_persistent(x, r, rs, p, ps, q, qs, n, bc_kind, chunk, ctx->partials, ctx->state,
                                       ctx->barrier, s, elide);
            note_launches(1);
            if (e != cudaSuccess) return ctx_cuda(ctx, e, "cooperative Bi-CG launch");
        }
    }
    note_launches(2);   // residual stencil + init (the memsets are not kernels)
    int batch = 0;
    int iter_before = 0;
    // algorithmic bytes of one timed operator launch: 8 B per unknown for
    // each field read or written
    const double unknowns = (double)(n - 1) * (n - 1) * (n - 1);
    std::vector<double> launch_bytes;
    long long enqueued = 0;    // iterations enqueued so far
    double* pc = p;            // directions of the current iteration
    double* psc = ps;
    double* pn = p2;           // buffer pair the next directions go to
    double* psn = ps2;
    for (; !persistent;) {
        e = ctx_read_back(ctx, ctx->host_state, ctx->state, sizeof(BicgState));
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return ctx_cuda(ctx, e, "Bi-CG state read");
        if (ctx->profile && batch > 0) {
            // credit only the iterations of the last batch that really ran
            const int ran = ctx->host_state->iter - iter_before;
            ProfRecord& rec = ctx->prof[n];
            for (int it = 0; it < ran && it < batch; ++it) {
                float a = 0.f, b2 = 0.f;
                cudaEventElapsedTime(&a, ctx->prof_events[3 * it], ctx->prof_events[3 * it + 1]);
                cudaEventElapsedTime(&b2, ctx->prof_events[3 * it + 1], ctx->prof_events[3 * it + 2]);
                rec.ms += (double)a + (double)b2;
                rec.launches += fused ? 1 : 2;
                rec.bytes += launch_bytes[it];
            }
        }
        if (ctx->host_state->done) break;
        iter_before = ctx->host_state->iter;
        batch = check_every;
        const int left = max_iter - ctx->host_state->iter;
        if (batch > left) batch = left;
        if (ctx->profile) {
            while ((int)ctx->prof_events.size() < 3 * batch) {
                cudaEvent_t ev;
                if (cudaEventCreate(&ev) != cudaSuccess) return ctx_cuda(ctx, cudaGetLastError(), "event");
                ctx->prof_events.push_back(ev);
            }
        }
        launch_bytes.assign(batch, 0.0);
        // the iterations of one batch, enqueued on stream `ss`
        auto enqueue = [&](cudaStream_t ss) -> cudaError_t {
            cudaError_t ee = cudaSuccess;
            for (int it = 0; it < batch && ee == cudaSuccess; ++it) {
                if (ctx->profile) cudaEventRecord(ctx->prof_events[3 * it], ss);
                if (fused) {
                    // A p_k and A^T p*_k in one z-march, sigma_k and alpha_k fused;
                    // from the second iteration on the launch first forms
                    // p_k = r_k + beta_{k-1} p_{k-1} (and p*_k) on the fly
                    if (enqueued == 0 || !dir_fused) {
                        ee = elide ? launch_cg_stencil(pc, q, n, bc_kind, ctx->partials, ctx->state, ss, dir_fused)
                                   : launch_bicg_stencil_pair(pc, q, psc, qs, n, bc_kind, ctx->partials, ctx->state,
                                                              ss, dir_fused);
                        // p (, p*) in; q (, q*) out
                        launch_bytes[it] = (elide ? 16.0 : 32.0) * unknowns;
                    } else {
                        ee = elide ? launch_cg_stencil_dir(r, pc, pn, q, n, bc_kind, ctx->partials, ctx->state, ss)
                                   : launch_bicg_stencil_pair_dir(r, rs, pc, psc, pn, psn, q, qs, n, bc_kind,
                                                                  ctx->partials, ctx->state, ss);
                        std::swap(pc, pn);
                        std::swap(psc, psn);
                        // r (, r*), p_old (, p*_old) in; p (, p*), q (, q*) out
                        launch_bytes[it] = (elide ? 32.0 : 64.0) * unknowns;
                    }
                    if (ctx->profile) {
                        cudaEventRecord(ctx->prof_events[3 * it + 1], ss);
                        cudaEventRecord(ctx->prof_events[3 * it + 2], ss);
                    }
                } else {
                    launch_bytes[it] = 32.0 * unknowns;       // two launches of u in, y out
                    ee = launch_stencil(p, q, nullptr, n, bc_kind, false, done, ss, ctx->stencil_variant);  // A p_k
                    if (ctx->profile) cudaEventRecord(ctx->prof_events[3 * it + 1], ss);
                    if (ee == cudaSuccess)
                        ee = launch_stencil(ps, qs, nullptr, n, bc_kind, true, done, ss,
                                            ctx->stencil_variant);  // A^T p*_k
                    if (ctx->profile) cudaEventRecord(ctx->prof_events[3 * it + 2], ss);
                    if (ee == cudaSuccess) ee = launch_bicg_sigma(ps, q, len, ctx->partials, ctx->state, ss);
                }
                if (ee == cudaSuccess)
                    ee = elide ? launch_cg_update(x, pc, r, q, len, ctx->partials, ctx->state, ss)
                               : launch_bicg_update(x, pc, r, q, rs, qs, len, ctx->partials, ctx->state, ss);
                if (ee == cudaSuccess && !dir_fused)
                    ee = elide ? launch_cg_pupdate(p, r, len, ctx->state, ss)
                               : launch_bicg_pupdate(p, r, ps, rs, len, ctx->state, ss);
                ++enqueued;
            }
            return ee;
        };
        // From the second batch on, a full batch is the same sequence of
        // launches every time (every kernel takes its scalars and its stop
        // flag from the device state, and the fused schedule's buffer pairs
        // come back after an even number of iterations): it is captured once
        // into a CUDA graph and replayed.
        const bool graph = ctx->graphs && !ctx->profile && enqueued >= check_every && batch == check_every &&
                           (check_every % 2 == 0 || !dir_fused);
        if (graph) {
            const std::vector<uintptr_t> key{(uintptr_t)n, (uintptr_t)bc_kind, (uintptr_t)elide, (uintptr_t)fused,
                                             (uintptr_t)dir_fused, (uintptr_t)ctx->stencil_variant,
                                             (uintptr_t)batch, (uintptr_t)x, (uintptr_t)r, (uintptr_t)rs,
                                             (uintptr_t)pc, (uintptr_t)psc, (uintptr_t)pn, (uintptr_t)psn,
                                             (uintptr_t)q, (uintptr_t)qs};
            cudaGraphExec_t exec = ctx_chunk_graph(ctx, key);
            if (!exec) {
                cudaStream_t cs = ctx_capture_stream(ctx);
                if (!cs) return ctx_cuda(ctx, cudaGetLastError(), "capture stream");
                cudaGraph_t g = nullptr;
                const long long enq0 = enqueued;
                double* const saved[4] = {pc, psc, pn, psn};
                e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    const cudaError_t ee = enqueue(cs);
                    e = cudaStreamEndCapture(cs, &g);
                    if (e == cudaSuccess) e = ee;
                }
                if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
                if (g) cudaGraphDestroy(g);
                if (e != cudaSuccess) return ctx_cuda(ctx, e, "Bi-CG graph capture");
                ctx_store_chunk_graph(ctx, key, exec);
                // the capture ran nothing: undo its bookkeeping
                enqueued = enq0;
                pc = saved[0];
                psc = saved[1];
                pn = saved[2];
                psn = saved[3];
            }
            e = cudaGraphLaunch(exec, s);
            enqueued += batch;   // an even batch leaves the direction pairs where they were
        } else {
            e = enqueue(s);
        }
        note_launches((dir_fused ? 2LL : (fused ? 3LL : 5LL)) * batch);
        if (e != cudaSuccess) return ctx_cuda(ctx, e, "Bi-CG iteration");
    }
    const BicgState& h = *ctx->host_state;
    if (iters_out) *iters_out = h.iter;
    const double rn = sqrt(h.rr);
    if (relres_out) *relres_out = bnorm > 0.0 ? rn / bnorm : rn;
    if (!std::isfinite(h.rr)) return ctx_fail(ctx, EXCMG_ERR_NAN, "Bi-CG residual is not finite");
    if (h.status == kBreakdown) return ctx_fail(ctx, EXCMG_ERR_BREAKDOWN, "Bi-CG breakdown");
    if (h.status == kTimeout) return ctx_fail(ctx, EXCMG_ERR_TIMEOUT, "grid barrier of the cooperative Bi-CG gave up");
    if (h.status == kCapped) return EXCMG_ERR_NOCONV;
    return EXCMG_OK;
}

}  // namespace excmg
