// Internal declarations shared by the CUDA translation units of the library.
// Nothing here is part of the C ABI (include/excmg.h is).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "excmg.h"

namespace excmg {

// ------------------------------------------------------------------ sizes
inline size_t node_count(int n) { return (size_t)(n + 1) * (size_t)(n + 1) * (size_t)(n + 1); }
inline size_t face_count(int n) { return 6 * (size_t)(n + 1) * (size_t)(n + 1); }

// Grid-stride launches of the flat vector kernels use a fixed grid so that
// their reductions always combine the same partial sums in the same order.
constexpr int kVecThreads = 256;
constexpr int kVecBlocks = 152 * 4;     // 4 CTAs on each of GB300's 152 SMs
constexpr int kMaxPartials = 8192;   // >= 2 * kVecBlocks and >= stencil CTAs

// Bi-CG state kept on the device so that a whole iteration runs without the
// host (Alg. 2 with M = I).
struct BicgState {
    double rho;        // (r*_k, r_k)
    double sigma;      // (p*_k, A p_k)
    double alpha;
    double beta;
    double rr;         // (r_k, r_k)
    double bnorm;      // ||b||_2 of the stopping test
    double tol;        // relative tolerance of the stopping test
    double pad0;
    int iter;
    int max_iter;
    int done;          // 1 once converged, capped or broken down
    int status;        // kRunning / kConverged / kCapped / kBreakdown
    unsigned int ticket;   // last-block counter of the reductions
    int pad1[3];
};
static_assert(sizeof(BicgState) % 8 == 0, "read back in 8-byte words");
enum { kRunning = 0, kConverged = 1, kCapped = 2, kBreakdown = 3, kTimeout = 4 };

// ------------------------------------------------------------- kernels
// Stencil (eq. (method1) + reflections): y = A u, or y = b - A u when b is
// non-null.  Writes interior entries of y only.  Returns immediately when
// *skip is non-zero (skip may be null).
enum { kStencilExact = 0, kStencilFp64 = 1 };
cudaError_t launch_stencil(const double* u, double* y, const double* b, int n, int bc_kind,
                           bool transpose, const int* skip, cudaStream_t s, int variant);
cudaError_t launch_zero_boundary(double* y, int n, cudaStream_t s);
// One z-march applying A to p (-> q) and A^T to p* (-> qs) with the integer
// arithmetic, fused with sigma = (p*, q) and alpha = rho / sigma (Alg. 2).
// Skips when st->done.  partials must hold stencil_cta_count(n) doubles.
cudaError_t launch_bicg_stencil_pair(const double* p, double* q, const double* ps, double* qs, int n,
                                     int bc_kind, double* partials, BicgState* st, cudaStream_t s, bool staged);
int stencil_cta_count(int n);
// As launch_bicg_stencil_pair, with the direction update of the previous
// iteration fused in: p = r + beta p_prev, p* = r* + beta p*_prev (beta from
// st), written to p / ps (which must not alias p_prev / ps_prev).
cudaError_t launch_bicg_stencil_pair_dir(const double* r, const double* rs, const double* p_prev,
                                         const double* ps_prev, double* p, double* ps, double* q, double* qs, int n,
                                         int bc_kind, double* partials, BicgState* st, cudaStream_t s);
// Small grids: whole Bi-CG iterations (up to `iters`) in one cooperative
// launch with bounded grid barriers; barrier_words: 3 device words.
constexpr int kPersistentMaxN = 64;
bool persistent_pointwise(int n);
// elide: the shadow-elided mode (rs, ps, qs unused, may be null).
cudaError_t launch_bicg_persistent(double* x, double* r, double* rs, double* p, double* ps, double* q, double* qs,
                                   int n, int bc_kind, int iters, double* partials, BicgState* st,
                                   unsigned int* barrier_words, cudaStream_t s, bool elide);
// Shadow-elided mode (r* = r, p* = p, A^T p* = A p not stored): the one-field
// operator launches with sigma = (p, A p) and alpha (the second also forms
// p = r + beta p_prev into p), and the matching set-up and update kernels.
// They run on the grids of the two-field kernels, so every sum adds the same
// partial sums in the same order and the iterates are bit for bit those of
// the full mode.
cudaError_t launch_cg_stencil(const double* p, double* q, int n, int bc_kind, double* partials, BicgState* st,
                              cudaStream_t s, bool staged);
cudaError_t launch_cg_pupdate(double* p, const double* r, size_t len, const BicgState* st, cudaStream_t s);
cudaError_t launch_cg_stencil_dir(const double* r, const double* p_prev, double* p, double* q, int n, int bc_kind,
                                  double* partials, BicgState* st, cudaStream_t s);
cudaError_t launch_cg_init(const double* r, double* p, size_t len, double* partials, BicgState* st, cudaStream_t s);
cudaError_t launch_cg_update(double* x, const double* p, double* r, const double* q, size_t len, double* partials,
                             BicgState* st, cudaStream_t s);

// Vectors (flat over all (n+1)^3 entries; boundary entries of the Bi-CG
// vectors are zero, so flat sums equal sums over the unknowns).
cudaError_t launch_dot(const double* a, const double* b, size_t len, double* partials,
                       unsigned int* ticket, double* out, cudaStream_t s);
// (a, a) over the interior nodes only (a's boundary entries are ignored).
cudaError_t launch_interior_dot(const double* a, int n, double* partials, unsigned int* ticket, double* out,
                                cudaStream_t s);
cudaError_t launch_bicg_init(const double* r, const double* shadow, double* rs, double* p, double* ps, size_t len,
                             double* partials, BicgState* st, cudaStream_t s);
cudaError_t launch_bicg_sigma(const double* ps, const double* q, size_t len, double* partials,
                              BicgState* st, cudaStream_t s);
cudaError_t launch_bicg_update(double* x, const double* p, double* r, const double* q, double* rs,
                               const double* qs, size_t len, double* partials, BicgState* st,
                               cudaStream_t s);
cudaError_t launch_bicg_pupdate(double* p, const double* r, double* ps, const double* rs, size_t len,
                                const BicgState* st, cudaStream_t s);

// Right-hand side and boundary data for a level with n intervals taken at
// every stride-th node of arrays with n*stride intervals.
cudaError_t launch_assemble_rhs(double* fh, int n, int bc_kind, const double* f, const double* g1,
                                const double* g2, int stride, cudaStream_t s);
cudaError_t launch_set_boundary(double* u, int n, const double* g1, int stride, cudaStream_t s);

// Level transfer.
cudaError_t launch_exp_finite(double* w, const double* u1, const double* u0, double* W_scratch,
                              int n_fine, cudaStream_t s);
cudaError_t launch_exp_true(double* ut, const double* uh, const double* u2h, int n_fine,
                            cudaStream_t s);

// DSOLVE: dense inverse of A_h (unknowns in lexicographic order, x fastest)
// and its application.
cudaError_t launch_dense_assemble(double* A, int n, int bc_kind, cudaStream_t s);
cudaError_t launch_gauss_jordan_step(double* A, int m, int k, double* rowk, double* colk,
                                     cudaStream_t s);
cudaError_t launch_dense_apply(const double* Ainv, const double* fh, double* u, int n,
                               cudaStream_t s);

}  // namespace excmg

// ------------------------------------------------------------ context
struct excmg_buffer {
    void* ptr = nullptr;
    size_t bytes = 0;
};

// Operator launches timed inside Bi-CG on one grid size: device time,
// launch count and the algorithmic bytes those launches read and wrote.
struct ProfRecord {
    double ms = 0.0;
    long long launches = 0;
    double bytes = 0.0;
};

struct excmg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0;           // 0 = unlimited
    size_t bytes = 0;            // currently held
    std::string last_error;
    // named, growable workspace buffers
    std::map<std::string, excmg_buffer> buffers;
    // DSOLVE inverses keyed by (n, bc_kind)
    std::map<std::pair<int, int>, excmg_buffer> inverses;
    // small device scratch for reductions and the Bi-CG state
    double* partials = nullptr;
    unsigned int* ticket = nullptr;
    double* scalar = nullptr;                 // one-off reduction results (8 doubles)
    excmg::BicgState* state = nullptr;        // device
    unsigned int* barrier = nullptr;          // device words of the cooperative solver's grid barrier
    // pinned, mapped host mirrors of `state` and `scalar` and their device
    // addresses: a one-CTA kernel writes them (ctx_read_back), so reading the
    // state back uses no copy engine and never queues behind a caller's large
    // copies
    excmg::BicgState* host_state = nullptr;
    double* host_scalar = nullptr;
    excmg::BicgState* host_state_dev = nullptr;
    double* host_scalar_dev = nullptr;
    int stencil_variant = excmg::kStencilExact;
    int shadow_mode = EXCMG_SHADOW_FULL;
    int schedule = EXCMG_SCHEDULE_FUSED;
    // CUDA graphs of full batches of launched Bi-CG iterations, keyed by the
    // grid size, the variant flags and the buffers they use (bicg.cu)
    bool graphs = true;
    cudaStream_t capture_stream = nullptr;
    std::map<std::vector<uintptr_t>, cudaGraphExec_t> chunk_graphs;
    // optional timing of the operator launches inside Bi-CG
    bool profile = false;
    std::vector<cudaEvent_t> prof_events;
    std::map<int, ProfRecord> prof;   // grid intervals n -> timed operator launches
    // grid-size tuner of the batch engine, per (precision, grid intervals);
    // kept here so that every batch on this context shares what it learned
    struct BatchTune {
        double ms[8];       // milliseconds per round of each candidate, -1 untried
        double cta_ms[8];   // CTA-milliseconds per instance round
        bool settled;
    };
    std::map<std::pair<int, int>, BatchTune> batch_tune;
};

struct excmg_level {
    excmg_ctx* ctx;
    int n;
    int bc_kind;
};

namespace excmg {
// Process-wide count of kernel launches made by the library (capi.cu).
void note_launches(long long k);
// Streaming multiprocessors of the current device (read once per device).
int device_sms();
// Resident CTAs per SM of `kernel` (a __global__ function) with `threads`
// threads and `smem` bytes of dynamic shared memory on the current device,
// at least 1.  A kernel given dynamic shared memory is opted in to that much
// on the current device first (cudaFuncAttributeMaxDynamicSharedMemorySize).  Cached per (kernel, device,
// threads, smem) under a lock: function attributes and occupancy belong to
// each device's context.
int kernel_occupancy(const void* kernel, int threads, size_t smem);
// Cached CUDA graph of a batch of Bi-CG iterations (null if none), storing
// one, and the context's private capture stream (capi.cu).
cudaGraphExec_t ctx_chunk_graph(excmg_ctx* ctx, const std::vector<uintptr_t>& key);
void ctx_store_chunk_graph(excmg_ctx* ctx, const std::vector<uintptr_t>& key, cudaGraphExec_t exec);
cudaStream_t ctx_capture_stream(excmg_ctx* ctx);
// Workspace helpers (capi.cu).
int ctx_fail(excmg_ctx* ctx, int status, const std::string& msg);
int ctx_cuda(excmg_ctx* ctx, cudaError_t err, const char* what);
// Enqueue on ctx's stream a copy of `bytes` (a multiple of 8) from device
// memory to one of the context's mapped host mirrors (host_state or
// host_scalar), written by a kernel; the caller synchronises the stream.
cudaError_t ctx_read_back(excmg_ctx* ctx, void* host_mirror, const void* dev_src, size_t bytes);
double* ctx_buffer(excmg_ctx* ctx, const char* name, size_t bytes, int* status);
// Bi-CG driver (bicg.cu): iterates on the context's stream.
int bicg_run(excmg_ctx* ctx, int n, int bc_kind, const double* b, double* x, double tol,
             double bnorm, int max_iter, int check_every, int* iters_out, double* relres_out,
             const double* shadow = nullptr);
// ||b - A x||_2 over the unknowns, via the context's workspace (result on host).
int true_residual_norm(excmg_ctx* ctx, int n, int bc_kind, const double* b, const double* x,
                       double* out);
int interior_norm(excmg_ctx* ctx, int n, const double* a, double* out);   // flat: zero boundary assumed
int unknowns_norm(excmg_ctx* ctx, int n, const double* a, double* out);   // interior nodes only
// DSOLVE (dsolve.cu)
int dsolve_run(excmg_ctx* ctx, int n, int bc_kind, const double* fh, double* u);
// FP32 inner solves + FP64 refinement on one level (mixed.cu).
int mixed_level_solve(excmg_ctx* ctx, int n, int bc_kind, const double* fh, double* u, double fnorm, double eps,
                      double inner_tol, int max_inner, int max_total, int check_every, int* iters_out,
                      int* outer_out, int* stag_out, double* rel_out);
}  // namespace excmg
