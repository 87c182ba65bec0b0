/*
 * excmg.h -- C ABI of the GB300 (sm_103a) EXCMG solver for the 3D biharmonic
 * equation  Laplacian^2 u = f  on (0,1)^3  with Dirichlet data of the first kind
 * (u = g1, du/dn = g2) or the second kind (u = g1, d2u/dn2 = g2), discretised
 * by the 25-point scheme and solved by extrapolation cascadic multigrid with
 * Bi-CG on every grid (Pan, He & Ni, arXiv 1901.05118).
 *
 * Data layout (every grid function):
 *   N intervals per axis, h = 1/N, nodes i,j,k = 0..N.  A node array holds
 *   (N+1)^3 doubles, x fastest:  idx = (k*(N+1) + j)*(N+1) + i.
 *   The unknowns of a grid are its interior nodes 1..N-1 on every axis.
 *   g2 holds 6 faces of (N+1)^2 doubles, faces ordered x=0, x=1, y=0, y=1,
 *   z=0, z=1; inside a face the two remaining axes (a,b) in x<y<z order give
 *   the index b*(N+1)+a.  For bc_kind = 1, g2 is the OUTWARD normal
 *   derivative du/dn; for bc_kind = 2 it is d2u/dn2.
 *
 * Ownership: every array pointer passed in is a DEVICE pointer (CUDA global
 * memory, e.g. a torch tensor's data_ptr()) owned by the caller; the library
 * never frees or keeps it beyond the call.  The library allocates its own
 * workspace (cudaMalloc) inside a context and frees it in excmg_ctx_destroy.
 *
 * Streams and synchronisation: a context is bound to one CUDA stream.
 * Calls enqueue their kernels on that stream; the caller's inputs must be
 * ready on it.  Every call is synchronous with respect to the host: it
 * returns once its results are complete on the stream, and its status
 * covers the device-side outcome of its own kernels (a Bi-CG breakdown, a
 * non-finite residual, a bounded device wait that gave up).  This differs
 * from an asynchronous convention with errors latched on the device and
 * reported at a later call, for two reasons: the WHILE loop of Alg. 1 and
 * the stopping test of Alg. 2 are steered by scalars the host reads back
 * between batches of Bi-CG iterations, so a solve cannot run ahead of the
 * host anyway; and a synchronous status names the call that failed.  Calls
 * without a context use a per-device default context on the legacy default
 * stream (stream 0).
 *
 * Errors: every call returns an excmg_status; nothing throws across the ABI.
 * excmg_last_error() gives a message for the last failing call on a context
 * (or on the default context when given NULL).  A CUDA error makes the call
 * return EXCMG_ERR_CUDA.
 */
#ifndef EXCMG_H
#define EXCMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EXCMG_OK = 0,
    EXCMG_ERR_ARG = -1,        /* invalid argument (size, bc_kind, null pointer, tolerance) */
    EXCMG_ERR_OOM = -2,        /* device allocation failed                                   */
    EXCMG_ERR_BREAKDOWN = -3,  /* Bi-CG breakdown: (r*,r) or (p*,Ap) zero or not finite      */
    EXCMG_ERR_NOCONV = -4,     /* Bi-CG reached its iteration cap above the tolerance        */
    EXCMG_ERR_NAN = -5,        /* non-finite value in a residual norm                        */
    EXCMG_ERR_CUDA = -6,       /* a CUDA runtime call or kernel launch failed                */
    EXCMG_ERR_TIMEOUT = -7,    /* a bounded device-side wait gave up                         */
    EXCMG_ERR_BUDGET = -9,     /* the context's HBM budget is too small for the request      */
    EXCMG_ERR_SIZE = -10,      /* a size beyond the fixed maximum of an allocation-free call */
    EXCMG_ERR_TOO_LARGE = -11  /* one batch instance needs more than the batch's whole budget */
} excmg_status;

typedef struct excmg_ctx excmg_ctx;      /* device, stream, workspace, DSOLVE factor cache */
typedef struct excmg_level excmg_level;  /* one grid: (context, N, bc_kind)                */

/* Tolerance schedule of Alg. 1: EXCMG_TOL_PAPER uses eps_i = tol * 10^(i-L)
 * (Alg. 1's tolerance schedule); EXCMG_TOL_UNIFORM uses eps_i = tol on every level. */
enum { EXCMG_TOL_PAPER = 0, EXCMG_TOL_UNIFORM = 1 };

/* Arithmetic of the Bi-CG levels.  EXCMG_PRECISION_FP64: Alg. 2 in FP64.
 * EXCMG_PRECISION_MIXED: FP64 iterative refinement -- the true residual
 * r = f_h - A u, the update u += ||r|| e, the stopping test of Alg. 1 and the
 * extrapolation steps in FP64 -- around Bi-CG (Alg. 2) on the scaled
 * correction equation A e = r / ||r|| run entirely in FP32. */
enum { EXCMG_PRECISION_FP64 = 0, EXCMG_PRECISION_MIXED = 1 };

typedef struct {
    double tol;          /* relative residual tolerance eps of Alg. 1 (> 0)                  */
    int tol_mode;        /* EXCMG_TOL_PAPER or EXCMG_TOL_UNIFORM                              */
    int max_iter;        /* cap on the iterations of one Bi-CG call (WHILE body, Alg. 1 l.8)  */
    int max_total;       /* cap on the Bi-CG iterations of one level                          */
    int check_every;     /* iterations enqueued between two host checks of convergence (>= 1) */
    int precision;       /* EXCMG_PRECISION_FP64 or EXCMG_PRECISION_MIXED                     */
    double inner_tol;    /* MIXED: residual reduction asked of each FP32 correction solve     */
} excmg_params;

#define EXCMG_MAX_LEVELS 16

typedef struct {
    int levels;                          /* number of grids, coarsest first            */
    int n[EXCMG_MAX_LEVELS];             /* intervals per axis of each grid            */
    int iters[EXCMG_MAX_LEVELS];         /* Bi-CG iterations (0 on DSOLVE levels)      */
    int calls[EXCMG_MAX_LEVELS];         /* Bi-CG calls of the WHILE loop (MIXED: refinement steps) */
    int stagnated[EXCMG_MAX_LEVELS];     /* 1 if the loop ended on the stagnation rule */
    double relres[EXCMG_MAX_LEVELS];     /* final true relative residual ||f-Au||/||f|| */
    double ms[EXCMG_MAX_LEVELS];         /* device time spent on the level (ms)        */
} excmg_stats;

/* ---------------------------------------------------------------- contexts */

/* Create a context on the current device, bound to `cuda_stream` (a
 * cudaStream_t; NULL = legacy default stream).  hbm_budget_bytes caps the
 * workspace the context may hold (0 = no cap); requests beyond it fail with
 * EXCMG_ERR_BUDGET. */
int excmg_ctx_create(void *cuda_stream, size_t hbm_budget_bytes, excmg_ctx **out);
int excmg_ctx_destroy(excmg_ctx *ctx);
/* Bytes of device workspace the context holds right now. */
size_t excmg_ctx_bytes(const excmg_ctx *ctx);

/* Arithmetic of the 25-point operator (eq. (method1)) on this context:
 * EXCMG_STENCIL_EXACT (default): each input plane of a thread block is put
 *   on one power-of-two scale as 64-bit integers, the 25 integer-weighted
 *   taps are summed exactly and the result is rounded once to double (error
 *   below 3.2e-14 of the largest input magnitude the block reads);
 * EXCMG_STENCIL_FP64: the taps are summed in double precision.
 * Both give results within 1e-13 relative of each other on the same input. */
enum { EXCMG_STENCIL_EXACT = 0, EXCMG_STENCIL_FP64 = 1 };
int excmg_ctx_set_stencil(excmg_ctx *ctx, int variant);

/* Shadow sequence of Bi-CG (Alg. 2) on this context.
 * EXCMG_SHADOW_FULL (default): r*, p* and A^T p* are carried in memory as
 *   Alg. 2 prints them.
 * EXCMG_SHADOW_ELIDED -- not the paper's algorithm as printed, a labelled
 *   variant: A_h is symmetric, and with r*_0 = r_0 and the exact operator
 *   (EXCMG_STENCIL_EXACT) A^T p* and A p are the same bits, so the shadow
 *   sequence equals the primal one bit for bit; it is then neither stored
 *   nor read (88 instead of 152 bytes per unknown and iteration on large
 *   grids) and every iterate, stopping decision and result is bit for bit
 *   that of EXCMG_SHADOW_FULL.  It applies to the exact operator only: with
 *   EXCMG_STENCIL_FP64, and in calls that pass their own r*_0
 *   (bicg_solve_ex), the full sequence runs.  The batch engine always runs
 *   the full sequence. */
enum { EXCMG_SHADOW_FULL = 0, EXCMG_SHADOW_ELIDED = 1 };
int excmg_ctx_set_shadow_mode(excmg_ctx *ctx, int mode);

/* How a Bi-CG iteration is split into kernels on grids above 64^3 (integer
 * operator); both give the same iterates up to the reduction order of sigma
 * (same bits within one schedule).  Grids up to 64^3 run a three-phase
 * cooperative launch in both.
 * EXCMG_SCHEDULE_FUSED (default): the operator launch first forms
 *   p = r + beta p and p* = r* + beta p* from the previous directions on
 *   every node it loads (writing the nodes it owns into a second buffer
 *   pair), then applies A and A^T with sigma and alpha; with the update
 *   (x, r, r*, rho, beta) that makes two launches and 136 bytes per unknown.
 * EXCMG_SCHEDULE_SEPARATE: operator pair (A p, A^T p*, sigma, alpha), update
 *   and direction update (p, p*) as three launches, 152 bytes per unknown. */
enum { EXCMG_SCHEDULE_SEPARATE = 0, EXCMG_SCHEDULE_FUSED = 1 };
int excmg_ctx_set_schedule(excmg_ctx *ctx, int schedule);

/* CUDA graphs (default on): on grids solved by launched kernels (above
 * 64^3), every full batch of Bi-CG iterations after the first -- the same
 * sequence of launches each time, all of them reading their scalars and
 * their stop flag from the device -- is captured once into a CUDA graph (on
 * a private stream of the context) and replayed, cached per grid size,
 * variant and buffer set.  Results are the same bits with graphs on or off.
 * Graphs are not used while operator timing (excmg_ctx_profile) is on. */
int excmg_ctx_set_graphs(excmg_ctx *ctx, int enable);
const char *excmg_last_error(const excmg_ctx *ctx);

/* Instrumentation.  excmg_launch_count: kernel launches the library has
 * made in this process (all contexts).  excmg_ctx_profile(ctx, 1) makes the
 * context time every operator launch inside Bi-CG with CUDA events on its
 * stream (and clears earlier records); excmg_ctx_profile_read returns, for
 * grids with n intervals, the summed device time (ms), the number of
 * operator launches timed since and (bytes may be NULL) the algorithmic
 * bytes those launches read and wrote: 8 B per unknown for every field in
 * or out (a launch of the fused pair that also forms the directions moves
 * eight fields, the plain pair four, one FP64 application two). */
long long excmg_launch_count(void);
int excmg_ctx_profile(excmg_ctx *ctx, int enable);
int excmg_ctx_profile_read(const excmg_ctx *ctx, int n, double *ms_total, long long *launches,
                           double *bytes);

/* One grid with N intervals (N >= 4) and the given kind of boundary data.
 * The level borrows the context (destroy levels before their context). */
int excmg_level_create(excmg_ctx *ctx, int n, int bc_kind, excmg_level **out);
int excmg_level_destroy(excmg_level *level);

/* ---------------------------------------------------------- the hot path */

/* y = A_h u  (transpose = 0)  or  y = A_h^T u  (transpose = 1).
 * A_h is the matrix of eq. (sec): the 25-point scheme of eq. (method1) on the
 * interior nodes, with the fictitious nodes outside the domain folded onto
 * their mirror nodes by eq. (reflection2) (first kind: +1 on the diagonal per
 * near-boundary axis) or eq. (reflection4) (second kind: -1).  Only the
 * interior entries of u are read (its boundary entries are ignored); the
 * interior entries of y are written and its boundary entries set to 0.
 * u and y are node arrays of the level, and must not overlap. */
int stencil_apply(const excmg_level *level, int transpose, const double *u, double *y);

/* Bi-CG with preconditioner (Alg. 2) in real arithmetic, M = I, shadow
 * residual r*_0 = r_0, on A_h x = b.  b: node array (interior entries read);
 * x_inout: node array, initial guess in, iterate out (boundary entries left
 * unchanged).  Iterates until the recursively updated residual satisfies
 * ||r_k||_2 <= tol * ||b||_2 or max_iter iterations, both norms taken over
 * the unknowns (b's boundary entries are not part of the system and are
 * ignored).  iters_out / relres_out (may be NULL) receive the iteration
 * count and ||r_k||_2 / ||b||_2.
 * Returns EXCMG_OK on convergence, EXCMG_ERR_NOCONV at the cap,
 * EXCMG_ERR_BREAKDOWN on a breakdown. */
int bicg_solve(const excmg_level *level, const double *b, double *x_inout, double tol,
               int max_iter, int *iters_out, double *relres_out);

/* bicg_solve with a caller-chosen shadow residual r*_0 (Alg. 2 leaves
 * x*_0 and b* free): shadow_r0 is a node array whose interior entries give
 * r*_0 ((r_0, r*_0) must not vanish); NULL means r*_0 = r_0. */
int bicg_solve_ex(const excmg_level *level, const double *b, double *x_inout, const double *shadow_r0,
                  double tol, int max_iter, int *iters_out, double *relres_out);

/* EXP_finite (Sec. 4.2.2-4.2.3, Steps 1-5; Alg. 1's initial guess): third-order
 * approximation w_h on the grid with n_fine intervals (n_fine divisible by
 * 4, >= 8) of the FD solution, from the FD solutions u_2h (n_fine/2
 * intervals) and u_4h (n_fine/4 intervals), all node arrays.  Steps 1-5 give
 * every node of w_h, boundary nodes included.  g1_fine: a node array on the
 * fine grid whose boundary entries (the Dirichlet data u = g1) then
 * overwrite w_h's boundary nodes, as Alg. 1 does before Bi-CG; NULL keeps the
 * interpolated boundary values (the distances ||w_h - u_h|| printed in the
 * paper's tables are those of the interpolated values).  Interior nodes do
 * not depend on g1_fine. */
int extrapolate_interpolate(int n_fine, const double *u_2h, const double *u_4h, const double *g1_fine,
                            double *w_h);

/* EXP_finite as above with g1_fine = NULL, allocating nothing (the paper has no counterpart: it
 * is a service for callers that cannot allocate device memory at this point
 * -- memory owned entirely by an arena or planner, a hard device-memory
 * budget, or a path where entering the CUDA allocator, which may synchronise
 * the device, is not allowed).  Its scratch lives in a fixed array inside
 * the library (2.2 MB, held by every GPU that loads the library until the
 * process exits), so n_fine is limited to 128; larger sizes return
 * EXCMG_ERR_SIZE.  The caller passes inputs and output as for
 * extrapolate_interpolate.  Runs on the legacy default stream and returns
 * when the result is complete.  Every call looks up the array's device
 * address on the current device; the first call on a device also loads the
 * library's device code there, so make that first call before any stream
 * capture.
 * All calls share the one array: calls that overlap on the GPU (other host
 * threads, other streams) race and must be serialised by the caller. */
int extrapolate_interpolate_noalloc(int n_fine, const double *u_2h, const double *u_4h, double *w_h);

/* EXP_true (Sec. 4.2.1, eqs. (t1), (chenlin); Alg. 1's final extrapolation): extrapolated
 * solution u_tilde = u_h + (1/3) * multilinear interpolation of (u_h - u_2h)
 * on the grid with n_fine intervals (even, >= 4).  Every node is written. */
int midpoint_extrapolate(int n_fine, const double *u_h, const double *u_2h, double *u_tilde);

/* Alg. 1: EXCMG from the coarsest grid n_coarsest to the finest n_finest =
 * n_coarsest * 2^(L+1), L >= 1 (n_coarsest >= 4).  f, g1: node arrays on the
 * finest grid (f's interior and g1's boundary entries are read; coarser grids
 * take every stride-th node); g2: the 6 faces on the finest grid.  The two
 * coarsest grids are solved directly (DSOLVE), every finer one by
 * EXP_finite + Bi-CG until ||f_h - A_h u_h||_2 <= tol ||f_h||_2 on every level.
 * u_out receives u_tilde = EXP_true(u_h, u_2h) on the finest grid. */
int excmg_solve(int n_finest, int n_coarsest, int bc_kind, const double *f, const double *g1,
                const double *g2, double tol, double *u_out);

/* Extended form of excmg_solve on an explicit context: parameters as above,
 * u_h_out (may be NULL) receives the finest FD solution u_h, u_tilde_out
 * (may be NULL) the extrapolated solution, stats (may be NULL) per-level
 * counters. */
int excmg_solve_ex(excmg_ctx *ctx, int n_finest, int n_coarsest, int bc_kind, const double *f,
                   const double *g1, const double *g2, const excmg_params *params,
                   double *u_h_out, double *u_tilde_out, excmg_stats *stats);

/* Context forms of the two transfer steps (same semantics, ctx's stream). */
int extrapolate_interpolate_ex(excmg_ctx *ctx, int n_fine, const double *u_2h, const double *u_4h,
                               const double *g1_fine, double *w_h);
int midpoint_extrapolate_ex(excmg_ctx *ctx, int n_fine, const double *u_h, const double *u_2h,
                            double *u_tilde);

/* Right-hand side f_h of eq. (sec) for a level: h^4 f plus every known
 * boundary value and ghost datum the 25-point rows touch, moved across
 * (Sec. 2, the 27 position cases).  f, g1, g2 are given on a finer grid with
 * n_src = stride * N intervals (stride >= 1); the level takes every
 * stride-th node.  fh: node array of the level (boundary entries set to 0). */
int excmg_assemble_rhs(const excmg_level *level, int n_src, const double *f, const double *g1,
                       const double *g2, double *fh);

/* DSOLVE (Alg. 1's direct solves): u = A_h^{-1} fh on the level's interior nodes
 * (u's boundary entries left unchanged).  The first call on a (N, bc_kind)
 * factorises A_h (dense Gauss-Jordan inverse, kept in the context); 4 <= N <= 16
 * (at most 15^3 = 3375 unknowns, a 91 MB inverse), else EXCMG_ERR_ARG. */
int excmg_dsolve(const excmg_level *level, const double *fh, double *u);

/* ------------------------------------------------------ many solves at once */

/* A batch engine runs many independent EXCMG solves (Alg. 1) concurrently on
 * one context's GPU and stream, each in FP64 (integer operator, FP64 Bi-CG)
 * or in the mixed-precision form (FP64 refinement around FP32 Bi-CG
 * correction solves, see EXCMG_PRECISION_MIXED).  Every instance keeps its
 * level hierarchy resident; the Bi-CG iterations of the instances that need
 * them run per level group (instances of one precision at one grid size),
 * each group on its own stream and taken back as soon as it completes: one
 * cooperative launch for all members of a group on grids up to 64^3 (and
 * for FP32 correction solves), the single solver's kernels per member on
 * larger FP64 grids.  Instances may be submitted at any time and leave when
 * done, so the batch refills continuously. */
typedef struct excmg_batch excmg_batch;

/* hbm_budget_bytes caps the device memory all live instances may hold
 * (0 = no cap); max_instances caps their number (1..1024). */
int excmg_batch_create(excmg_ctx *ctx, size_t hbm_budget_bytes, int max_instances, excmg_batch **out);
int excmg_batch_destroy(excmg_batch *batch);
const char *excmg_batch_last_error(const excmg_batch *batch);
/* Device memory held by live instances now, and what one instance needs. */
size_t excmg_batch_bytes(const excmg_batch *batch);
size_t excmg_batch_instance_bytes(int n_finest, int n_coarsest, int precision);

/* Admit one solve: arguments as for excmg_solve_ex (params->precision picks
 * FP64 or mixed; max_iter caps one Bi-CG call, inner_tol is used in mixed
 * mode).  f, g1, g2 and u_out must stay valid until the instance is done;
 * u_out receives u_tilde.  Returns EXCMG_ERR_BUDGET (nothing admitted) when
 * the budget or the slot count is full right now -- submit again after a
 * step -- and EXCMG_ERR_TOO_LARGE when the instance alone needs more than
 * the whole budget, so that it can never be admitted.  n_finest is limited to
 * grids whose operator launch has at most 8192 CTAs (2048 intervals);
 * larger ones return EXCMG_ERR_ARG. */
int excmg_batch_submit(excmg_batch *batch, int n_finest, int n_coarsest, int bc_kind, const double *f,
                       const double *g1, const double *g2, const excmg_params *params, double *u_out,
                       int *id_out);

/* Advance every live instance (all pending per-instance steps, then one
 * batched launch of FP32 Bi-CG iterations).  *n_live (may be NULL) receives
 * the number of instances still running. */
int excmg_batch_step(excmg_batch *batch, int *n_live);

/* *done = 1 once instance `id` has finished; then *status is its outcome,
 * stats (may be NULL) its per-level counters and *latency_s (may be NULL)
 * the wall time from submit to finish. */
int excmg_batch_query(excmg_batch *batch, int id, int *done, int *status, excmg_stats *stats,
                      double *latency_s);
/* Kernel launches made by the batch so far. */
long long excmg_batch_launches(const excmg_batch *batch);

/* Where a batch's time went, summed since it was created: its cooperative
 * Bi-CG launches (one per level group and step), their rounds, rounds times
 * members (member slots, busy or idle), member iterations actually taken,
 * the launches' device time (CUDA events on their streams), and the wall
 * time of excmg_batch_step outside / inside its wait for a running launch. */
typedef struct {
    long long group_launches;
    long long rounds;
    long long member_rounds;
    long long member_iters;
    double group_ms;
    double host_s;
    double wait_s;
} excmg_batch_profile;
int excmg_batch_get_profile(const excmg_batch *batch, excmg_batch_profile *out);

/* ------------------------------------------------------- the 2D problem */

/* The two-dimensional problem of eq. (bvp2d): Laplacian^2 u = f on (0,1)^2
 * with first- or second-kind Dirichlet data, discretised by the 13-point
 * scheme (the paper names it without printing it; here the one built as
 * eq. (method1) is built: 20 u - 8 (4 axis neighbours) + (4 at distance 2)
 * + 2 (4 diagonal neighbours) = h^4 f, the square of the five-point
 * Laplacian) with the reflection formulas of Sec. 2 along each axis, and
 * solved by Alg. 1 / Alg. 2 with the 2D forms of the transfer steps.
 * Node arrays hold (N+1)^2 doubles, x fastest: idx = j*(N+1) + i; g2 holds 4
 * edges of N+1 doubles (x=0, x=1, y=0, y=1), indexed by the other
 * coordinate (outward du/dn for bc_kind 1, d2u/dn2 for bc_kind 2).  Device
 * pointers owned by the caller; every call is synchronous on ctx's stream.
 * The operator sums its integer-weighted taps exactly on one power-of-two
 * scale per 32 x 16 tile (the tile's largest input exponent) and rounds
 * each output once.  Errors: EXCMG_ERR_ARG for a null pointer, bc_kind not
 * 1 or 2, N < 4 (EXP_finite: n_fine < 8 or not a multiple of 4; EXP_true:
 * n_fine odd), N > 2049 in the Bi-CG and solve calls (one partial sum per
 * 32 x 16 tile, at most 8192), u == y in excmg2d_stencil_apply; the other
 * statuses as for the 3D calls (EXCMG_ERR_NOCONV from excmg2d_bicg_solve at
 * its iteration cap, EXCMG_ERR_BREAKDOWN, EXCMG_ERR_NAN, EXCMG_ERR_OOM,
 * EXCMG_ERR_BUDGET, EXCMG_ERR_CUDA). */
/* y = A_h u (transpose: A_h^T u, the same bits); interior entries of u read,
 * boundary entries of y set to 0. */
int excmg2d_stencil_apply(excmg_ctx *ctx, int n, int bc_kind, int transpose, const double *u, double *y);
/* Alg. 2 (M = I, r*_0 = r_0) on the 2D system, as bicg_solve. */
int excmg2d_bicg_solve(excmg_ctx *ctx, int n, int bc_kind, const double *b, double *x_inout, double tol,
                       int max_iter, int *iters_out, double *relres_out);
/* EXP_finite in 2D (corners eq. (secfff), edge midpoints eq. (bfsec), cell
 * centres the mean of the two diagonal rules, bi-quadratic interpolation);
 * g1_fine as for extrapolate_interpolate (NULL: interpolated boundary). */
int excmg2d_extrapolate_interpolate(excmg_ctx *ctx, int n_fine, const double *u_2h, const double *u_4h,
                                    const double *g1_fine, double *w_h);
/* EXP_true in 2D: u_tilde = u_h + (1/3) bilinear interpolation of u_h - u_2h. */
int excmg2d_midpoint_extrapolate(excmg_ctx *ctx, int n_fine, const double *u_h, const double *u_2h,
                                 double *u_tilde);
/* Alg. 1 in 2D (FP64), arguments as excmg_solve_ex; n_coarsest 4..16 (the two
 * direct-solve grids have at most 31^2 unknowns). */
int excmg2d_solve(excmg_ctx *ctx, int n_finest, int n_coarsest, int bc_kind, const double *f, const double *g1,
                  const double *g2, const excmg_params *params, double *u_h_out, double *u_tilde_out,
                  excmg_stats *stats);

/* ------------------------------------------------------------- diagnostics */

/* Failure-path self-test (the paper has no counterpart): makes one of the
 * library's bounded device-side waits run out on purpose -- without a fault,
 * trap or hang -- so that the path that reports EXCMG_ERR_TIMEOUT can be
 * tested.  which = 0 (the only wait kind): the grid barrier of the
 * cooperative kernels; a cooperative launch of 8 CTAs waits for a ninth
 * arrival that never comes, and each CTA gives up after `limit` polls (at
 * least 32 ns each).  1 <= limit <= 10^8.
 * Returns EXCMG_ERR_TIMEOUT when the wait gave up as designed, EXCMG_OK if it
 * did not (the mechanism failed), EXCMG_ERR_ARG, or EXCMG_ERR_CUDA.  Uses
 * fixed device memory (allocates nothing), runs on the legacy default stream
 * and returns when done. */
int excmg_selftest_wait_timeout(int which, long long limit);

#ifdef __cplusplus
}
#endif

#endif /* EXCMG_H */
