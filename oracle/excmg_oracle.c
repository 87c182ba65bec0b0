/*
 * Plain FP64 CPU oracle for the EXCMG / 25-point-scheme solver of the 3D
 * biharmonic equation (Pan, He & Ni, arXiv 1901.05118).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: it exists so that tests/, the smoke check and the CPU
 * baseline leg of bench.py can check the CUDA library against a slow,
 * obviously-correct restatement of the paper.  It shares no code, header,
 * table or helper with the CUDA sources.
 *
 * Conventions (shared with the C-ABI only as an interface, not as code):
 *   N intervals per axis, h = 1/N, nodes i,j,k = 0..N.
 *   Grid functions are node arrays of (N+1)^3 doubles, x fastest:
 *       idx = (k*(N+1) + j)*(N+1) + i.
 *   Unknowns are the interior nodes 1..N-1 on every axis.
 *   g2 is stored as 6 faces of (N+1)^2 doubles, faces ordered
 *   x=0, x=1, y=0, y=1, z=0, z=1; inside a face the two remaining axes
 *   (a,b) in x<y<z order give the index b*(N+1)+a.
 *   bc_kind = 1: g2 = du/dn (outward normal), eq. (BC);
 *   bc_kind = 2: g2 = d2u/dn2, eq. (BC2).
 *
 * Everything is double precision; compile with -ffp-contract=off so that no
 * multiply-add is fused behind the reader's back.
 *
 * Threads: when built with OpenMP, loops whose iterations are independent
 * (one output entry each: the operator, the vector updates) are split over
 * threads; every entry is still computed by one thread in the same order of
 * operations, and every sum over entries (the inner products) stays a single
 * sequential loop, so the results are the same bits for any thread count.
 * orc_set_threads() chooses the count (default 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OOM (-2)
#define ORC_ERR_BREAKDOWN (-3)
#define ORC_ERR_PIVOT (-8)

static int orc_threads = 1;

/* Threads of the parallel loops (1 = sequential; ignored without OpenMP).
 * Returns the count in effect. */
int orc_set_threads(int n) {
#ifdef _OPENMP
    orc_threads = n < 1 ? 1 : n;
#else
    (void)n;
    orc_threads = 1;
#endif
    return orc_threads;
}

static size_t nidx(int N, int i, int j, int k) {
    return ((size_t)k * (size_t)(N + 1) + (size_t)j) * (size_t)(N + 1) + (size_t)i;
}

/* ------------------------------------------------------------------------
 * The 25-point stencil of eq. (method1), taps listed in the order in which
 * the equation prints them: centre (42), the six axis neighbours (-12),
 * the six axis neighbours two steps away (+1) and the twelve in-plane
 * diagonal neighbours (+2).
 * ---------------------------------------------------------------------- */
typedef struct { int dx, dy, dz; double c; } orc_tap;

static const orc_tap TAPS[25] = {
    {0, 0, 0, 42.0},
    {-1, 0, 0, -12.0}, {1, 0, 0, -12.0}, {0, -1, 0, -12.0},
    {0, 1, 0, -12.0},  {0, 0, -1, -12.0}, {0, 0, 1, -12.0},
    {-2, 0, 0, 1.0}, {2, 0, 0, 1.0}, {0, -2, 0, 1.0},
    {0, 2, 0, 1.0},  {0, 0, -2, 1.0}, {0, 0, 2, 1.0},
    {-1, -1, 0, 2.0}, {-1, 1, 0, 2.0}, {1, -1, 0, 2.0}, {1, 1, 0, 2.0},
    {-1, 0, -1, 2.0}, {1, 0, -1, 2.0}, {0, -1, -1, 2.0}, {0, 1, -1, 2.0},
    {-1, 0, 1, 2.0},  {1, 0, 1, 2.0},  {0, -1, 1, 2.0},  {0, 1, 1, 2.0},
};

/* How the tap p+d of an interior row p enters the linear system. */
enum { TAP_UNKNOWN = 0, TAP_BOUNDARY = 1, TAP_GHOST = 2 };

typedef struct {
    int kind;          /* TAP_UNKNOWN / TAP_BOUNDARY / TAP_GHOST            */
    int qi, qj, qk;    /* unknown column (the mirror node for a ghost)      */
    int bi, bj, bk;    /* boundary node holding the data (ghost / boundary) */
    int face;          /* ghost only: face 0..5 of the boundary node        */
} orc_tapinfo;

/* Classify tap d of interior node (i,j,k).  A ghost arises only from the
 * +-2 axis taps of a node one step from the boundary (Sec. 2, eqs.
 * (reflection1)-(reflection4)); its value is replaced through the mirror
 * node across the boundary face. */
static orc_tapinfo classify(int N, int i, int j, int k, const orc_tap *t) {
    orc_tapinfo r;
    int q[3] = {i + t->dx, j + t->dy, k + t->dz};
    int axis = -1, side = 0, a;
    memset(&r, 0, sizeof r);
    for (a = 0; a < 3; ++a) {
        if (q[a] < 0) { axis = a; side = 0; }
        if (q[a] > N) { axis = a; side = 1; }
    }
    if (axis >= 0) {
        int m[3] = {q[0], q[1], q[2]};
        int b[3] = {q[0], q[1], q[2]};
        m[axis] = side ? (N - 1) : 1;     /* u_{-1} -> u_1, u_{N+1} -> u_{N-1} */
        b[axis] = side ? N : 0;
        r.kind = TAP_GHOST;
        r.qi = m[0]; r.qj = m[1]; r.qk = m[2];
        r.bi = b[0]; r.bj = b[1]; r.bk = b[2];
        r.face = 2 * axis + side;
        return r;
    }
    for (a = 0; a < 3; ++a) {
        if (q[a] == 0 || q[a] == N) {
            r.kind = TAP_BOUNDARY;
            r.bi = q[0]; r.bj = q[1]; r.bk = q[2];
            return r;
        }
    }
    r.kind = TAP_UNKNOWN;
    r.qi = q[0]; r.qj = q[1]; r.qk = q[2];
    return r;
}

/* face-local index of boundary node (bi,bj,bk) on face f */
static size_t face_index(int N, int f, int bi, int bj, int bk) {
    int axis = f / 2;
    int a, b;
    if (axis == 0) { a = bj; b = bk; }
    else if (axis == 1) { a = bi; b = bk; }
    else { a = bi; b = bj; }
    return (size_t)f * (size_t)(N + 1) * (size_t)(N + 1) + (size_t)b * (size_t)(N + 1) + (size_t)a;
}

/* sign with which a ghost folds onto its mirror unknown:
 * first kind  u_ghost = u_mirror + 2h g2            (eq. reflection2)
 * second kind u_ghost = -u_mirror + 2 g1 + h^2 g2   (eq. reflection4) */
static double ghost_sign(int bc_kind) { return bc_kind == 1 ? 1.0 : -1.0; }

/* ------------------------------------------------------------------------
 * y = A_h u (transpose = 0) or y = A_h^T u (transpose = 1), eq. (sec).
 * Only interior entries of u are read; interior entries of y are written,
 * boundary entries of y are set to zero.  The transpose is formed by
 * scattering each row into its columns, so it does not presume symmetry.
 * ---------------------------------------------------------------------- */
int orc_stencil_apply(int N, int bc_kind, int transpose, const double *u, double *y) {
    int i, j, k, t;
    size_t total;
    double s;
    if (N < 4 || (bc_kind != 1 && bc_kind != 2) || !u || !y) return ORC_ERR_ARG;
    total = (size_t)(N + 1) * (size_t)(N + 1) * (size_t)(N + 1);
    s = ghost_sign(bc_kind);
    if (!transpose) {
#pragma omp parallel for num_threads(orc_threads) private(i, j, t) schedule(static)
        for (k = 0; k <= N; ++k)
            for (j = 0; j <= N; ++j)
                for (i = 0; i <= N; ++i) {
                    double acc = 0.0;
                    if (i < 1 || i > N - 1 || j < 1 || j > N - 1 || k < 1 || k > N - 1) {
                        y[nidx(N, i, j, k)] = 0.0;
                        continue;
                    }
                    if (i >= 3 && i <= N - 3 && j >= 3 && j <= N - 3 && k >= 3 && k <= N - 3) {
                        /* three or more steps from every face: all 25 taps are unknowns */
                        for (t = 0; t < 25; ++t)
                            acc += TAPS[t].c * u[nidx(N, i + TAPS[t].dx, j + TAPS[t].dy, k + TAPS[t].dz)];
                        y[nidx(N, i, j, k)] = acc;
                        continue;
                    }
                    for (t = 0; t < 25; ++t) {
                        orc_tapinfo ti = classify(N, i, j, k, &TAPS[t]);
                        if (ti.kind == TAP_UNKNOWN)
                            acc += TAPS[t].c * u[nidx(N, ti.qi, ti.qj, ti.qk)];
                        else if (ti.kind == TAP_GHOST)
                            acc += s * TAPS[t].c * u[nidx(N, ti.qi, ti.qj, ti.qk)];
                    }
                    y[nidx(N, i, j, k)] = acc;
                }
    } else if (orc_threads <= 1) {
        memset(y, 0, total * sizeof(double));
        for (k = 1; k <= N - 1; ++k)
            for (j = 1; j <= N - 1; ++j)
                for (i = 1; i <= N - 1; ++i) {
                    double up = u[nidx(N, i, j, k)];
                    if (i >= 3 && i <= N - 3 && j >= 3 && j <= N - 3 && k >= 3 && k <= N - 3) {
                        for (t = 0; t < 25; ++t)
                            y[nidx(N, i + TAPS[t].dx, j + TAPS[t].dy, k + TAPS[t].dz)] += TAPS[t].c * up;
                        continue;
                    }
                    for (t = 0; t < 25; ++t) {
                        orc_tapinfo ti = classify(N, i, j, k, &TAPS[t]);
                        if (ti.kind == TAP_UNKNOWN)
                            y[nidx(N, ti.qi, ti.qj, ti.qk)] += TAPS[t].c * up;
                        else if (ti.kind == TAP_GHOST)
                            y[nidx(N, ti.qi, ti.qj, ti.qk)] += s * TAPS[t].c * up;
                    }
                }
    } else {
        /* The same scatter on several threads.  Rows are visited in the same
         * lexicographic order, but the writes are grouped by the plane kt of
         * the column they land in: plane kt of y receives them from rows
         * kt-2 .. kt+2 only (a ghost folds onto its own row's plane), in the
         * order the single pass above delivers them, so the planes of y are
         * independent and every entry gets the same bits. */
        int kt, by_dz[5][25], n_dz[5] = {0, 0, 0, 0, 0};
        /* the taps of each plane offset dz = -2..2, in table order */
        for (t = 0; t < 25; ++t) by_dz[TAPS[t].dz + 2][n_dz[TAPS[t].dz + 2]++] = t;
        memset(y, 0, total * sizeof(double));
#pragma omp parallel for num_threads(orc_threads) private(i, j, k, t) schedule(dynamic, 1)
        for (kt = 1; kt <= N - 1; ++kt)
            for (k = (kt - 2 > 1 ? kt - 2 : 1); k <= (kt + 2 < N - 1 ? kt + 2 : N - 1); ++k)
                for (j = 1; j <= N - 1; ++j)
                    for (i = 1; i <= N - 1; ++i) {
                        double up = u[nidx(N, i, j, k)];
                        if (i >= 3 && i <= N - 3 && j >= 3 && j <= N - 3 && k >= 3 && k <= N - 3) {
                            const int g = kt - k + 2;
                            int m;
                            for (m = 0; m < n_dz[g]; ++m) {
                                const orc_tap *tp = &TAPS[by_dz[g][m]];
                                y[nidx(N, i + tp->dx, j + tp->dy, kt)] += tp->c * up;
                            }
                            continue;
                        }
                        for (t = 0; t < 25; ++t) {
                            orc_tapinfo ti;
                            if (k + TAPS[t].dz != kt && k != kt) continue;   /* cannot land in plane kt */
                            ti = classify(N, i, j, k, &TAPS[t]);
                            if (ti.qk != kt) continue;
                            if (ti.kind == TAP_UNKNOWN)
                                y[nidx(N, ti.qi, ti.qj, ti.qk)] += TAPS[t].c * up;
                            else if (ti.kind == TAP_GHOST)
                                y[nidx(N, ti.qi, ti.qj, ti.qk)] += s * TAPS[t].c * up;
                        }
                    }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Right-hand side f_h of eq. (sec): h^4 f at each interior node, minus every
 * known value the row touches, moved across (Sec. 2, the 27 position
 * cases).  f, g1 are node arrays of this level, g2 the 6 faces of this
 * level.  Boundary entries of fh are set to zero.
 * ---------------------------------------------------------------------- */
int orc_assemble_rhs(int N, int bc_kind, const double *f, const double *g1, const double *g2, double *fh) {
    int i, j, k, t;
    double h, h4;
    if (N < 4 || (bc_kind != 1 && bc_kind != 2) || !f || !g1 || !g2 || !fh) return ORC_ERR_ARG;
    h = 1.0 / (double)N;
    h4 = h * h * h * h;
    for (k = 0; k <= N; ++k)
        for (j = 0; j <= N; ++j)
            for (i = 0; i <= N; ++i) {
                double rhs;
                if (i < 1 || i > N - 1 || j < 1 || j > N - 1 || k < 1 || k > N - 1) {
                    fh[nidx(N, i, j, k)] = 0.0;
                    continue;
                }
                rhs = h4 * f[nidx(N, i, j, k)];
                for (t = 0; t < 25; ++t) {
                    orc_tapinfo ti = classify(N, i, j, k, &TAPS[t]);
                    if (ti.kind == TAP_BOUNDARY) {
                        rhs -= TAPS[t].c * g1[nidx(N, ti.bi, ti.bj, ti.bk)];
                    } else if (ti.kind == TAP_GHOST) {
                        double gb = g2[face_index(N, ti.face, ti.bi, ti.bj, ti.bk)];
                        double known;
                        if (bc_kind == 1)
                            known = 2.0 * h * gb;                              /* eq. (reflection2) */
                        else
                            known = 2.0 * g1[nidx(N, ti.bi, ti.bj, ti.bk)] + h * h * gb; /* eq. (reflection4) */
                        rhs -= TAPS[t].c * known;
                    }
                }
                fh[nidx(N, i, j, k)] = rhs;
            }
    return ORC_OK;
}

/* Injection of a finer node array / face set onto a coarser level whose
 * nodes are every `stride`-th node of the finer one (the grids of Alg. 1
 * are nested). */
int orc_inject_nodes(int Nf, int stride, const double *src, double *dst) {
    int Nc, i, j, k;
    if (stride < 1 || Nf % stride) return ORC_ERR_ARG;
    Nc = Nf / stride;
    for (k = 0; k <= Nc; ++k)
        for (j = 0; j <= Nc; ++j)
            for (i = 0; i <= Nc; ++i)
                dst[nidx(Nc, i, j, k)] = src[nidx(Nf, stride * i, stride * j, stride * k)];
    return ORC_OK;
}

int orc_inject_faces(int Nf, int stride, const double *src, double *dst) {
    int Nc, f, a, b;
    size_t fsf, fsc;
    if (stride < 1 || Nf % stride) return ORC_ERR_ARG;
    Nc = Nf / stride;
    fsf = (size_t)(Nf + 1) * (size_t)(Nf + 1);
    fsc = (size_t)(Nc + 1) * (size_t)(Nc + 1);
    for (f = 0; f < 6; ++f)
        for (b = 0; b <= Nc; ++b)
            for (a = 0; a <= Nc; ++a)
                dst[f * fsc + (size_t)b * (Nc + 1) + a] =
                    src[f * fsf + (size_t)(stride * b) * (Nf + 1) + (size_t)(stride * a)];
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Dense matrix of the operator in lexicographic unknown order
 * (x fastest over interior nodes).  For tests and for DSOLVE.
 * ---------------------------------------------------------------------- */
static size_t uidx(int N, int i, int j, int k) {
    size_t m = (size_t)(N - 1);
    return ((size_t)(k - 1) * m + (size_t)(j - 1)) * m + (size_t)(i - 1);
}

int orc_assemble_dense(int N, int bc_kind, double *A) {
    int i, j, k, t;
    size_t n;
    double s;
    if (N < 4 || (bc_kind != 1 && bc_kind != 2) || !A) return ORC_ERR_ARG;
    n = (size_t)(N - 1) * (size_t)(N - 1) * (size_t)(N - 1);
    s = ghost_sign(bc_kind);
    memset(A, 0, n * n * sizeof(double));
    for (k = 1; k <= N - 1; ++k)
        for (j = 1; j <= N - 1; ++j)
            for (i = 1; i <= N - 1; ++i) {
                size_t row = uidx(N, i, j, k);
                for (t = 0; t < 25; ++t) {
                    orc_tapinfo ti = classify(N, i, j, k, &TAPS[t]);
                    if (ti.kind == TAP_UNKNOWN)
                        A[row * n + uidx(N, ti.qi, ti.qj, ti.qk)] += TAPS[t].c;
                    else if (ti.kind == TAP_GHOST)
                        A[row * n + uidx(N, ti.qi, ti.qj, ti.qk)] += s * TAPS[t].c;
                }
            }
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * DSOLVE (Alg. 1's direct solves): a direct solve of A_h u_h = f_h.  Gaussian
 * elimination without pivoting in band storage; in lexicographic order the
 * half bandwidth is 2 (N-1)^2 (the z +-2 taps).  Writes the interior of u;
 * boundary entries of u are left as they are.
 * ---------------------------------------------------------------------- */
int orc_dsolve(int N, int bc_kind, const double *fh, double *u) {
    int i, j, k, t;
    size_t n, bw, w, r, c, col;
    double s, *band, *x;
    if (N < 4 || (bc_kind != 1 && bc_kind != 2) || !fh || !u) return ORC_ERR_ARG;
    n = (size_t)(N - 1) * (size_t)(N - 1) * (size_t)(N - 1);
    bw = 2 * (size_t)(N - 1) * (size_t)(N - 1);
    w = 2 * bw + 1;
    s = ghost_sign(bc_kind);
    band = (double *)calloc(n * w, sizeof(double));  /* band[r*w + (c - r + bw)] = A[r][c] */
    x = (double *)malloc(n * sizeof(double));
    if (!band || !x) { free(band); free(x); return ORC_ERR_OOM; }
    for (k = 1; k <= N - 1; ++k)
        for (j = 1; j <= N - 1; ++j)
            for (i = 1; i <= N - 1; ++i) {
                size_t row = uidx(N, i, j, k);
                x[row] = fh[nidx(N, i, j, k)];
                for (t = 0; t < 25; ++t) {
                    orc_tapinfo ti = classify(N, i, j, k, &TAPS[t]);
                    if (ti.kind == TAP_UNKNOWN)
                        band[row * w + (uidx(N, ti.qi, ti.qj, ti.qk) + bw - row)] += TAPS[t].c;
                    else if (ti.kind == TAP_GHOST)
                        band[row * w + (uidx(N, ti.qi, ti.qj, ti.qk) + bw - row)] += s * TAPS[t].c;
                }
            }
    /* forward elimination */
    for (c = 0; c < n; ++c) {
        double piv = band[c * w + bw];
        size_t rend = c + bw < n - 1 ? c + bw : n - 1;
        if (piv == 0.0 || !isfinite(piv)) { free(band); free(x); return ORC_ERR_PIVOT; }
        for (r = c + 1; r <= rend; ++r) {
            double l = band[r * w + (c + bw - r)] / piv;
            if (l == 0.0) continue;
            band[r * w + (c + bw - r)] = 0.0;
            for (col = c + 1; col <= rend; ++col)
                band[r * w + (col + bw - r)] -= l * band[c * w + (col + bw - c)];
            x[r] -= l * x[c];
        }
    }
    /* back substitution */
    for (r = n; r-- > 0;) {
        size_t cend = r + bw < n - 1 ? r + bw : n - 1;
        double acc = x[r];
        for (col = r + 1; col <= cend; ++col) acc -= band[r * w + (col + bw - r)] * x[col];
        x[r] = acc / band[r * w + bw];
    }
    for (k = 1; k <= N - 1; ++k)
        for (j = 1; j <= N - 1; ++j)
            for (i = 1; i <= N - 1; ++i) u[nidx(N, i, j, k)] = x[uidx(N, i, j, k)];
    free(band);
    free(x);
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Vector helpers over interior nodes.
 * ---------------------------------------------------------------------- */
static double idot(int N, const double *a, const double *b) {
    int i, j, k;
    double s = 0.0;
    for (k = 1; k <= N - 1; ++k)
        for (j = 1; j <= N - 1; ++j)
            for (i = 1; i <= N - 1; ++i) s += a[nidx(N, i, j, k)] * b[nidx(N, i, j, k)];
    return s;
}

/* ||f_h - A_h u||_2 over the unknowns (the true-residual test of Alg. 1). */
double orc_residual_norm(int N, int bc_kind, const double *fh, const double *u) {
    size_t total = (size_t)(N + 1) * (size_t)(N + 1) * (size_t)(N + 1), p;
    double *au = (double *)malloc(total * sizeof(double)), s;
    if (!au) return -1.0;
    orc_stencil_apply(N, bc_kind, 0, u, au);
    for (p = 0; p < total; ++p) au[p] = fh[p] - au[p];
    s = sqrt(idot(N, au, au));
    free(au);
    return s;
}

double orc_interior_norm2(int N, const double *a) { return sqrt(idot(N, a, a)); }

/* ------------------------------------------------------------------------
 * Bi-CG with preconditioner, Alg. 2, in real arithmetic with M = I and the
 * shadow system started from r*_0 = r_0.  The dual iterate x*_k is never
 * used by the method and is not formed.  Stops when the recursively updated
 * residual satisfies ||r_k||_2 <= tol * bnorm, after max_iter iterations,
 * or on a breakdown (rho or sigma exactly zero / not finite).
 * x: node array; its interior is updated, its boundary left alone.
 * ---------------------------------------------------------------------- */
int orc_bicg_shadow(int N, int bc_kind, const double *b, double *x, const double *rs0, double tol,
                    double bnorm, int max_iter, int *iters_out, double *relres_out);

int orc_bicg(int N, int bc_kind, const double *b, double *x, double tol, double bnorm,
             int max_iter, int *iters_out, double *relres_out) {
    return orc_bicg_shadow(N, bc_kind, b, x, NULL, tol, bnorm, max_iter, iters_out, relres_out);
}

/* Alg. 2 with a caller-chosen shadow residual r*_0 (line 2 of the algorithm
 * leaves x*_0 and b* free, i.e. any r*_0 with (r_0, r*_0) != 0); rs0 = NULL
 * takes r*_0 = r_0. */
int orc_bicg_shadow(int N, int bc_kind, const double *b, double *x, const double *rs0, double tol,
                    double bnorm, int max_iter, int *iters_out, double *relres_out) {
    size_t total = (size_t)(N + 1) * (size_t)(N + 1) * (size_t)(N + 1), q;
    double *r, *rs, *p, *ps, *Ap, *Atps;
    double rho, rho_new, sigma, alpha, beta, rnorm;
    int it = 0, status = ORC_OK, i, j, k;
    if (N < 4 || !b || !x) return ORC_ERR_ARG;
    r = (double *)calloc(total, sizeof(double));
    rs = (double *)calloc(total, sizeof(double));
    p = (double *)calloc(total, sizeof(double));
    ps = (double *)calloc(total, sizeof(double));
    Ap = (double *)calloc(total, sizeof(double));
    Atps = (double *)calloc(total, sizeof(double));
    if (!r || !rs || !p || !ps || !Ap || !Atps) { status = ORC_ERR_OOM; goto done; }

    /* r_0 = b - A x_0;  r*_0 = r_0;  p_0 = M^{-1} r_0;  p*_0 = r*_0 M^{-1} */
    orc_stencil_apply(N, bc_kind, 0, x, Ap);
    for (k = 1; k <= N - 1; ++k)
        for (j = 1; j <= N - 1; ++j)
            for (i = 1; i <= N - 1; ++i) {
                q = nidx(N, i, j, k);
                r[q] = b[q] - Ap[q];
                rs[q] = rs0 ? rs0[q] : r[q];
                p[q] = r[q];
                ps[q] = rs[q];
            }
    rho = idot(N, rs, r);
    rnorm = sqrt(idot(N, r, r));
    while (rnorm > tol * bnorm && it < max_iter) {
        if (rho == 0.0 || !isfinite(rho)) { status = ORC_ERR_BREAKDOWN; break; }
        orc_stencil_apply(N, bc_kind, 0, p, Ap);     /* A p_k        */
        orc_stencil_apply(N, bc_kind, 1, ps, Atps);  /* (p*_k A)^T   */
        sigma = idot(N, ps, Ap);
        if (sigma == 0.0 || !isfinite(sigma)) { status = ORC_ERR_BREAKDOWN; break; }
        alpha = rho / sigma;
#pragma omp parallel for num_threads(orc_threads) private(i, j, q) schedule(static)
        for (k = 1; k <= N - 1; ++k)
            for (j = 1; j <= N - 1; ++j)
                for (i = 1; i <= N - 1; ++i) {
                    q = nidx(N, i, j, k);
                    x[q] = x[q] + alpha * p[q];
                    r[q] = r[q] - alpha * Ap[q];
                    rs[q] = rs[q] - alpha * Atps[q];
                }
        rho_new = idot(N, rs, r);
        beta = rho_new / rho;
#pragma omp parallel for num_threads(orc_threads) private(i, j, q) schedule(static)
        for (k = 1; k <= N - 1; ++k)
            for (j = 1; j <= N - 1; ++j)
                for (i = 1; i <= N - 1; ++i) {
                    q = nidx(N, i, j, k);
                    p[q] = r[q] + beta * p[q];
                    ps[q] = rs[q] + beta * ps[q];
                }
        rho = rho_new;
        rnorm = sqrt(idot(N, r, r));
        ++it;
    }
done:
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = bnorm > 0.0 ? rnorm / bnorm : rnorm;
    free(r); free(rs); free(p); free(ps); free(Ap); free(Atps);
    return status;
}

/* ------------------------------------------------------------------------
 * EXP_finite (Sec. 4.2.2 and 4.2.3, Steps 1-5): third-order approximation
 * w of the FD solution on the fine grid (Nf intervals) from the FD
 * solutions u1 (Nf/2 intervals) and u0 (Nf/4 intervals).  Each cell of the
 * coarsest of the three grids holds 5x5x5 fine nodes; Steps 1-4 give the
 * 27 nodes it shares with the middle grid, Step 5 the other 98 by
 * tri-quadratic Lagrange interpolation, eqs. (inter)-(iinter).  Every fine
 * node is produced this way, boundary nodes included: the distances
 * ||w_h - u_h||_2 printed in Tables 1-4 are reproduced only when w_h keeps
 * the interpolated values on the boundary (the FD solution u_h carries the
 * Dirichlet data there).  The unknowns of the next Bi-CG solve are the
 * interior nodes, so the boundary values of w never enter the iteration.
 * ---------------------------------------------------------------------- */

/* Lagrange basis of degree 2 on the nodes 0, 1/2, 1, eq. (iinter) */
static double lagrange2(int a, double xi) {
    static const double nodes[3] = {0.0, 0.5, 1.0};
    double v = 1.0;
    int m;
    for (m = 0; m < 3; ++m)
        if (m != a) v *= (xi - nodes[m]) / (nodes[a] - nodes[m]);
    return v;
}

int orc_exp_finite(int Nf, const double *u1, const double *u0, double *w) {
    int N1, N0, ci, cj, ck, a, b, c, i, j, k;
    if (Nf < 8 || Nf % 4 || !u1 || !u0 || !w) return ORC_ERR_ARG;
    N1 = Nf / 2;
    N0 = Nf / 4;
    for (ck = 0; ck < N0; ++ck)
        for (cj = 0; cj < N0; ++cj)
            for (ci = 0; ci < N0; ++ci) {
                /* W[c][b][a]: the 27 values on the middle-grid nodes of this
                 * cell, local middle-grid offsets a,b,c in {0,1,2} */
                double W[3][3][3];
                double d[2][2][2];  /* u1 - u0 at the 8 corners */
                int ox = 2 * ci, oy = 2 * cj, oz = 2 * ck;  /* cell origin, middle grid */
                for (c = 0; c < 2; ++c)
                    for (b = 0; b < 2; ++b)
                        for (a = 0; a < 2; ++a)
                            d[c][b][a] = u1[nidx(N1, ox + 2 * a, oy + 2 * b, oz + 2 * c)] -
                                         u0[nidx(N0, ci + a, cj + b, ck + c)];
                /* Step 1: corners, eq. (secfff): w = (5 u1 - u0) / 4 */
                for (c = 0; c < 2; ++c)
                    for (b = 0; b < 2; ++b)
                        for (a = 0; a < 2; ++a)
                            W[2 * c][2 * b][2 * a] =
                                (5.0 * u1[nidx(N1, ox + 2 * a, oy + 2 * b, oz + 2 * c)] -
                                 u0[nidx(N0, ci + a, cj + b, ck + c)]) / 4.0;
                /* Step 2: the 12 edge midpoints, eq. (bfsec):
                 * w_mid = u1_mid + (1/8) (u1 - u0 at both ends of the edge) */
                for (c = 0; c < 2; ++c)
                    for (b = 0; b < 2; ++b)  /* x-edges */
                        W[2 * c][2 * b][1] = u1[nidx(N1, ox + 1, oy + 2 * b, oz + 2 * c)] +
                                             (d[c][b][0] + d[c][b][1]) / 8.0;
                for (c = 0; c < 2; ++c)
                    for (a = 0; a < 2; ++a)  /* y-edges */
                        W[2 * c][1][2 * a] = u1[nidx(N1, ox + 2 * a, oy + 1, oz + 2 * c)] +
                                             (d[c][0][a] + d[c][1][a]) / 8.0;
                for (b = 0; b < 2; ++b)
                    for (a = 0; a < 2; ++a)  /* z-edges */
                        W[1][2 * b][2 * a] = u1[nidx(N1, ox + 2 * a, oy + 2 * b, oz + 1)] +
                                             (d[0][b][a] + d[1][b][a]) / 8.0;
                /* Step 3: face centres, the mean of eq. (bfsec) along the two
                 * face diagonals */
                for (c = 0; c < 2; ++c) {  /* faces normal to z */
                    double um = u1[nidx(N1, ox + 1, oy + 1, oz + 2 * c)];
                    double e1 = um + (d[c][0][0] + d[c][1][1]) / 8.0;
                    double e2 = um + (d[c][0][1] + d[c][1][0]) / 8.0;
                    W[2 * c][1][1] = (e1 + e2) / 2.0;
                }
                for (b = 0; b < 2; ++b) {  /* faces normal to y */
                    double um = u1[nidx(N1, ox + 1, oy + 2 * b, oz + 1)];
                    double e1 = um + (d[0][b][0] + d[1][b][1]) / 8.0;
                    double e2 = um + (d[0][b][1] + d[1][b][0]) / 8.0;
                    W[1][2 * b][1] = (e1 + e2) / 2.0;
                }
                for (a = 0; a < 2; ++a) {  /* faces normal to x */
                    double um = u1[nidx(N1, ox + 2 * a, oy + 1, oz + 1)];
                    double e1 = um + (d[0][0][a] + d[1][1][a]) / 8.0;
                    double e2 = um + (d[0][1][a] + d[1][0][a]) / 8.0;
                    W[1][1][2 * a] = (e1 + e2) / 2.0;
                }
                /* Step 4: body centre, the mean of eq. (bfsec) along the four
                 * space diagonals */
                {
                    double um = u1[nidx(N1, ox + 1, oy + 1, oz + 1)];
                    double e1 = um + (d[0][0][0] + d[1][1][1]) / 8.0;
                    double e2 = um + (d[0][0][1] + d[1][1][0]) / 8.0;
                    double e3 = um + (d[0][1][0] + d[1][0][1]) / 8.0;
                    double e4 = um + (d[0][1][1] + d[1][0][0]) / 8.0;
                    W[1][1][1] = (e1 + e2 + e3 + e4) / 4.0;
                }
                /* Step 5: tri-quadratic interpolation at the 125 fine nodes of
                 * the cell, natural coordinates xi = 0, 1/4, 1/2, 3/4, 1 */
                for (k = 0; k <= 4; ++k)
                    for (j = 0; j <= 4; ++j)
                        for (i = 0; i <= 4; ++i) {
                            double xi = i / 4.0, eta = j / 4.0, zeta = k / 4.0, v = 0.0;
                            for (c = 0; c < 3; ++c)
                                for (b = 0; b < 3; ++b)
                                    for (a = 0; a < 3; ++a)
                                        v += lagrange2(a, xi) * lagrange2(b, eta) * lagrange2(c, zeta) * W[c][b][a];
                            w[nidx(Nf, 4 * ci + i, 4 * cj + j, 4 * ck + k)] = v;
                        }
            }
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * EXP_true (Sec. 4.2.1, Alg. 1's final extrapolation): extrapolated solution on the
 * finest grid from u_h (Nf intervals) and u_2h (Nf/2 intervals).
 * At nodes shared with the coarse grid, eq. (t1): (4 u_h - u_2h) / 3.
 * Elsewhere the paper prints the 1D midpoint rule, eq. (chenlin):
 *   u_h,mid + (1/6) (d_left + d_right),  d = u_h - u_2h,
 * which is u_h + (1/3) x (linear interpolation of d).  In 3D a fine node
 * that is a midpoint along m axes lies at the centre of 2^m coarse nodes,
 * and the same rule reads u_h + (1/3) x (mean of d over those nodes).
 * ---------------------------------------------------------------------- */
int orc_exp_true(int Nf, const double *uh, const double *u2h, double *ut) {
    int Nc, i, j, k;
    if (Nf < 4 || Nf % 2 || !uh || !u2h || !ut) return ORC_ERR_ARG;
    Nc = Nf / 2;
    for (k = 0; k <= Nf; ++k)
        for (j = 0; j <= Nf; ++j)
            for (i = 0; i <= Nf; ++i) {
                size_t p = nidx(Nf, i, j, k);
                if (i % 2 == 0 && j % 2 == 0 && k % 2 == 0) {
                    ut[p] = (4.0 * uh[p] - u2h[nidx(Nc, i / 2, j / 2, k / 2)]) / 3.0;  /* eq. (t1) */
                } else {
                    /* coarse nodes around (i,j,k): along an even axis the single
                     * index i/2, along an odd axis both (i-1)/2 and (i+1)/2 */
                    int ia[2], ja[2], ka[2], ni, nj, nk, a, b, c, cnt = 0;
                    double sum = 0.0;
                    if (i % 2) { ia[0] = (i - 1) / 2; ia[1] = (i + 1) / 2; ni = 2; } else { ia[0] = i / 2; ni = 1; }
                    if (j % 2) { ja[0] = (j - 1) / 2; ja[1] = (j + 1) / 2; nj = 2; } else { ja[0] = j / 2; nj = 1; }
                    if (k % 2) { ka[0] = (k - 1) / 2; ka[1] = (k + 1) / 2; nk = 2; } else { ka[0] = k / 2; nk = 1; }
                    for (c = 0; c < nk; ++c)
                        for (b = 0; b < nj; ++b)
                            for (a = 0; a < ni; ++a) {
                                sum += uh[nidx(Nf, 2 * ia[a], 2 * ja[b], 2 * ka[c])] -
                                       u2h[nidx(Nc, ia[a], ja[b], ka[c])];
                                ++cnt;
                            }
                    ut[p] = uh[p] + sum / (3.0 * (double)cnt);
                }
            }
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * EXCMG, Alg. 1.  Levels N_l = n_coarsest * 2^l, l = 0 .. L+1; the finest is
 * n_finest.  f, g1 are node arrays and g2 the faces on the finest grid;
 * every coarser level takes every stride-th value (the grids are nested).
 *
 * Each Bi-CG level runs the WHILE loop of Alg. 1:
 *   while ||A u - f_h||_2 > eps_i ||f_h||_2:  u <- Bi-CG(A, u, f_h)
 * where one Bi-CG call iterates until its recursively updated residual
 * meets eps_i (or max_iter).  The loop also ends when two calls in a row
 * fail to halve the true residual ("stagnated": the floating-point floor),
 * or when the level has used max_total iterations.
 * tol_mode 0: eps_i = tol * 10^(i-L) (Alg. 1's tolerance schedule); 1: eps_i = tol.
 *
 * stats (may be NULL), per level l = 0 .. L+1, 4 doubles each:
 *   [iterations, final true relative residual, Bi-CG calls, stagnated flag]
 * ---------------------------------------------------------------------- */
int orc_excmg(int n_finest, int n_coarsest, int bc_kind, const double *f, const double *g1,
              const double *g2, double tol, int tol_mode, int max_iter, int max_total,
              double *u_h_out, double *u_tilde_out, double *stats) {
    int L, nl, l, status = ORC_OK;
    double **u = NULL;
    if (n_coarsest < 4 || n_finest < 4 * n_coarsest || (bc_kind != 1 && bc_kind != 2) ||
        !f || !g1 || !g2 || !(tol > 0.0))
        return ORC_ERR_ARG;
    /* n_finest = n_coarsest * 2^(L+1), L >= 1 */
    nl = 0;
    {
        int n = n_coarsest;
        while (n < n_finest) { n *= 2; ++nl; }
        if (n != n_finest) return ORC_ERR_ARG;
    }
    L = nl - 1;
    nl = L + 2;
    u = (double **)calloc((size_t)nl, sizeof(double *));
    if (!u) return ORC_ERR_OOM;
    for (l = 0; l < nl; ++l) {
        int N = n_coarsest << l;
        int stride = n_finest / N;
        size_t tot = (size_t)(N + 1) * (size_t)(N + 1) * (size_t)(N + 1);
        size_t ftot = 6 * (size_t)(N + 1) * (size_t)(N + 1);
        double *fl = (double *)malloc(tot * sizeof(double));
        double *g1l = (double *)malloc(tot * sizeof(double));
        double *g2l = (double *)malloc(ftot * sizeof(double));
        double *fh = (double *)malloc(tot * sizeof(double));
        double eps_i, fnorm, rel;
        int iters = 0, calls = 0, stag = 0, bad = 0;
        u[l] = (double *)calloc(tot, sizeof(double));
        if (!fl || !g1l || !g2l || !fh || !u[l]) {
            free(fl); free(g1l); free(g2l); free(fh);
            status = ORC_ERR_OOM;
            goto out;
        }
        orc_inject_nodes(n_finest, stride, f, fl);
        orc_inject_nodes(n_finest, stride, g1, g1l);
        orc_inject_faces(n_finest, stride, g2, g2l);
        orc_assemble_rhs(N, bc_kind, fl, g1l, g2l, fh);
        fnorm = orc_interior_norm2(N, fh);
        if (l <= 1) {
            /* Alg. 1's direct solves: DSOLVE on the two coarsest grids */
            memcpy(u[l], g1l, tot * sizeof(double));
            status = orc_dsolve(N, bc_kind, fh, u[l]);
            rel = fnorm > 0.0 ? orc_residual_norm(N, bc_kind, fh, u[l]) / fnorm : 0.0;
        } else {
            int i = l - 1;  /* Alg. 1 loop counter, 1..L */
            eps_i = tol_mode == 0 ? tol * pow(10.0, (double)(i - L)) : tol;
            /* Alg. 1's initial guess: w_h = EXP_finite(u_2h, u_4h) */
            status = orc_exp_finite(N, u[l - 1], u[l - 2], u[l]);
            /* the FD solution carries the Dirichlet data g1 on the boundary
             * (Sec. 2); the interior of w_h is the initial guess */
            {
                int a, b, c;
                for (c = 0; c <= N; ++c)
                    for (b = 0; b <= N; ++b)
                        for (a = 0; a <= N; ++a)
                            if (a == 0 || a == N || b == 0 || b == N || c == 0 || c == N)
                                u[l][nidx(N, a, b, c)] = g1l[nidx(N, a, b, c)];
            }
            rel = fnorm > 0.0 ? orc_residual_norm(N, bc_kind, fh, u[l]) / fnorm : 0.0;
            while (status == ORC_OK && rel > eps_i && iters < max_total) {
                int it = 0;
                double rr, prev = rel;
                int cap = max_iter < max_total - iters ? max_iter : max_total - iters;
                status = orc_bicg(N, bc_kind, fh, u[l], eps_i, fnorm, cap, &it, &rr);
                iters += it;
                ++calls;
                rel = orc_residual_norm(N, bc_kind, fh, u[l]) / fnorm;
                if (rel > 0.5 * prev) {
                    if (++bad >= 2) { stag = 1; break; }
                } else {
                    bad = 0;
                }
            }
        }
        if (stats) {
            stats[4 * l + 0] = iters;
            stats[4 * l + 1] = rel;
            stats[4 * l + 2] = calls;
            stats[4 * l + 3] = stag;
        }
        free(fl); free(g1l); free(g2l); free(fh);
        if (status != ORC_OK) goto out;
    }
    {
        int Nf = n_finest;
        size_t tot = (size_t)(Nf + 1) * (size_t)(Nf + 1) * (size_t)(Nf + 1);
        if (u_h_out) memcpy(u_h_out, u[nl - 1], tot * sizeof(double));
        /* Alg. 1's final extrapolation */
        if (u_tilde_out) status = orc_exp_true(Nf, u[nl - 1], u[nl - 2], u_tilde_out);
    }
out:
    for (l = 0; l < nl; ++l) free(u[l]);
    free(u);
    return status;
}

/* Discrete norms of e = a - b as the error columns of Tables 1-5 use them:
 * out[0] = sqrt(sum e^2 / (N+1)^3) over all (N+1)^3 nodes (the root mean
 * square; with this normalisation the oracle reproduces the printed 32^3
 * rows of Tables 1-4 to the printed three digits), out[1] = max |e|. */
void orc_error_norms(int N, const double *a, const double *b, double *out) {
    size_t total = (size_t)(N + 1) * (size_t)(N + 1) * (size_t)(N + 1), p;
    double s = 0.0, m = 0.0;
    for (p = 0; p < total; ++p) {
        double e = a[p] - b[p];
        s += e * e;
        if (fabs(e) > m) m = fabs(e);
    }
    out[0] = sqrt(s / (double)total);
    out[1] = m;
}
