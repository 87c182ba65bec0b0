/*
 * Plain FP64 CPU oracle of the two-dimensional variant of the problem,
 * eq. (bvp2d): Delta^2 u = f on (0,1)^2 with Dirichlet data of the first kind
 * (u = g1, du/dn = g2) or the second kind (u = g1, d2u/dn2 = g2).
 *
 * TEST INFRASTRUCTURE ONLY, like excmg_oracle.c: nothing in the product path
 * links, loads or calls it.  It shares no code with the CUDA sources.
 *
 * The scheme is the 2D counterpart of Sec. 2: the paper names the 13-point
 * discretisation of the 2D biharmonic equation but prints no stencil; the one
 * taken here is the 13-point scheme that is to eq. (bvp2d) what eq. (method1)
 * is to eq. (bvp):
 *     20 u_{i,j} - 8 (u_{i-1,j} + u_{i+1,j} + u_{i,j-1} + u_{i,j+1})
 *     + (u_{i-2,j} + u_{i+2,j} + u_{i,j-2} + u_{i,j+2})
 *     + 2 (u_{i-1,j-1} + u_{i-1,j+1} + u_{i+1,j-1} + u_{i+1,j+1}) = h^4 f_{i,j}
 * with the fictitious nodes one step outside the square folded onto their
 * mirrors by the reflection formulas of Sec. 2 applied along the crossing
 * axis (first kind: ghost = mirror + 2h du/dn; second kind: ghost =
 * 2 u_boundary - mirror + h^2 d2u/dn2), known values moved to the right-hand
 * side.  Alg. 1 and Alg. 2 are as in 3D; the transfer steps are the 2D forms
 * of Sec. 4.2: Richardson extrapolation (secfff) at the coarse nodes, the
 * edge rule (bfsec) at edge midpoints, the mean of the two diagonal rules at
 * cell centres, bi-quadratic Lagrange interpolation at the fine nodes, and
 * EXP_true with bilinear interpolation of u_h - u_2h.
 *
 * Layout: node arrays of (N+1)^2 doubles, x fastest: idx = j*(N+1) + i.
 * g2: 4 edges of (N+1) doubles, edges x=0, x=1, y=0, y=1, indexed by the
 * other coordinate.  FP64, compiled with -ffp-contract=off.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC2_OK 0
#define ORC2_ERR_ARG (-1)
#define ORC2_ERR_OOM (-2)
#define ORC2_ERR_BREAKDOWN (-3)
#define ORC2_ERR_PIVOT (-8)

static size_t n2(int N, int i, int j) { return (size_t)j * (size_t)(N + 1) + (size_t)i; }

typedef struct {
    int dx, dy;
    double c;
} orc2_tap;

/* the 13 taps, in the order of the scheme as written above */
static const orc2_tap TAPS2[13] = {
    {0, 0, 20.0},
    {-1, 0, -8.0}, {1, 0, -8.0}, {0, -1, -8.0}, {0, 1, -8.0},
    {-2, 0, 1.0},  {2, 0, 1.0},  {0, -2, 1.0},  {0, 2, 1.0},
    {-1, -1, 2.0}, {-1, 1, 2.0}, {1, -1, 2.0},  {1, 1, 2.0},
};

enum { T2_UNKNOWN = 0, T2_BOUNDARY = 1, T2_GHOST = 2 };

typedef struct {
    int kind;
    int qi, qj;   /* unknown column (the mirror for a ghost) */
    int bi, bj;   /* boundary node of the datum              */
    int edge;     /* ghost: edge 0..3                         */
} orc2_tapinfo;

/* How tap t of interior node (i,j) enters the system: an unknown, a known
 * boundary value, or a ghost one step outside an edge. */
static orc2_tapinfo classify2(int N, int i, int j, const orc2_tap *t) {
    orc2_tapinfo r;
    int q[2] = {i + t->dx, j + t->dy};
    int axis = -1, side = 0, a;
    memset(&r, 0, sizeof r);
    for (a = 0; a < 2; ++a) {
        if (q[a] < 0) { axis = a; side = 0; }
        if (q[a] > N) { axis = a; side = 1; }
    }
    if (axis >= 0) {
        int m[2] = {q[0], q[1]}, b[2] = {q[0], q[1]};
        m[axis] = side ? N - 1 : 1;
        b[axis] = side ? N : 0;
        r.kind = T2_GHOST;
        r.qi = m[0]; r.qj = m[1];
        r.bi = b[0]; r.bj = b[1];
        r.edge = 2 * axis + side;
        return r;
    }
    for (a = 0; a < 2; ++a)
        if (q[a] == 0 || q[a] == N) {
            r.kind = T2_BOUNDARY;
            r.bi = q[0]; r.bj = q[1];
            return r;
        }
    r.kind = T2_UNKNOWN;
    r.qi = q[0]; r.qj = q[1];
    return r;
}

static size_t edge_index(int N, int e, int bi, int bj) {
    return (size_t)e * (size_t)(N + 1) + (size_t)(e < 2 ? bj : bi);
}

/* y = A_h u (transpose = 0) or A_h^T u (transpose = 1, formed by scattering
 * rows); interior entries of u are read, boundary entries of y set to 0. */
int orc2d_stencil_apply(int N, int bc_kind, int transpose, const double *u, double *y) {
    int i, j, t;
    const double s = bc_kind == 1 ? 1.0 : -1.0;
    if (N < 4 || (bc_kind != 1 && bc_kind != 2) || !u || !y) return ORC2_ERR_ARG;
    if (!transpose) {
        for (j = 0; j <= N; ++j)
            for (i = 0; i <= N; ++i) {
                double acc = 0.0;
                if (i < 1 || i > N - 1 || j < 1 || j > N - 1) {
                    y[n2(N, i, j)] = 0.0;
                    continue;
                }
                for (t = 0; t < 13; ++t) {
                    orc2_tapinfo ti = classify2(N, i, j, &TAPS2[t]);
                    if (ti.kind == T2_UNKNOWN) acc += TAPS2[t].c * u[n2(N, ti.qi, ti.qj)];
                    else if (ti.kind == T2_GHOST) acc += s * TAPS2[t].c * u[n2(N, ti.qi, ti.qj)];
                }
                y[n2(N, i, j)] = acc;
            }
    } else {
        memset(y, 0, (size_t)(N + 1) * (size_t)(N + 1) * sizeof(double));
        for (j = 1; j <= N - 1; ++j)
            for (i = 1; i <= N - 1; ++i) {
                const double up = u[n2(N, i, j)];
                for (t = 0; t < 13; ++t) {
                    orc2_tapinfo ti = classify2(N, i, j, &TAPS2[t]);
                    if (ti.kind == T2_UNKNOWN) y[n2(N, ti.qi, ti.qj)] += TAPS2[t].c * up;
                    else if (ti.kind == T2_GHOST) y[n2(N, ti.qi, ti.qj)] += s * TAPS2[t].c * up;
                }
            }
    }
    return ORC2_OK;
}

/* f_h = h^4 f minus every known value a row touches (boundary values g1,
 * ghost data through the reflection formulas); boundary entries 0. */
int orc2d_assemble_rhs(int N, int bc_kind, const double *f, const double *g1, const double *g2, double *fh) {
    int i, j, t;
    const double h = 1.0 / (double)N, h4 = h * h * h * h;
    if (N < 4 || (bc_kind != 1 && bc_kind != 2) || !f || !g1 || !g2 || !fh) return ORC2_ERR_ARG;
    for (j = 0; j <= N; ++j)
        for (i = 0; i <= N; ++i) {
            double rhs;
            if (i < 1 || i > N - 1 || j < 1 || j > N - 1) {
                fh[n2(N, i, j)] = 0.0;
                continue;
            }
            rhs = h4 * f[n2(N, i, j)];
            for (t = 0; t < 13; ++t) {
                orc2_tapinfo ti = classify2(N, i, j, &TAPS2[t]);
                if (ti.kind == T2_BOUNDARY) {
                    rhs -= TAPS2[t].c * g1[n2(N, ti.bi, ti.bj)];
                } else if (ti.kind == T2_GHOST) {
                    const double gb = g2[edge_index(N, ti.edge, ti.bi, ti.bj)];
                    const double known = bc_kind == 1 ? 2.0 * h * gb : 2.0 * g1[n2(N, ti.bi, ti.bj)] + h * h * gb;
                    rhs -= TAPS2[t].c * known;
                }
            }
            fh[n2(N, i, j)] = rhs;
        }
    return ORC2_OK;
}

/* the level with Nf / stride intervals takes every stride-th node / edge value */
int orc2d_inject(int Nf, int stride, const double *src, double *dst) {
    const int Nc = Nf / stride;
    int i, j;
    if (stride < 1 || Nf % stride) return ORC2_ERR_ARG;
    for (j = 0; j <= Nc; ++j)
        for (i = 0; i <= Nc; ++i) dst[n2(Nc, i, j)] = src[n2(Nf, i * stride, j * stride)];
    return ORC2_OK;
}

int orc2d_inject_edges(int Nf, int stride, const double *src, double *dst) {
    const int Nc = Nf / stride;
    int e, a;
    if (stride < 1 || Nf % stride) return ORC2_ERR_ARG;
    for (e = 0; e < 4; ++e)
        for (a = 0; a <= Nc; ++a) dst[(size_t)e * (Nc + 1) + a] = src[(size_t)e * (Nf + 1) + (size_t)a * stride];
    return ORC2_OK;
}

/* The dense matrix of A_h over the unknowns (x fastest), column by column
 * from the operator applied to unit vectors. */
int orc2d_assemble_dense(int N, int bc_kind, double *A) {
    const int m = N - 1, n = m * m;
    const size_t tot = (size_t)(N + 1) * (size_t)(N + 1);
    double *e = (double *)calloc(tot, sizeof(double)), *y = (double *)malloc(tot * sizeof(double));
    int c, i, j;
    if (!e || !y) { free(e); free(y); return ORC2_ERR_OOM; }
    for (c = 0; c < n; ++c) {
        const int ci = 1 + c % m, cj = 1 + c / m;
        e[n2(N, ci, cj)] = 1.0;
        orc2d_stencil_apply(N, bc_kind, 0, e, y);
        e[n2(N, ci, cj)] = 0.0;
        for (j = 1; j <= m; ++j)
            for (i = 1; i <= m; ++i) A[(size_t)((j - 1) * m + (i - 1)) * n + c] = y[n2(N, i, j)];
    }
    free(e);
    free(y);
    return ORC2_OK;
}

/* DSOLVE: Gaussian elimination with partial pivoting on the dense matrix. */
int orc2d_dsolve(int N, int bc_kind, const double *fh, double *u) {
    const int m = N - 1, n = m * m;
    double *A = (double *)malloc((size_t)n * n * sizeof(double)), *b = (double *)malloc((size_t)n * sizeof(double));
    int r, c, k, i, j, st = ORC2_OK;
    if (!A || !b) { free(A); free(b); return ORC2_ERR_OOM; }
    orc2d_assemble_dense(N, bc_kind, A);
    for (j = 1; j <= m; ++j)
        for (i = 1; i <= m; ++i) b[(j - 1) * m + (i - 1)] = fh[n2(N, i, j)];
    for (k = 0; k < n && st == ORC2_OK; ++k) {
        int piv = k;
        for (r = k + 1; r < n; ++r)
            if (fabs(A[(size_t)r * n + k]) > fabs(A[(size_t)piv * n + k])) piv = r;
        if (A[(size_t)piv * n + k] == 0.0) { st = ORC2_ERR_PIVOT; break; }
        if (piv != k) {
            double tb = b[k];
            for (c = 0; c < n; ++c) {
                double tt = A[(size_t)k * n + c];
                A[(size_t)k * n + c] = A[(size_t)piv * n + c];
                A[(size_t)piv * n + c] = tt;
            }
            b[k] = b[piv];
            b[piv] = tb;
        }
        for (r = k + 1; r < n; ++r) {
            const double lf = A[(size_t)r * n + k] / A[(size_t)k * n + k];
            if (lf == 0.0) continue;
            for (c = k; c < n; ++c) A[(size_t)r * n + c] -= lf * A[(size_t)k * n + c];
            b[r] -= lf * b[k];
        }
    }
    if (st == ORC2_OK)
        for (k = n - 1; k >= 0; --k) {
            double acc = b[k];
            for (c = k + 1; c < n; ++c) acc -= A[(size_t)k * n + c] * b[c];
            b[k] = acc / A[(size_t)k * n + k];
        }
    if (st == ORC2_OK)
        for (j = 1; j <= m; ++j)
            for (i = 1; i <= m; ++i) u[n2(N, i, j)] = b[(j - 1) * m + (i - 1)];
    free(A);
    free(b);
    return st;
}

static double idot2(int N, const double *a, const double *b) {
    int i, j;
    double s = 0.0;
    for (j = 1; j <= N - 1; ++j)
        for (i = 1; i <= N - 1; ++i) s += a[n2(N, i, j)] * b[n2(N, i, j)];
    return s;
}

double orc2d_residual_norm(int N, int bc_kind, const double *fh, const double *u) {
    const size_t tot = (size_t)(N + 1) * (size_t)(N + 1);
    double *au = (double *)malloc(tot * sizeof(double)), s;
    size_t p;
    if (!au) return -1.0;
    orc2d_stencil_apply(N, bc_kind, 0, u, au);
    for (p = 0; p < tot; ++p) au[p] = fh[p] - au[p];
    s = sqrt(idot2(N, au, au));
    free(au);
    return s;
}

double orc2d_interior_norm2(int N, const double *a) { return sqrt(idot2(N, a, a)); }

/* Alg. 2 with M = I and r*_0 = r_0 on the 2D system, as orc_bicg. */
int orc2d_bicg(int N, int bc_kind, const double *b, double *x, double tol, double bnorm, int max_iter,
               int *iters_out, double *relres_out) {
    const size_t tot = (size_t)(N + 1) * (size_t)(N + 1);
    double *r = (double *)calloc(tot, sizeof(double)), *rs = (double *)calloc(tot, sizeof(double));
    double *p = (double *)calloc(tot, sizeof(double)), *ps = (double *)calloc(tot, sizeof(double));
    double *Ap = (double *)calloc(tot, sizeof(double)), *Atps = (double *)calloc(tot, sizeof(double));
    double rho, rho_new, sigma, alpha, beta, rnorm = 0.0;
    int it = 0, status = ORC2_OK, i, j;
    size_t q;
    if (!r || !rs || !p || !ps || !Ap || !Atps) { status = ORC2_ERR_OOM; goto done; }
    orc2d_stencil_apply(N, bc_kind, 0, x, Ap);
    for (j = 1; j <= N - 1; ++j)
        for (i = 1; i <= N - 1; ++i) {
            q = n2(N, i, j);
            r[q] = b[q] - Ap[q];
            rs[q] = r[q];
            p[q] = r[q];
            ps[q] = rs[q];
        }
    rho = idot2(N, rs, r);
    rnorm = sqrt(idot2(N, r, r));
    while (rnorm > tol * bnorm && it < max_iter) {
        if (rho == 0.0 || !isfinite(rho)) { status = ORC2_ERR_BREAKDOWN; break; }
        orc2d_stencil_apply(N, bc_kind, 0, p, Ap);
        orc2d_stencil_apply(N, bc_kind, 1, ps, Atps);
        sigma = idot2(N, ps, Ap);
        if (sigma == 0.0 || !isfinite(sigma)) { status = ORC2_ERR_BREAKDOWN; break; }
        alpha = rho / sigma;
        for (j = 1; j <= N - 1; ++j)
            for (i = 1; i <= N - 1; ++i) {
                q = n2(N, i, j);
                x[q] = x[q] + alpha * p[q];
                r[q] = r[q] - alpha * Ap[q];
                rs[q] = rs[q] - alpha * Atps[q];
            }
        rho_new = idot2(N, rs, r);
        beta = rho_new / rho;
        for (j = 1; j <= N - 1; ++j)
            for (i = 1; i <= N - 1; ++i) {
                q = n2(N, i, j);
                p[q] = r[q] + beta * p[q];
                ps[q] = rs[q] + beta * ps[q];
            }
        rho = rho_new;
        rnorm = sqrt(idot2(N, r, r));
        ++it;
    }
done:
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = bnorm > 0.0 ? rnorm / bnorm : rnorm;
    free(r); free(rs); free(p); free(ps); free(Ap); free(Atps);
    return status;
}

/* Lagrange basis of degree 2 on 0, 1/2, 1 */
static double lag2(int a, double xi) {
    static const double nodes[3] = {0.0, 0.5, 1.0};
    double v = 1.0;
    int m;
    for (m = 0; m < 3; ++m)
        if (m != a) v *= (xi - nodes[m]) / (nodes[a] - nodes[m]);
    return v;
}

/* EXP_finite in 2D: on each cell of the coarsest grid (4h wide) the 9 nodes
 * it shares with the middle grid get, from d = u1 - u0 at the cell corners,
 *   corners:         u1 + d / 4                       (eq. (secfff))
 *   edge midpoints:  u1 + (d_a + d_b) / 8             (eq. (bfsec))
 *   centre:          mean of the two diagonal rules u1 + (d_a + d_b) / 8
 * and the 25 fine nodes of the cell the bi-quadratic Lagrange interpolant of
 * those 9 values.  Every fine node is produced, boundary nodes included. */
int orc2d_exp_finite(int Nf, const double *u1, const double *u0, double *w) {
    const int N1 = Nf / 2, N0 = Nf / 4;
    int ci, cj, a, b, i, j;
    if (Nf < 8 || Nf % 4 || !u1 || !u0 || !w) return ORC2_ERR_ARG;
    for (cj = 0; cj < N0; ++cj)
        for (ci = 0; ci < N0; ++ci) {
            double W[3][3], d[2][2];
            for (b = 0; b < 2; ++b)
                for (a = 0; a < 2; ++a)
                    d[b][a] = u1[n2(N1, 2 * (ci + a), 2 * (cj + b))] - u0[n2(N0, ci + a, cj + b)];
            for (b = 0; b < 3; ++b)
                for (a = 0; a < 3; ++a) {
                    const double base = u1[n2(N1, 2 * ci + a, 2 * cj + b)];
                    if (a != 1 && b != 1) {
                        W[b][a] = base + d[b / 2][a / 2] / 4.0;
                    } else if (a == 1 && b != 1) {
                        W[b][a] = base + (d[b / 2][0] + d[b / 2][1]) / 8.0;
                    } else if (b == 1 && a != 1) {
                        W[b][a] = base + (d[0][a / 2] + d[1][a / 2]) / 8.0;
                    } else {
                        const double diag1 = base + (d[0][0] + d[1][1]) / 8.0;
                        const double diag2 = base + (d[0][1] + d[1][0]) / 8.0;
                        W[b][a] = (diag1 + diag2) / 2.0;
                    }
                }
            for (j = 0; j <= 4; ++j)
                for (i = 0; i <= 4; ++i) {
                    const double xi = i / 4.0, eta = j / 4.0;
                    double v = 0.0;
                    for (b = 0; b < 3; ++b)
                        for (a = 0; a < 3; ++a) v += W[b][a] * lag2(a, xi) * lag2(b, eta);
                    w[n2(Nf, 4 * ci + i, 4 * cj + j)] = v;
                }
        }
    return ORC2_OK;
}

/* EXP_true in 2D: u~ = u_h + (1/3) * bilinear interpolation of u_h - u_2h. */
int orc2d_exp_true(int Nf, const double *uh, const double *u2h, double *ut) {
    const int Nc = Nf / 2;
    int i, j;
    if (Nf < 4 || Nf % 2 || !uh || !u2h || !ut) return ORC2_ERR_ARG;
    for (j = 0; j <= Nf; ++j)
        for (i = 0; i <= Nf; ++i) {
            const int i0 = i / 2, j0 = j / 2, i1 = (i + 1) / 2, j1 = (j + 1) / 2;
            const double d00 = uh[n2(Nf, 2 * i0, 2 * j0)] - u2h[n2(Nc, i0, j0)];
            const double d10 = uh[n2(Nf, 2 * i1, 2 * j0)] - u2h[n2(Nc, i1, j0)];
            const double d01 = uh[n2(Nf, 2 * i0, 2 * j1)] - u2h[n2(Nc, i0, j1)];
            const double d11 = uh[n2(Nf, 2 * i1, 2 * j1)] - u2h[n2(Nc, i1, j1)];
            const double dd = (d00 + d10 + d01 + d11) / 4.0;
            ut[n2(Nf, i, j)] = uh[n2(Nf, i, j)] + dd / 3.0;
        }
    return ORC2_OK;
}

/* Alg. 1 in 2D; arguments and stats as orc_excmg. */
int orc2d_excmg(int n_finest, int n_coarsest, int bc_kind, const double *f, const double *g1, const double *g2,
                double tol, int tol_mode, int max_iter, int max_total, double *u_h_out, double *u_tilde_out,
                double *stats) {
    int L, nl = 0, l, status = ORC2_OK, n = n_coarsest;
    double **u = NULL;
    if (n_coarsest < 4 || n_finest < 4 * n_coarsest || (bc_kind != 1 && bc_kind != 2) || !f || !g1 || !g2 ||
        !(tol > 0.0))
        return ORC2_ERR_ARG;
    while (n < n_finest) { n *= 2; ++nl; }
    if (n != n_finest) return ORC2_ERR_ARG;
    L = nl - 1;
    nl = L + 2;
    u = (double **)calloc((size_t)nl, sizeof(double *));
    if (!u) return ORC2_ERR_OOM;
    for (l = 0; l < nl; ++l) {
        const int N = n_coarsest << l, stride = n_finest / N;
        const size_t tot = (size_t)(N + 1) * (size_t)(N + 1);
        double *fl = (double *)malloc(tot * sizeof(double)), *g1l = (double *)malloc(tot * sizeof(double));
        double *g2l = (double *)malloc(4 * (size_t)(N + 1) * sizeof(double));
        double *fh = (double *)malloc(tot * sizeof(double));
        double fnorm, rel;
        int iters = 0, calls = 0, stag = 0, bad = 0;
        u[l] = (double *)calloc(tot, sizeof(double));
        if (!fl || !g1l || !g2l || !fh || !u[l]) {
            free(fl); free(g1l); free(g2l); free(fh);
            status = ORC2_ERR_OOM;
            goto out;
        }
        orc2d_inject(n_finest, stride, f, fl);
        orc2d_inject(n_finest, stride, g1, g1l);
        orc2d_inject_edges(n_finest, stride, g2, g2l);
        orc2d_assemble_rhs(N, bc_kind, fl, g1l, g2l, fh);
        fnorm = orc2d_interior_norm2(N, fh);
        if (l <= 1) {
            memcpy(u[l], g1l, tot * sizeof(double));
            status = orc2d_dsolve(N, bc_kind, fh, u[l]);
            rel = fnorm > 0.0 ? orc2d_residual_norm(N, bc_kind, fh, u[l]) / fnorm : 0.0;
        } else {
            const int i = l - 1;
            const double eps_i = tol_mode == 0 ? tol * pow(10.0, (double)(i - L)) : tol;
            int a, b;
            status = orc2d_exp_finite(N, u[l - 1], u[l - 2], u[l]);
            for (b = 0; b <= N; ++b)
                for (a = 0; a <= N; ++a)
                    if (a == 0 || a == N || b == 0 || b == N) u[l][n2(N, a, b)] = g1l[n2(N, a, b)];
            rel = fnorm > 0.0 ? orc2d_residual_norm(N, bc_kind, fh, u[l]) / fnorm : 0.0;
            while (status == ORC2_OK && rel > eps_i && iters < max_total) {
                int it = 0;
                double rr, prev = rel;
                const int cap = max_iter < max_total - iters ? max_iter : max_total - iters;
                status = orc2d_bicg(N, bc_kind, fh, u[l], eps_i, fnorm, cap, &it, &rr);
                iters += it;
                ++calls;
                rel = orc2d_residual_norm(N, bc_kind, fh, u[l]) / fnorm;
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
        if (status != ORC2_OK) goto out;
    }
    {
        const size_t tot = (size_t)(n_finest + 1) * (size_t)(n_finest + 1);
        if (u_h_out) memcpy(u_h_out, u[nl - 1], tot * sizeof(double));
        if (u_tilde_out) status = orc2d_exp_true(n_finest, u[nl - 1], u[nl - 2], u_tilde_out);
    }
out:
    for (l = 0; l < nl; ++l) free(u[l]);
    free(u);
    return status;
}
