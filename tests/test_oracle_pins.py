"""Pins of the CPU oracle to facts fixed by the paper and by the mathematics.

Each test checks the oracle against something other than itself: a closed
form, an identity proved from the printed formulas, an independent library
construction, a dense direct solve, or numbers printed in the paper's tables
(tests/golden/).  A plausible slip in the oracle (a wrong coefficient or sign,
a swapped index, a dropped term) fails at least one of them.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_1901_05118_gb300 import problems as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def poly3_eval(C, N):
    """Evaluate sum C[a,b,c] x^a y^b z^c on the node grid (shape [k,j,i])."""
    x, y, z = P.Manufactured.axes(N)
    out = np.zeros((N + 1,) * 3)
    for (a, b, c), v in np.ndenumerate(C):
        if v != 0.0:
            out = out + v * x**a * y**b * z**c
    return out


def poly3_deriv(C, axis, m):
    """Coefficient tensor of the m-th derivative along axis (0=x, 1=y, 2=z)."""
    D = np.array(C, dtype=float)
    for _ in range(m):
        n = D.shape[axis]
        if n <= 1:
            return np.zeros_like(D)
        idx = np.arange(1, n, dtype=float)
        sl = [slice(None)] * 3
        sl[axis] = slice(1, None)
        shape = [1, 1, 1]
        shape[axis] = n - 1
        D = D[tuple(sl)] * idx.reshape(shape)
        pad = [(0, 0)] * 3
        pad[axis] = (0, 1)
        D = np.pad(D, pad)
    return D


def bilaplacian(C):
    d4 = [poly3_deriv(C, a, 4) for a in range(3)]
    xxyy = poly3_deriv(poly3_deriv(C, 0, 2), 1, 2)
    xxzz = poly3_deriv(poly3_deriv(C, 0, 2), 2, 2)
    yyzz = poly3_deriv(poly3_deriv(C, 1, 2), 2, 2)
    return d4[0] + d4[1] + d4[2] + 2 * (xxyy + xxzz + yyzz)


def random_poly(rng, deg_total=None, deg_each=None):
    C = np.zeros((6, 6, 6)) if deg_total else np.zeros((deg_each + 1,) * 3)
    for idx in np.ndindex(C.shape):
        if deg_total is not None and sum(idx) > deg_total:
            continue
        C[idx] = rng.uniform(-1, 1)
    return C


def interior(a, lo=1):
    N = a.shape[0] - 1
    return a[lo:N + 1 - lo, lo:N + 1 - lo, lo:N + 1 - lo]


# ------------------------------------------------ P1: the interior stencil
@pytest.mark.parametrize("N", [8, 11])
def test_interior_stencil_exact_on_total_degree_5(N):
    """Eq. (method1) is h^4 times the biharmonic operator applied exactly to
    every polynomial of total degree <= 5 (it is the square of the 7-point
    Laplacian, whose error starts with fourth derivatives).  Checked at rows
    whose 25 taps are all unknowns (3 <= i,j,k <= N-3)."""
    rng = np.random.Generator(np.random.PCG64(11))
    for _ in range(3):
        C = random_poly(rng, deg_total=5)
        u = poly3_eval(C, N)
        y = oracle.stencil_apply(N, 1, u)
        ref = poly3_eval(bilaplacian(C), N) / N**4
        scale = 144 * np.abs(u).max()
        assert np.abs(interior(y, 3) - interior(ref, 3)).max() <= 1e-13 * scale


def test_interior_stencil_detects_degree_6():
    """Negative control: a sixth-degree term (x^6) is NOT reproduced exactly,
    so the previous pin has power to detect a wrong coefficient."""
    N = 10
    C = np.zeros((7, 1, 1))
    C[6, 0, 0] = 1.0
    u = poly3_eval(C, N)
    y = oracle.stencil_apply(N, 1, u)
    ref = poly3_eval(bilaplacian(C), N) / N**4
    assert np.abs(interior(y, 3) - interior(ref, 3)).max() > 1e-9


# ----------------------------- P3 at operator level: closure + right-hand side
@pytest.mark.parametrize("N", [4, 7, 8])
@pytest.mark.parametrize("bc_kind,deg", [(1, 2), (2, 3)])
def test_operator_and_rhs_exact_on_polynomials(N, bc_kind, deg):
    """With first-kind data, the reflection (reflection2) is exact for
    quadratics in the normal direction; with second-kind data, (reflection4)
    is exact for cubics.  The interior scheme is exact for polynomials of
    degree <= 3 in each variable.  Hence A_h u = f_h holds exactly for the
    nodal values of a tri-quadratic (first kind) or tri-cubic (second kind)
    u, which pins the stencil, the ghost folding and the 27 boundary cases
    of the right-hand side together (including the outward sign of du/dn)."""
    rng = np.random.Generator(np.random.PCG64(100 + N + 10 * bc_kind))
    coeffs = [rng.uniform(-1, 1, deg + 1) for _ in range(3)]
    extra = [(rng.uniform(-1, 1), rng.uniform(-1, 1, deg + 1), rng.uniform(-1, 1, deg + 1),
              rng.uniform(-1, 1, deg + 1))]
    prob = P.polynomial(*coeffs, extra=extra)
    f, g1, g2 = prob.data(N, bc_kind)
    fh = oracle.assemble_rhs(N, bc_kind, f, g1, g2)
    u = prob.exact(N)
    Au = oracle.stencil_apply(N, bc_kind, u)
    scale = 144 * np.abs(u).max()
    assert np.abs(interior(Au) - interior(fh)).max() <= 1e-13 * scale


@pytest.mark.parametrize("bc_kind", [1, 2])
def test_rhs_sign_sensitivity(bc_kind):
    """Negative control: flipping the sign of g2 breaks the exactness above."""
    N = 7
    prob = P.polynomial([0.3, 1.0, -0.7], [0.1, 0.5, 0.9], [-0.2, 0.8, 0.4])
    f, g1, g2 = prob.data(N, bc_kind)
    fh = oracle.assemble_rhs(N, bc_kind, f, g1, -g2)
    Au = oracle.stencil_apply(N, bc_kind, prob.exact(N))
    assert np.abs(interior(Au) - interior(fh)).max() > 1e-6


def test_first_kind_not_exact_for_cubics():
    """Negative control: the first-kind reflection is only second-order
    accurate, so a cubic in x leaves a residual at the x-boundary rows."""
    N = 8
    prob = P.polynomial([0.0, 0.0, 0.0, 1.0], [1.0], [1.0])
    f, g1, g2 = prob.data(N, 1)
    fh = oracle.assemble_rhs(N, 1, f, g1, g2)
    Au = oracle.stencil_apply(N, 1, prob.exact(N))
    assert np.abs(interior(Au) - interior(fh)).max() > 1e-6


# ----------------------------------------- P2: structure of the matrix A_h
def dirichlet_laplacian(N):
    """7-point Laplacian [6; -1 x 6] on the (N-1)^3 interior, built from
    Kronecker products (x fastest) -- an independent construction."""
    m = N - 1
    T = sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])
    I = sp.identity(m)
    return (sp.kron(sp.kron(I, I), T) + sp.kron(sp.kron(I, T), I) + sp.kron(sp.kron(T, I), I)).tocsr()


def near_boundary_count(N):
    m = N - 1
    c1 = np.zeros(m)
    c1[0] += 1
    c1[-1] += 1
    cz, cy, cx = np.meshgrid(c1, c1, c1, indexing="ij")
    return (cx + cy + cz).ravel()


@pytest.mark.parametrize("N", [4, 5, 6, 8])
@pytest.mark.parametrize("bc_kind", [1, 2])
def test_matrix_is_square_of_laplacian_plus_diagonal(N, bc_kind):
    """The assembled A_h equals L_D^2 + (1+sigma) diag(c): second kind folds
    each ghost with -1, first kind with +1, and c counts the axes on which a
    node is one step from a face."""
    A = oracle.assemble_dense(N, bc_kind)
    L = dirichlet_laplacian(N)
    sigma = 1.0 if bc_kind == 1 else -1.0
    ref = (L @ L).toarray() + np.diag((1.0 + sigma) * near_boundary_count(N))
    np.testing.assert_array_equal(A, ref)


@pytest.mark.parametrize("N", [4, 6, 8])
@pytest.mark.parametrize("bc_kind", [1, 2])
def test_matrix_symmetric_positive_definite(N, bc_kind):
    """A_h is symmetric positive definite for both kinds of data (the paper
    states otherwise; the reading taken here follows the assembled matrix)."""
    A = oracle.assemble_dense(N, bc_kind)
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0.0


@pytest.mark.parametrize("bc_kind", [1, 2])
def test_apply_and_transpose_match_dense(bc_kind):
    N = 7
    A = oracle.assemble_dense(N, bc_kind)
    u = P.random_field(N, 5)
    ui = interior(u).ravel()
    y = oracle.stencil_apply(N, bc_kind, u)
    yt = oracle.stencil_apply(N, bc_kind, u, transpose=True)
    np.testing.assert_allclose(interior(y).ravel(), A @ ui, rtol=0, atol=1e-12)
    np.testing.assert_allclose(interior(yt).ravel(), A.T @ ui, rtol=0, atol=1e-12)
    # boundary entries of the result are zero, boundary entries of u are ignored
    u2 = u.copy()
    u2[0] = 1e3
    u2[:, :, -1] = -7.0
    y2 = oracle.stencil_apply(N, bc_kind, u2)
    np.testing.assert_array_equal(y2, y)
    mask = np.ones_like(y, dtype=bool)
    mask[1:-1, 1:-1, 1:-1] = False
    assert np.all(y[mask] == 0.0) and np.all(yt[mask] == 0.0)


# ------------------------------------------------------ P4: direct solves
@pytest.mark.parametrize("N", [4, 6, 8])
@pytest.mark.parametrize("bc_kind", [1, 2])
def test_dsolve_matches_dense_lapack(N, bc_kind):
    A = oracle.assemble_dense(N, bc_kind)
    fh = P.random_field(N, 17)
    x = np.linalg.solve(A, interior(fh).ravel())
    u = oracle.dsolve(N, bc_kind, fh, np.zeros_like(fh))
    np.testing.assert_allclose(interior(u).ravel(), x, rtol=1e-12, atol=1e-12 * np.abs(x).max())


# -------------------------------------------------------------- P6: Bi-CG
@pytest.mark.parametrize("bc_kind", [1, 2])
def test_bicg_finite_termination_small(bc_kind):
    """Sec. 5: Bi-CG terminates in at most n steps; n = 27 unknowns at N=4."""
    N = 4
    A = oracle.assemble_dense(N, bc_kind)
    b = P.random_field(N, 3)
    b_int = interior(b).ravel()
    x, it, rel, rc = oracle.bicg(N, bc_kind, b, np.zeros_like(b), 1e-13)
    assert rc == 0 and it <= 27 and rel <= 1e-13
    np.testing.assert_allclose(interior(x).ravel(), np.linalg.solve(A, b_int), rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("bc_kind", [1, 2])
def test_bicg_matches_direct_solve(bc_kind):
    N = 8
    fh = P.random_field(N, 23)
    xd = oracle.dsolve(N, bc_kind, fh, np.zeros_like(fh))
    x, it, rel, rc = oracle.bicg(N, bc_kind, fh, np.zeros_like(fh), 1e-13)
    assert rc == 0 and rel <= 1e-13
    np.testing.assert_allclose(interior(x), interior(xd), rtol=0, atol=1e-10 * np.abs(xd).max())
    # the recursively updated residual agrees with the true one at convergence
    assert oracle.residual_norm(N, bc_kind, fh, x) <= 1e-12 * oracle.interior_norm2(N, fh)


# ------------------------------------------- P5: the level-transfer steps
def test_exp_finite_1d_formulas():
    """For data that vary along x only, Steps 1-5 reduce to the printed 1D
    formulas: (secfff) at coarse nodes, (bfsec) at midpoints, (sifen1) and
    (sifen2) at quarter points."""
    Nf = 16
    rng = np.random.Generator(np.random.PCG64(7))
    a1 = rng.uniform(-1, 1, Nf // 2 + 1)
    a0 = rng.uniform(-1, 1, Nf // 4 + 1)
    u1 = np.broadcast_to(a1[None, None, :], (Nf // 2 + 1,) * 3)
    u0 = np.broadcast_to(a0[None, None, :], (Nf // 4 + 1,) * 3)
    w = oracle.exp_finite(Nf, u1, u0)
    line = w[Nf // 2, Nf // 2, :]
    for j in range(Nf // 4):
        uj1, um1, uk1 = a1[2 * j], a1[2 * j + 1], a1[2 * j + 2]
        uj0, uk0 = a0[j], a0[j + 1]
        base = 4 * j
        assert line[base] == pytest.approx((5 * uj1 - uj0) / 4, abs=1e-14)
        assert line[base + 2] == pytest.approx(um1 + (uj1 - uj0 + uk1 - uk0) / 8, abs=1e-14)
        assert line[base + 1] == pytest.approx(((9 * uj1 + 12 * um1 - uk1) - (3 * uj0 + uk0)) / 16, abs=1e-14)
        assert line[base + 3] == pytest.approx(((9 * uk1 + 12 * um1 - uj1) - (3 * uk0 + uj0)) / 16, abs=1e-14)


def trilinear_field(N, coef):
    x, y, z = P.Manufactured.axes(N)
    a, b, c, d, e, f, g, h = coef
    return np.broadcast_to(a + b * x + c * y + d * z + e * x * y + f * x * z + g * y * z + h * x * y * z,
                           (N + 1,) * 3)


def triquadratic_field(N, C):
    return poly3_eval(C, N)


def test_exp_finite_exact_for_smooth_error_expansion():
    """If u0 = u + a h0^2 and u1 = u + a h1^2 with u tri-quadratic and a
    trilinear (the error expansion (secf) without its O(h^4) part), then
    Steps 1-4 give u + a h2^2 exactly at the 27 middle-grid nodes of every
    cell and Step 5 keeps it exact: w = u + a h2^2 at every fine node."""
    Nf = 16
    rng = np.random.Generator(np.random.PCG64(9))
    C = np.zeros((3, 3, 3))
    for idx in np.ndindex(C.shape):
        C[idx] = rng.uniform(-1, 1)
    coef = rng.uniform(-1, 1, 8)
    h2, h1, h0 = 1 / Nf, 2 / Nf, 4 / Nf
    uf = triquadratic_field(Nf, C) + trilinear_field(Nf, coef) * h2**2
    u1 = triquadratic_field(Nf // 2, C) + trilinear_field(Nf // 2, coef) * h1**2
    u0 = triquadratic_field(Nf // 4, C) + trilinear_field(Nf // 4, coef) * h0**2
    w = oracle.exp_finite(Nf, u1, u0)
    np.testing.assert_allclose(w, uf, rtol=0, atol=1e-13)


def test_exp_finite_cells_agree_on_shared_faces():
    """Neighbouring cells interpolate a shared face from the same nine
    middle-grid values; a random input must give one continuous field whose
    values at middle-grid nodes follow Steps 1-4 (secfff)/(bfsec)."""
    Nf = 8
    u1 = P.random_field(Nf // 2, 1)
    u0 = P.random_field(Nf // 4, 2)
    w = oracle.exp_finite(Nf, u1, u0)
    # coarse nodes: (5 u1 - u0) / 4
    np.testing.assert_allclose(w[::4, ::4, ::4], (5 * u1[::2, ::2, ::2] - u0) / 4, rtol=0, atol=1e-14)
    # x-edge midpoints of the coarse grid: u1_mid + (d_left + d_right) / 8
    d = u1[::2, ::2, ::2] - u0
    np.testing.assert_allclose(w[::4, ::4, 2::4], u1[::2, ::2, 1::2] + (d[:, :, :-1] + d[:, :, 1:]) / 8,
                               rtol=0, atol=1e-14)


def test_excmg_boundary_carries_dirichlet_data():
    prob = P.exp_sum()
    f, g1, g2 = prob.data(16, 1)
    uh, ut, st = oracle.excmg(16, 4, 1, f, g1, g2, 1e-10)
    mask = np.ones_like(uh, dtype=bool)
    mask[1:-1, 1:-1, 1:-1] = False
    np.testing.assert_array_equal(uh[mask], g1[mask])
    np.testing.assert_allclose(ut[mask], g1[mask], rtol=1e-15, atol=0)  # (4g - g)/3 rounds


def test_exp_true_1d_formulas_and_exactness():
    """(t1) at coarse nodes, (chenlin) at midpoints, and exact recovery of u
    from u_h = u + a h^2, u_2h = u + 4 a h^2 (a trilinear)."""
    Nf = 12
    rng = np.random.Generator(np.random.PCG64(4))
    ah = rng.uniform(-1, 1, Nf + 1)
    a2 = rng.uniform(-1, 1, Nf // 2 + 1)
    uh = np.ascontiguousarray(np.broadcast_to(ah[None, None, :], (Nf + 1,) * 3))
    u2h = np.ascontiguousarray(np.broadcast_to(a2[None, None, :], (Nf // 2 + 1,) * 3))
    ut = oracle.exp_true(Nf, uh, u2h)
    line = ut[4, 6, :]
    for j in range(Nf // 2):
        assert line[2 * j] == pytest.approx((4 * ah[2 * j] - a2[j]) / 3, abs=1e-14)
        assert line[2 * j + 1] == pytest.approx(
            ah[2 * j + 1] + (ah[2 * j] - a2[j] + ah[2 * j + 2] - a2[j + 1]) / 6, abs=1e-14)
    C = rng.uniform(-1, 1, (3, 3, 3))
    coef = rng.uniform(-1, 1, 8)
    h = 1 / Nf
    u_f = poly3_eval(C, Nf)
    uh = u_f + trilinear_field(Nf, coef) * h**2
    u2h = poly3_eval(C, Nf // 2) + trilinear_field(Nf // 2, coef) * (2 * h) ** 2
    np.testing.assert_allclose(oracle.exp_true(Nf, uh, u2h), u_f, rtol=0, atol=1e-13)


# --------------------------------------- P3 on the whole solve (Alg. 1)
def test_excmg_exact_for_triquadratic_first_kind():
    """Every level's discrete solution equals the nodal u, so EXP_finite
    returns it exactly and the Bi-CG levels need no iteration."""
    prob = P.polynomial([0.5, -0.3, 0.8], [1.0, 0.2, -0.6], [0.1, 0.7, 0.3])
    f, g1, g2 = prob.data(16, 1)
    uh, ut, st = oracle.excmg(16, 4, 1, f, g1, g2, 1e-12)
    ue = prob.exact(16)
    assert np.abs(uh - ue).max() <= 1e-12
    assert np.abs(ut - ue).max() <= 1e-12
    assert st[2, 0] == 0


def test_excmg_exact_for_tricubic_second_kind():
    prob = P.polynomial([0.5, -0.3, 0.8, 0.4], [1.0, 0.2, -0.6, 0.5], [0.1, 0.7, 0.3, -0.9])
    f, g1, g2 = prob.data(16, 2)
    uh, ut, st = oracle.excmg(16, 4, 2, f, g1, g2, 1e-13)
    ue = prob.exact(16)
    assert np.abs(uh - ue).max() <= 1e-10


# -------------------------------------------- P7: the paper's own numbers
def _levels_32(prob):
    """The paper's setting at 32^3: 8^3 and 16^3 solved directly, then
    EXP_finite to 32^3 (the first Bi-CG level)."""
    sol = {}
    f, g1, g2 = prob.data(32, 1)
    for N in (8, 16):
        s = 32 // N
        fl, g1l, g2l = oracle.inject_nodes(32, s, f), oracle.inject_nodes(32, s, g1), oracle.inject_faces(32, s, g2)
        fh = oracle.assemble_rhs(N, 1, fl, g1l, g2l)
        sol[N] = oracle.dsolve(N, 1, fh, g1l)
    w = oracle.exp_finite(32, sol[16], sol[8])
    uh, ut, st = oracle.excmg(32, 8, 1, f, g1, g2, 1e-11)
    return w, uh, prob.exact(32)


@pytest.mark.parametrize("name", ["paper_p1", "paper_p2", "paper_p3", "paper_p4"])
def test_paper_tables_at_32(name):
    """The 32^3 rows of Tables 1-4: discretisation errors of u_h and the
    distance of the EXP_finite guess w_h from u_h, to the printed 3 digits.
    Norms over all (N+1)^3 nodes (root mean square); w_h keeps its
    interpolated boundary values."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_tables.json")))["problems"][name]["rows"]["32"]
    w, uh, ue = _levels_32(P.by_name(name))
    l2, linf = oracle.error_norms(32, uh, ue)
    wl2, _ = oracle.error_norms(32, w, uh)
    assert l2 == pytest.approx(gold["l2"], rel=0.006)
    assert linf == pytest.approx(gold["linf"], rel=0.006)
    assert wl2 == pytest.approx(gold["wl2"], rel=0.006)


def test_orders_second_and_extrapolated():
    """u_h is second order (Tables 1-5: order ~2); the extrapolated solution
    of Alg. 1's final extrapolation is markedly more accurate."""
    prob = P.sin_pi()
    errs, terrs = [], []
    for nf in (16, 32):
        f, g1, g2 = prob.data(nf, 1)
        uh, ut, st = oracle.excmg(nf, 4, 1, f, g1, g2, 1e-11)
        errs.append(oracle.error_norms(nf, uh, prob.exact(nf))[1])
        terrs.append(oracle.error_norms(nf, ut, prob.exact(nf))[1])
    order = np.log2(errs[0] / errs[1])
    assert 1.9 < order < 2.1
    assert terrs[1] < 0.1 * errs[1]


@pytest.mark.slow
@pytest.mark.parametrize("name", ["paper_p1", "paper_p2"])
def test_paper_tables_at_64(name):
    gold = json.load(open(os.path.join(GOLDEN, "paper_tables.json")))["problems"][name]["rows"]["64"]
    prob = P.by_name(name)
    f, g1, g2 = prob.data(64, 1)
    uh, ut, st = oracle.excmg(64, 8, 1, f, g1, g2, 1e-11)
    l2, linf = oracle.error_norms(64, uh, prob.exact(64))
    assert l2 == pytest.approx(gold["l2"], rel=0.006)
    assert linf == pytest.approx(gold["linf"], rel=0.006)


# -------------------------------------------- the inputs themselves
def test_problem_forcing_terms_match_symbolic():
    """The manufactured f = Laplacian^2 u and the boundary derivatives used as
    inputs agree with a symbolic computation (the printed (force2),
    (force4) included)."""
    sympy = pytest.importorskip("sympy")
    x, y, z = sympy.symbols("x y z")
    exprs = {
        "paper_p1": (1 - sympy.cos(2 * sympy.pi * x)) * (1 - sympy.cos(2 * sympy.pi * y)) * (1 - sympy.cos(2 * sympy.pi * z)),
        "paper_p2": sympy.exp(x * y * z),
        "paper_p3": sympy.sinh(x) * sympy.sinh(y) * sympy.sinh(z),
        "paper_p4": x * y * z * sympy.log(1 + x + y + z),
        "sin_pi": sympy.sin(sympy.pi * x) * sympy.sin(sympy.pi * y) * sympy.sin(sympy.pi * z),
        "exp_sum": sympy.exp(x + y + z),
        "sin2pi_plus_poly": sympy.sin(2 * sympy.pi * x) * sympy.sin(2 * sympy.pi * y) * sympy.sin(2 * sympy.pi * z) + x**2 * y**2 * z**2,
    }
    rng = np.random.Generator(np.random.PCG64(0))
    pts = rng.uniform(0, 1, (5, 3))
    for name, u in exprs.items():
        prob = P.by_name(name)
        lap = lambda e: sympy.diff(e, x, 2) + sympy.diff(e, y, 2) + sympy.diff(e, z, 2)
        f = sympy.lambdify((x, y, z), lap(lap(u)), "numpy")
        gx = sympy.lambdify((x, y, z), [sympy.diff(u, v) for v in (x, y, z)], "numpy")
        hx = sympy.lambdify((x, y, z), [sympy.diff(u, v, 2) for v in (x, y, z)], "numpy")
        for px, py, pz in pts:
            assert prob.f(px, py, pz) == pytest.approx(f(px, py, pz), rel=1e-10, abs=1e-10)
            np.testing.assert_allclose(prob.grad(px, py, pz), gx(px, py, pz), rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(prob.d2(px, py, pz), hx(px, py, pz), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("bc_kind", [1, 2])
def test_bicg_with_chosen_shadow_matches_direct_solve(bc_kind):
    """Alg. 2 leaves the shadow vectors free: any r*_0 with (r_0, r*_0) != 0
    leads to the same solution (here against the direct solve)."""
    N = 8
    fh = P.random_field(N, 61)
    xd = oracle.dsolve(N, bc_kind, fh, np.zeros_like(fh))
    x, it, rel, rc = oracle.bicg(N, bc_kind, fh, np.zeros_like(fh), 1e-13, shadow=P.random_field(N, 62))
    assert rc == 0 and rel <= 1e-13
    np.testing.assert_allclose(interior(x), interior(xd), rtol=0, atol=1e-9 * np.abs(xd).max())


# ------------------------------------- the tolerance schedule of Alg. 1
@pytest.mark.parametrize("bc_kind", [1, 2])
def test_excmg_paper_tolerance_schedule(bc_kind):
    """eps_i = eps * 10^(i - L): level i of L (i = L the finest) stops at a
    true relative residual of at most eps * 10^(i-L), i.e. every coarser
    Bi-CG grid is solved ten times tighter than the next finer one; with the
    uniform schedule every level stops at eps.  A swapped exponent sign would
    leave the coarse levels at 10 eps and fail the first assertion."""
    prob = P.exp_sum()
    n, nc, eps = 64, 4, 1e-5
    f, g1, g2 = prob.data(n, bc_kind)
    _, _, st_p = oracle.excmg(n, nc, bc_kind, f, g1, g2, eps, tol_mode="paper")
    _, _, st_u = oracle.excmg(n, nc, bc_kind, f, g1, g2, eps, tol_mode="uniform")
    levels = st_p.shape[0]                 # grids 4, 8 (direct), 16, 32, 64
    L = levels - 2
    for l in range(2, levels):
        i = l - 1                          # Alg. 1 loop counter 1..L
        eps_i = eps * 10.0 ** (i - L)
        assert st_p[l, 1] <= eps_i, (l, st_p[l, 1], eps_i)
        assert st_u[l, 1] <= eps
        if i < L:   # the tighter coarse levels cost at least as many iterations
            assert st_p[l, 0] >= st_u[l, 0]
    assert st_p[2, 0] > st_u[2, 0]          # the coarsest Bi-CG grid: 100x tighter
    # the uniform schedule does not meet the coarsest level's paper bound
    assert st_u[2, 1] > eps * 10.0 ** (1 - L)


# ------------------------------------- threads change no bit of the oracle
def test_oracle_threads_give_the_same_bits():
    """The operator (A and the scattered A^T), Bi-CG and a whole solve return
    identical bits with one thread and with several (the parallel loops have
    independent iterations; inner products stay sequential)."""
    prob = P.exp_sum()
    N = 24
    u = P.random_field(N, 77)
    f, g1, g2 = prob.data(N, 2)
    out = {}
    for th in (1, 4):
        got = oracle.set_threads(th)
        out[th] = (oracle.stencil_apply(N, 1, u), oracle.stencil_apply(N, 2, u, transpose=True),
                   oracle.bicg(N, 1, u, np.zeros_like(u), 0.0, max_iter=15)[0],
                   oracle.excmg(N, 6, 2, f, g1, g2, 1e-9)[1])
        assert got == th or got == 1
    oracle.set_threads(1)
    for a, b in zip(out[1], out[4]):
        np.testing.assert_array_equal(a, b)
