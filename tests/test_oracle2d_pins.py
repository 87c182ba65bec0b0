"""Pins of the 2D oracle (eq. (bvp2d)) to facts fixed by the mathematics.

The paper names the 13-point discretisation of the 2D problem without
printing it; the oracle takes the 13-point scheme built as eq. (method1) is
built (the square of the five-point Laplacian, with the reflection formulas
of Sec. 2 along each axis).  Each test checks the oracle against something
other than itself: a closed form, an independent sparse construction, LAPACK,
or an exactness property of the scheme or of the transfer steps.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_1901_05118_gb300 import problems as P


def poly2(C, N):
    x, y = P.Manufactured2D.axes(N)
    out = np.zeros((N + 1, N + 1))
    for (a, b), v in np.ndenumerate(C):
        if v:
            out = out + v * x ** a * y ** b
    return out


def bilap2(C):
    """Coefficients of Delta^2 of sum C[a,b] x^a y^b."""
    out = np.zeros_like(C)
    for (a, b), v in np.ndenumerate(C):
        if not v:
            continue
        if a >= 4:
            out[a - 4, b] += v * a * (a - 1) * (a - 2) * (a - 3)
        if b >= 4:
            out[a, b - 4] += v * b * (b - 1) * (b - 2) * (b - 3)
        if a >= 2 and b >= 2:
            out[a - 2, b - 2] += 2 * v * a * (a - 1) * b * (b - 1)
    return out


@pytest.mark.parametrize("N", [9, 12])
def test_interior_13_point_exact_on_total_degree_5(N):
    """A u = h^4 Delta^2 u at every row whose 13 taps are all unknowns
    (3 <= i, j <= N-3), for random polynomials of total degree <= 5."""
    rng = np.random.Generator(np.random.PCG64(5))
    C = np.zeros((6, 6))
    for a in range(6):
        for b in range(6 - a):
            C[a, b] = rng.uniform(-1, 1)
    u = poly2(C, N)
    y = oracle.stencil_apply2d(N, 1, u)
    f = poly2(bilap2(C), N) / N ** 4
    inner = (slice(3, N - 2), slice(3, N - 2))
    scale = 64 * np.abs(u).max()
    assert np.abs(y[inner] - f[inner]).max() <= 1e-13 * scale


def test_interior_13_point_detects_degree_6():
    N = 10
    C = np.zeros((7, 7))
    C[6, 0] = 1.0
    u = poly2(C, N)
    y = oracle.stencil_apply2d(N, 1, u)
    f = poly2(bilap2(C), N) / N ** 4
    inner = (slice(3, N - 2), slice(3, N - 2))
    assert np.abs(y[inner] - f[inner]).max() > 1e-6 * np.abs(f[inner]).max()


@pytest.mark.parametrize("N", [4, 7, 8])
@pytest.mark.parametrize("bc_kind,coef", [(1, ([0.3, -0.7, 0.9], [1.0, 0.4, -0.5])),
                                          (2, ([0.2, 0.5, -0.4, 0.7], [1.0, -0.3, 0.6, 0.25]))])
def test_operator_and_rhs_exact_on_polynomials(N, bc_kind, coef):
    """On every interior row, A u equals the assembled right-hand side for a
    bi-quadratic u with first-kind data and a bi-cubic u with second-kind
    data: the scheme, the reflection formulas (central differences, exact for
    quadratics / cubics in the normal direction) and the moved boundary terms
    are all exact there, near-boundary rows included."""
    prob = P.polynomial_2d(*coef)
    f, g1, g2 = prob.data(N, bc_kind)
    y = oracle.stencil_apply2d(N, bc_kind, prob.exact(N))
    fh = oracle.assemble_rhs2d(N, bc_kind, f, g1, g2)
    np.testing.assert_allclose(y, fh, rtol=0, atol=1e-13 * max(1.0, np.abs(fh).max()))


@pytest.mark.parametrize("bc_kind", [1, 2])
def test_rhs_detects_a_flipped_normal_derivative(bc_kind):
    """Negative control: with g2's sign flipped the identity above fails."""
    N = 8
    prob = P.polynomial_2d([0.3, -0.7, 0.9, 0.2 * (bc_kind - 1)], [1.0, 0.4, -0.5])
    f, g1, g2 = prob.data(N, bc_kind)
    y = oracle.stencil_apply2d(N, bc_kind, prob.exact(N))
    fh = oracle.assemble_rhs2d(N, bc_kind, f, g1, -g2)
    assert np.abs(y - fh).max() > 1e-6


def laplacian_dirichlet_2d(N):
    m = N - 1
    T = sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])
    I = sp.identity(m)
    return (sp.kron(I, T) + sp.kron(T, I)).tocsr()


@pytest.mark.parametrize("N", [4, 6, 9])
@pytest.mark.parametrize("bc_kind", [1, 2])
def test_matrix_is_square_of_laplacian_plus_diagonal(N, bc_kind):
    """A_h = L_D^2 + (1 + sigma) diag(c), c = number of axes on which the node
    is one step from the boundary, sigma = +1 (first kind) / -1 (second)."""
    L = laplacian_dirichlet_2d(N)
    m = N - 1
    idx = np.arange(1, N)
    cx = (idx == 1).astype(float) + (idx == N - 1)
    c = (cx[None, :] + cx[:, None]).ravel()        # unknowns x fastest
    sigma = 1.0 if bc_kind == 1 else -1.0
    ref = (L @ L).toarray() + (1 + sigma) * np.diag(c)
    A = oracle.assemble_dense2d(N, bc_kind)
    np.testing.assert_array_equal(A, ref)
    assert A.shape == (m * m, m * m)


@pytest.mark.parametrize("bc_kind", [1, 2])
def test_matrix_symmetric_positive_definite_and_transpose(bc_kind):
    N = 8
    A = oracle.assemble_dense2d(N, bc_kind)
    np.testing.assert_array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0
    u = P.random_field_2d(N, 3)
    inner = (slice(1, N), slice(1, N))
    y = oracle.stencil_apply2d(N, bc_kind, u)
    yt = oracle.stencil_apply2d(N, bc_kind, u, transpose=True)
    ref = (A @ u[inner].ravel()).reshape(N - 1, N - 1)
    np.testing.assert_allclose(y[inner], ref, rtol=0, atol=1e-12)
    np.testing.assert_allclose(yt[inner], (A.T @ u[inner].ravel()).reshape(N - 1, N - 1), rtol=0, atol=1e-12)


@pytest.mark.parametrize("N,bc_kind", [(4, 1), (8, 2), (12, 1)])
def test_dsolve_matches_lapack(N, bc_kind):
    A = oracle.assemble_dense2d(N, bc_kind)
    fh = P.random_field_2d(N, 8)
    fh[0, :] = fh[-1, :] = fh[:, 0] = fh[:, -1] = 0.0
    u = oracle.dsolve2d(N, bc_kind, fh, np.zeros_like(fh))
    ref = np.linalg.solve(A, fh[1:N, 1:N].ravel()).reshape(N - 1, N - 1)
    np.testing.assert_allclose(u[1:N, 1:N], ref, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("bc_kind", [1, 2])
def test_bicg_terminates_and_matches_direct_solve(bc_kind):
    """Bi-CG on (N-1)^2 = 9 unknowns: at most 9 steps in exact arithmetic; a
    few more in FP64 reach the direct solution."""
    N = 4
    fh = P.random_field_2d(N, 9)
    x, it, rel, rc = oracle.bicg2d(N, bc_kind, fh, np.zeros_like(fh), 1e-13)
    assert rc == 0 and it <= 12
    ref = oracle.dsolve2d(N, bc_kind, fh, np.zeros_like(fh))
    np.testing.assert_allclose(x[1:N, 1:N], ref[1:N, 1:N], rtol=1e-10, atol=1e-12)
    N = 16
    fh = P.random_field_2d(N, 10)
    x, it, rel, rc = oracle.bicg2d(N, bc_kind, fh, np.zeros_like(fh), 1e-13)
    ref = oracle.dsolve2d(N, bc_kind, fh, np.zeros_like(fh))
    assert rc == 0
    np.testing.assert_allclose(x[1:N, 1:N], ref[1:N, 1:N], rtol=1e-9, atol=1e-9 * np.abs(ref).max())


def test_exp_finite_exact_on_the_error_expansion():
    """With u bi-quadratic and a bilinear, u^1 = u + a h_1^2 and
    u^0 = u + a h_0^2 on the middle and coarsest grids (eq. (secf)),
    Steps 1-4 return u + a h_2^2 at every fine node."""
    Nf = 16
    rng = np.random.Generator(np.random.PCG64(11))
    Cu = rng.uniform(-1, 1, (3, 3))
    Ca = np.zeros((3, 3))
    Ca[:2, :2] = rng.uniform(-1, 1, (2, 2))
    h2, h1, h0 = 1.0 / Nf, 2.0 / Nf, 4.0 / Nf
    u1 = poly2(Cu, Nf // 2) + poly2(Ca, Nf // 2) * h1 ** 2
    u0 = poly2(Cu, Nf // 4) + poly2(Ca, Nf // 4) * h0 ** 2
    w = oracle.exp_finite2d(Nf, u1, u0)
    ref = poly2(Cu, Nf) + poly2(Ca, Nf) * h2 ** 2
    np.testing.assert_allclose(w, ref, rtol=0, atol=1e-13)


def test_exp_finite_corner_and_edge_formulas():
    """(secfff) at the coarsest nodes and (bfsec) at edge midpoints along x."""
    Nf = 12
    u1 = P.random_field_2d(Nf // 2, 12)
    u0 = P.random_field_2d(Nf // 4, 13)
    w = oracle.exp_finite2d(Nf, u1, u0)
    np.testing.assert_allclose(w[::4, ::4], (5 * u1[::2, ::2] - u0) / 4, rtol=0, atol=1e-14)
    d = u1[::2, ::2] - u0
    np.testing.assert_allclose(w[::4, 2::4], u1[::2, 1::2] + (d[:, :-1] + d[:, 1:]) / 8, rtol=0, atol=1e-14)


def test_exp_true_recovers_u():
    """u_h = u + a h^2, u_2h = u + 4 a h^2 with a bilinear: EXP_true returns u."""
    Nf = 12
    rng = np.random.Generator(np.random.PCG64(14))
    Cu = rng.uniform(-1, 1, (4, 4))
    Ca = np.zeros((2, 2))
    Ca[:, :] = rng.uniform(-1, 1, (2, 2))
    h = 1.0 / Nf
    uh = poly2(Cu, Nf) + poly2(Ca, Nf) * h ** 2
    u2 = poly2(Cu, Nf // 2) + poly2(Ca, Nf // 2) * 4 * h ** 2
    np.testing.assert_allclose(oracle.exp_true2d(Nf, uh, u2), poly2(Cu, Nf), rtol=0, atol=1e-13)


def test_excmg2d_exact_for_biquadratic_first_kind():
    """First-kind data of a bi-quadratic u: the scheme, the reflections and
    EXP_finite are exact, so every Bi-CG level starts converged."""
    prob = P.polynomial_2d([0.3, -0.7, 0.9], [1.0, 0.4, -0.5])
    N = 32
    f, g1, g2 = prob.data(N, 1)
    uh, ut, st = oracle.excmg2d(N, 4, 1, f, g1, g2, 1e-12)
    assert np.abs(uh - prob.exact(N)).max() <= 1e-12
    assert all(v == 0 for v in st[:, 0])


def test_excmg2d_exact_for_bicubic_second_kind():
    prob = P.polynomial_2d([0.2, 0.5, -0.4, 0.7], [1.0, -0.3, 0.6, 0.25])
    N = 32
    f, g1, g2 = prob.data(N, 2)
    uh, ut, st = oracle.excmg2d(N, 4, 2, f, g1, g2, 1e-13)
    assert np.abs(uh - prob.exact(N)).max() <= 1e-10


@pytest.mark.parametrize("bc_kind", [1, 2])
def test_excmg2d_orders(bc_kind):
    """u_h - u falls like h^2; EXP_true improves on it by an order or more."""
    prob = P.sin_pi_2d()
    err, errt = {}, {}
    for N in (32, 64):
        f, g1, g2 = prob.data(N, bc_kind)
        uh, ut, st = oracle.excmg2d(N, 4, bc_kind, f, g1, g2, 1e-12)
        ue = prob.exact(N)
        err[N] = np.abs(uh - ue).max()
        errt[N] = np.abs(ut - ue).max()
    assert 3.6 <= err[32] / err[64] <= 4.4
    assert errt[64] < err[64] / 4


def test_manufactured_2d_data_against_symbolic():
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y")
    for prob, expr in ((P.sin_pi_2d(), sympy.sin(sympy.pi * x) * sympy.sin(sympy.pi * y)),
                       (P.exp_sum_2d(), sympy.exp(x + y))):
        N = 8
        f = sympy.lambdify((x, y), sympy.diff(expr, x, 4) + 2 * sympy.diff(expr, x, 2, y, 2) + sympy.diff(expr, y, 4))
        s = np.arange(N + 1) / N
        X, Y = np.meshgrid(s, s)
        np.testing.assert_allclose(prob.rhs(N), np.broadcast_to(f(X, Y), (N + 1, N + 1)), rtol=1e-12, atol=1e-12)
        g2 = prob.boundary_g2(N, 1)
        ux = sympy.lambdify((x, y), sympy.diff(expr, x))
        np.testing.assert_allclose(g2[0], -np.broadcast_to(ux(0.0, s), (N + 1,)), rtol=1e-12, atol=1e-12)
        uyy = sympy.lambdify((x, y), sympy.diff(expr, y, 2))
        np.testing.assert_allclose(prob.boundary_g2(N, 2)[3], np.broadcast_to(uyy(s, 1.0), (N + 1,)), rtol=1e-12,
                                   atol=1e-12)
