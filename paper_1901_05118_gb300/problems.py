"""Seeded, synthetic inputs: manufactured solutions of the biharmonic problem.

This module only evaluates closed forms (u, f = Laplacian^2 u, and the boundary
data g1, g2 of eqs. (BC) / (BC2)) on the nested uniform grids of the paper.  It
contains none of the method's arithmetic and is the one module that both the
CUDA path's tests/bench and the CPU oracle's tests draw their inputs from.

Array conventions: node arrays of shape (N+1, N+1, N+1) indexed [k, j, i]
(x fastest in memory); boundary data g2 of shape (6, N+1, N+1) with faces
x=0, x=1, y=0, y=1, z=0, z=1 and the two in-face axes (a, b) in x<y<z order
stored as [face, b, a].  bc_kind 1: g2 = du/dn (outward normal); bc_kind 2:
g2 = d2u/dn2.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Sequence

import numpy as np

PI = np.pi


@dataclass(frozen=True)
class Manufactured:
    """u and its derivatives as numpy callables of broadcast (x, y, z) grids."""

    name: str
    u: Callable
    f: Callable                 # Laplacian^2 u
    grad: Callable              # -> (u_x, u_y, u_z)
    d2: Callable                # -> (u_xx, u_yy, u_zz)

    # ------------------------------------------------------------------ grids
    @staticmethod
    def axes(N: int):
        s = np.arange(N + 1, dtype=np.float64) / N
        return s[None, None, :], s[None, :, None], s[:, None, None]

    def nodes(self, fn: Callable, N: int) -> np.ndarray:
        x, y, z = self.axes(N)
        return np.array(np.broadcast_to(fn(x, y, z), (N + 1,) * 3), dtype=np.float64, order="C")

    def exact(self, N: int) -> np.ndarray:
        return self.nodes(self.u, N)

    def rhs(self, N: int) -> np.ndarray:
        return self.nodes(self.f, N)

    def boundary_g2(self, N: int, bc_kind: int) -> np.ndarray:
        s = np.arange(N + 1, dtype=np.float64) / N
        g2 = np.empty((6, N + 1, N + 1))
        zero, one = np.zeros(()), np.ones(())
        # in-face grids: first index b, second a
        for face in range(6):
            axis, side = divmod(face, 2)
            c = one if side else zero
            if axis == 0:    # (a, b) = (y, z)
                x, y, z = c[None, None], s[None, :], s[:, None]
            elif axis == 1:  # (a, b) = (x, z)
                x, y, z = s[None, :], c[None, None], s[:, None]
            else:            # (a, b) = (x, y)
                x, y, z = s[None, :], s[:, None], c[None, None]
            if bc_kind == 1:
                d = self.grad(x, y, z)[axis]
                val = d if side else -d          # outward normal derivative
            elif bc_kind == 2:
                val = self.d2(x, y, z)[axis]     # second normal derivative
            else:
                raise ValueError("bc_kind must be 1 or 2")
            g2[face] = np.broadcast_to(val, (N + 1, N + 1))
        return g2

    def data(self, N: int, bc_kind: int):
        """(f, g1, g2) on the grid with N intervals; g1 is the full exact u."""
        return self.rhs(N), self.exact(N), self.boundary_g2(N, bc_kind)


def _ones_like(*a):
    return np.ones(np.broadcast(*a).shape)


# ---------------------------------------------------------------- separable
def separable(name: str, terms: Sequence[tuple]) -> Manufactured:
    """u = sum_m A_m X_m(x) Y_m(y) Z_m(z) with each factor given as
    (fn, d1, d2, d4) callables; f = sum of the six fourth-derivative terms."""

    def u(x, y, z):
        return sum(A * X[0](x) * Y[0](y) * Z[0](z) for A, X, Y, Z in terms)

    def f(x, y, z):
        out = 0.0
        for A, X, Y, Z in terms:
            x0, x2, x4 = X[0](x), X[2](x), X[3](x)
            y0, y2, y4 = Y[0](y), Y[2](y), Y[3](y)
            z0, z2, z4 = Z[0](z), Z[2](z), Z[3](z)
            out = out + A * (x4 * y0 * z0 + x0 * y4 * z0 + x0 * y0 * z4
                             + 2 * x2 * y2 * z0 + 2 * x2 * y0 * z2 + 2 * x0 * y2 * z2)
        return out

    def grad(x, y, z):
        gx = sum(A * X[1](x) * Y[0](y) * Z[0](z) for A, X, Y, Z in terms)
        gy = sum(A * X[0](x) * Y[1](y) * Z[0](z) for A, X, Y, Z in terms)
        gz = sum(A * X[0](x) * Y[0](y) * Z[1](z) for A, X, Y, Z in terms)
        return gx, gy, gz

    def d2(x, y, z):
        hx = sum(A * X[2](x) * Y[0](y) * Z[0](z) for A, X, Y, Z in terms)
        hy = sum(A * X[0](x) * Y[2](y) * Z[0](z) for A, X, Y, Z in terms)
        hz = sum(A * X[0](x) * Y[0](y) * Z[2](z) for A, X, Y, Z in terms)
        return hx, hy, hz

    return Manufactured(name, u, f, grad, d2)


def sin_factor(a: float):
    w = a * PI
    return (lambda s: np.sin(w * s), lambda s: w * np.cos(w * s),
            lambda s: -w * w * np.sin(w * s), lambda s: w ** 4 * np.sin(w * s))


def exp_factor():
    return (np.exp, np.exp, np.exp, np.exp)


def sinh_factor():
    return (np.sinh, np.cosh, np.sinh, np.sinh)


def one_minus_cos2pi():
    w = 2 * PI
    return (lambda s: 1 - np.cos(w * s), lambda s: w * np.sin(w * s),
            lambda s: w * w * np.cos(w * s), lambda s: -w ** 4 * np.cos(w * s))


def poly_factor(c: Sequence[float]):
    """Polynomial factor sum_n c[n] s^n."""
    p = np.polynomial.Polynomial(c)
    d1, d2, d4 = p.deriv(1), p.deriv(2), p.deriv(4)
    return (lambda s: p(s), lambda s: d1(s), lambda s: d2(s), lambda s: d4(s))


# ------------------------------------------------------- named problems
def sin_pi() -> Manufactured:
    """u = sin(pi x) sin(pi y) sin(pi z); f = 9 pi^4 u, g1 = 0."""
    s = sin_factor(1.0)
    return separable("sin_pi", [(1.0, s, s, s)])


def exp_sum() -> Manufactured:
    """u = exp(x + y + z); f = 9 u."""
    e = exp_factor()
    return separable("exp_sum", [(1.0, e, e, e)])


def sin2pi_plus_poly() -> Manufactured:
    """u = sin(2 pi x) sin(2 pi y) sin(2 pi z) + x^2 y^2 z^2."""
    s = sin_factor(2.0)
    q = poly_factor([0.0, 0.0, 1.0])
    return separable("sin2pi_plus_poly", [(1.0, s, s, s), (1.0, q, q, q)])


def random_sine_terms(seed: int, n_terms: int = 4):
    """[(A, a, b, c)]: a, b, c integers in [1, 4], A ~ N(0, 1), numpy PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    terms = []
    for _ in range(n_terms):
        a, b, c = (int(v) for v in rng.integers(1, 5, size=3))
        A = float(rng.standard_normal())
        terms.append((A, a, b, c))
    return terms


def random_sines(seed: int, n_terms: int = 4) -> Manufactured:
    """u = sum of n_terms A sin(a pi x) sin(b pi y) sin(c pi z), a,b,c in [1,4]
    integers and A ~ N(0,1), drawn from numpy's PCG64 with the given seed."""
    terms = [(A, sin_factor(a), sin_factor(b), sin_factor(c)) for A, a, b, c in random_sine_terms(seed, n_terms)]
    return separable(f"random_sines[{seed}]", terms)


def random_sines_torch(seed: int, N: int, bc_kind: int, device, n_terms: int = 4):
    """(f, g1, g2) of random_sines(seed) evaluated with torch on `device`
    (used to build many request inputs quickly on the GPU).  The same closed
    forms as the numpy version: f = sum A pi^4 (a^2+b^2+c^2)^2 s(x)s(y)s(z);
    g1 = u; g2 the outward normal derivative (first kind) or the second
    normal derivative (second kind) on the six faces."""
    import torch

    s = torch.arange(N + 1, dtype=torch.float64, device=device) / N
    f = torch.zeros((N + 1,) * 3, dtype=torch.float64, device=device)
    u = torch.zeros_like(f)
    g2 = torch.zeros((6, N + 1, N + 1), dtype=torch.float64, device=device)
    pi = float(PI)
    for A, a, b, c in random_sine_terms(seed, n_terms):
        sx, sy, sz = torch.sin(a * pi * s), torch.sin(b * pi * s), torch.sin(c * pi * s)
        prod = sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
        u += A * prod
        f += A * pi ** 4 * (a * a + b * b + c * c) ** 2 * prod
        w = (a * pi, b * pi, c * pi)
        for face in range(6):
            axis, side = divmod(face, 2)
            c1 = 1.0 if side else 0.0
            if axis == 0:    # in-face (a, b) = (y, z): rows z, columns y
                other = sz[:, None] * sy[None, :]
            elif axis == 1:  # (x, z)
                other = sz[:, None] * sx[None, :]
            else:            # (x, y)
                other = sy[:, None] * sx[None, :]
            k = w[axis]
            if bc_kind == 1:
                d = k * np.cos(k * c1)
                g2[face] += A * (d if side else -d) * other
            else:
                g2[face] += A * (-k * k * np.sin(k * c1)) * other
    return f, u, g2


def paper_problem1() -> Manufactured:
    """Test Problem 1: u = (1-cos 2 pi x)(1-cos 2 pi y)(1-cos 2 pi z)."""
    g = one_minus_cos2pi()
    return separable("paper_p1", [(1.0, g, g, g)])


def paper_problem3() -> Manufactured:
    """Test Problem 3: u = sinh x sinh y sinh z (f = u)."""
    g = sinh_factor()
    return separable("paper_p3", [(1.0, g, g, g)])


def paper_problem2() -> Manufactured:
    """Test Problem 2: u = exp(xyz)."""

    def u(x, y, z):
        return np.exp(x * y * z)

    def f(x, y, z):  # eq. (force2) as printed
        return np.exp(x * y * z) * (
            x**4 * y**4 + 2 * x**4 * y**2 * z**2 + x**4 * z**4 + 8 * x**3 * y * z
            + 2 * x**2 * y**4 * z**2 + 2 * x**2 * y**2 * z**4 + 4 * x**2 + 8 * x * y**3 * z
            + 8 * x * y * z**3 + y**4 * z**4 + 4 * y**2 + 4 * z**2)

    def grad(x, y, z):
        e = np.exp(x * y * z)
        return y * z * e, x * z * e, x * y * e

    def d2(x, y, z):
        e = np.exp(x * y * z)
        return (y * z) ** 2 * e, (x * z) ** 2 * e, (x * y) ** 2 * e

    return Manufactured("paper_p2", u, f, grad, d2)


def paper_problem4() -> Manufactured:
    """Test Problem 4: u = xyz log(1 + x + y + z)."""

    def u(x, y, z):
        return x * y * z * np.log(1 + x + y + z)

    def f(x, y, z):  # eq. (force4) as printed
        return -(2 * (4 * x**3 + 8 * x**2 + 15 * x * y * z + 4 * x * y + 4 * x * z + 4 * x
                      + 4 * y**3 + 8 * y**2 + 4 * y * z + 4 * y + 4 * z**3 + 8 * z**2 + 4 * z)) \
            / (x + y + z + 1) ** 4

    def grad(x, y, z):
        s = 1 + x + y + z
        lg = np.log(s)
        return (y * z * (lg + x / s), x * z * (lg + y / s), x * y * (lg + z / s))

    def d2(x, y, z):
        s = 1 + x + y + z
        # d2/dx2 [x log s] = 2/s - x/s^2
        return (y * z * (2 / s - x / s**2), x * z * (2 / s - y / s**2), x * y * (2 / s - z / s**2))

    return Manufactured("paper_p4", u, f, grad, d2)


def polynomial(cx: Sequence[float], cy: Sequence[float], cz: Sequence[float],
               extra: Sequence[tuple] = ()) -> Manufactured:
    """Sum of separable polynomial terms: (1, cx, cy, cz) plus `extra` as
    (A, cx, cy, cz) tuples."""
    terms = [(1.0, poly_factor(cx), poly_factor(cy), poly_factor(cz))]
    for A, ex, ey, ez in extra:
        terms.append((A, poly_factor(ex), poly_factor(ey), poly_factor(ez)))
    return separable("polynomial", terms)


def by_name(name: str) -> Manufactured:
    table = {
        "sin_pi": sin_pi, "exp_sum": exp_sum, "sin2pi_plus_poly": sin2pi_plus_poly,
        "paper_p1": paper_problem1, "paper_p2": paper_problem2,
        "paper_p3": paper_problem3, "paper_p4": paper_problem4,
    }
    if name.startswith("random_sines:"):
        return random_sines(int(name.split(":", 1)[1]))
    return table[name]()


def random_field(N: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Seeded uniform random node array (for operator parity on rough inputs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=(N + 1,) * 3)


# -------------------------------------------------------------- 2D variant
# The two-dimensional problem (eq. (bvp2d)) on (0,1)^2.  Node arrays of shape
# (N+1, N+1) indexed [j, i] (x fastest); g2 of shape (4, N+1): edges x=0,
# x=1, y=0, y=1, indexed by the other coordinate.
@dataclass(frozen=True)
class Manufactured2D:
    """u = sum_m A_m X_m(x) Y_m(y) with each factor given as (fn, d1, d2, d4)."""

    name: str
    terms: tuple

    @staticmethod
    def axes(N: int):
        s = np.arange(N + 1, dtype=np.float64) / N
        return s[None, :], s[:, None]

    def _sum(self, kx: int, ky: int, x, y):
        return sum(A * X[kx](x) * Y[ky](y) for A, X, Y in self.terms)

    def exact(self, N: int) -> np.ndarray:
        x, y = self.axes(N)
        return np.array(np.broadcast_to(self._sum(0, 0, x, y), (N + 1, N + 1)), dtype=np.float64, order="C")

    def rhs(self, N: int) -> np.ndarray:
        """f = u_xxxx + 2 u_xxyy + u_yyyy."""
        x, y = self.axes(N)
        f = self._sum(3, 0, x, y) + 2 * self._sum(2, 2, x, y) + self._sum(0, 3, x, y)
        return np.array(np.broadcast_to(f, (N + 1, N + 1)), dtype=np.float64, order="C")

    def boundary_g2(self, N: int, bc_kind: int) -> np.ndarray:
        s = np.arange(N + 1, dtype=np.float64) / N
        g2 = np.empty((4, N + 1))
        for e in range(4):
            axis, side = divmod(e, 2)
            c = np.ones(N + 1) if side else np.zeros(N + 1)
            x, y = (c, s) if axis == 0 else (s, c)
            if bc_kind == 1:
                d = self._sum(1, 0, x, y) if axis == 0 else self._sum(0, 1, x, y)
                g2[e] = d if side else -d                     # outward normal derivative
            elif bc_kind == 2:
                g2[e] = self._sum(2, 0, x, y) if axis == 0 else self._sum(0, 2, x, y)
            else:
                raise ValueError("bc_kind must be 1 or 2")
        return g2

    def data(self, N: int, bc_kind: int):
        return self.rhs(N), self.exact(N), self.boundary_g2(N, bc_kind)


def sin_pi_2d() -> Manufactured2D:
    """u = sin(pi x) sin(pi y), f = 4 pi^4 u."""
    return Manufactured2D("sin_pi_2d", ((1.0, sin_factor(1.0), sin_factor(1.0)),))


def exp_sum_2d() -> Manufactured2D:
    """u = e^(x+y), f = 4u."""
    return Manufactured2D("exp_sum_2d", ((1.0, exp_factor(), exp_factor()),))


def polynomial_2d(cx: Sequence[float], cy: Sequence[float]) -> Manufactured2D:
    """u = p(x) q(y) with the given coefficient lists (lowest degree first)."""
    return Manufactured2D("poly_2d", ((1.0, poly_factor(cx), poly_factor(cy)),))


def random_field_2d(N: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=(N + 1, N + 1))
