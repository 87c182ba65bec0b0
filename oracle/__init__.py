"""Plain FP64 CPU oracle of the EXCMG / 25-point biharmonic solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never touches it.

The arithmetic lives in ``excmg_oracle.c`` and, for the 2D problem of eq.
(bvp2d), ``excmg2d_oracle.c`` (plain C, compiled with ``-ffp-contract=off``,
OpenMP over loops with independent iterations); this module only builds them
and marshals numpy arrays through ctypes (2D node arrays of shape (N+1, N+1)
in (y, x) order, 2D g2 of shape (4, N+1) with edges x=0, x=1, y=0, y=1).  Array conventions: node arrays of shape (N+1, N+1, N+1) in
(z, y, x) order, i.e. x fastest in memory; g2 as shape (6, N+1, N+1) with faces
x=0, x=1, y=0, y=1, z=0, z=1 and the two in-face axes (a, b) in x<y<z order
stored as [face, b, a].
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "excmg_oracle.c")
_SRC2 = os.path.join(_HERE, "excmg2d_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, FP64, no FMA
    contraction; with OpenMP where the compiler has it)."""
    stale = not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(src) for src in (_SRC, _SRC2))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, _SRC2, "-lm"]
        try:
            subprocess.check_call(base[:-1] + ["-fopenmp", "-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.orc_stencil_apply.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]
        lib.orc_assemble_rhs.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
        lib.orc_inject_nodes.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        lib.orc_inject_faces.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        lib.orc_assemble_dense.argtypes = [ctypes.c_int, ctypes.c_int, _D]
        lib.orc_dsolve.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        lib.orc_residual_norm.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        lib.orc_residual_norm.restype = ctypes.c_double
        lib.orc_interior_norm2.argtypes = [ctypes.c_int, _D]
        lib.orc_interior_norm2.restype = ctypes.c_double
        lib.orc_bicg.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_int, _I, _D]
        lib.orc_bicg_shadow.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int, _I, _D]
        lib.orc_exp_finite.argtypes = [ctypes.c_int, _D, _D, _D]
        lib.orc_exp_true.argtypes = [ctypes.c_int, _D, _D, _D]
        lib.orc_excmg.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D,
                                  ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  _D, _D, _D]
        lib.orc_error_norms.argtypes = [ctypes.c_int, _D, _D, _D]
        lib.orc_error_norms.restype = None
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads.restype = ctypes.c_int
        lib.orc2d_stencil_apply.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]
        lib.orc2d_assemble_rhs.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
        lib.orc2d_inject.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        lib.orc2d_inject_edges.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        lib.orc2d_assemble_dense.argtypes = [ctypes.c_int, ctypes.c_int, _D]
        lib.orc2d_dsolve.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        lib.orc2d_residual_norm.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        lib.orc2d_residual_norm.restype = ctypes.c_double
        lib.orc2d_interior_norm2.argtypes = [ctypes.c_int, _D]
        lib.orc2d_interior_norm2.restype = ctypes.c_double
        lib.orc2d_bicg.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int, _I, _D]
        lib.orc2d_exp_finite.argtypes = [ctypes.c_int, _D, _D, _D]
        lib.orc2d_exp_true.argtypes = [ctypes.c_int, _D, _D, _D]
        lib.orc2d_excmg.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D]
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def set_threads(n: int) -> int:
    """Threads of the oracle's independent loops (the operator and the vector
    updates); sums keep their sequential order, so results are the same bits
    for any count.  Returns the count in effect (1 without OpenMP)."""
    return int(_load().orc_set_threads(int(n)))


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _node(a, N):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != (N + 1, N + 1, N + 1):
        raise ValueError(f"expected node array of shape {(N + 1,) * 3}, got {a.shape}")
    return a


def _faces(a, N):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != (6, N + 1, N + 1):
        raise ValueError(f"expected faces of shape {(6, N + 1, N + 1)}, got {a.shape}")
    return a


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


def stencil_apply(N: int, bc_kind: int, u, transpose: bool = False) -> np.ndarray:
    """y = A_h u (or A_h^T u); only the interior of u is read, y's boundary is 0."""
    u = _node(u, N)
    y = np.empty_like(u)
    _check(_load().orc_stencil_apply(N, bc_kind, int(bool(transpose)), _p(u), _p(y)), "stencil_apply")
    return y


def assemble_rhs(N: int, bc_kind: int, f, g1, g2) -> np.ndarray:
    f, g1, g2 = _node(f, N), _node(g1, N), _faces(g2, N)
    fh = np.empty_like(f)
    _check(_load().orc_assemble_rhs(N, bc_kind, _p(f), _p(g1), _p(g2), _p(fh)), "assemble_rhs")
    return fh


def inject_nodes(Nf: int, stride: int, src) -> np.ndarray:
    src = _node(src, Nf)
    Nc = Nf // stride
    dst = np.empty((Nc + 1,) * 3)
    _check(_load().orc_inject_nodes(Nf, stride, _p(src), _p(dst)), "inject_nodes")
    return dst


def inject_faces(Nf: int, stride: int, src) -> np.ndarray:
    src = _faces(src, Nf)
    Nc = Nf // stride
    dst = np.empty((6, Nc + 1, Nc + 1))
    _check(_load().orc_inject_faces(Nf, stride, _p(src), _p(dst)), "inject_faces")
    return dst


def assemble_dense(N: int, bc_kind: int) -> np.ndarray:
    n = (N - 1) ** 3
    A = np.empty((n, n))
    _check(_load().orc_assemble_dense(N, bc_kind, _p(A)), "assemble_dense")
    return A


def dsolve(N: int, bc_kind: int, fh, u_boundary) -> np.ndarray:
    """Direct solve; returns a node array with u_boundary's boundary and the solution inside."""
    fh = _node(fh, N)
    u = _node(u_boundary, N).copy()
    _check(_load().orc_dsolve(N, bc_kind, _p(fh), _p(u)), "dsolve")
    return u


def residual_norm(N: int, bc_kind: int, fh, u) -> float:
    fh, u = _node(fh, N), _node(u, N)
    return float(_load().orc_residual_norm(N, bc_kind, _p(fh), _p(u)))


def interior_norm2(N: int, a) -> float:
    a = _node(a, N)
    return float(_load().orc_interior_norm2(N, _p(a)))


def bicg(N: int, bc_kind: int, b, x0, tol: float, bnorm: float | None = None, max_iter: int = 10**6,
         shadow=None):
    """Alg. 2 with M = I; r*_0 = shadow (node array, interior read) or r_0.
    Returns (x, iterations, relres, status)."""
    b = _node(b, N)
    x = _node(x0, N).copy()
    if bnorm is None:
        bnorm = interior_norm2(N, b)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    if shadow is None:
        rc = _load().orc_bicg(N, bc_kind, _p(b), _p(x), float(tol), float(bnorm), int(max_iter),
                              ctypes.byref(it), ctypes.byref(rr))
    else:
        sh = _node(shadow, N)
        rc = _load().orc_bicg_shadow(N, bc_kind, _p(b), _p(x), _p(sh), float(tol), float(bnorm), int(max_iter),
                                     ctypes.byref(it), ctypes.byref(rr))
    return x, it.value, rr.value, rc


def exp_finite(Nf: int, u1, u0) -> np.ndarray:
    """Steps 1-5 at every fine node (boundary nodes included)."""
    u1, u0 = _node(u1, Nf // 2), _node(u0, Nf // 4)
    w = np.empty((Nf + 1,) * 3)
    _check(_load().orc_exp_finite(Nf, _p(u1), _p(u0), _p(w)), "exp_finite")
    return w


def exp_true(Nf: int, uh, u2h) -> np.ndarray:
    uh, u2h = _node(uh, Nf), _node(u2h, Nf // 2)
    ut = np.empty_like(uh)
    _check(_load().orc_exp_true(Nf, _p(uh), _p(u2h), _p(ut)), "exp_true")
    return ut


def excmg(n_finest: int, n_coarsest: int, bc_kind: int, f, g1, g2, tol: float,
          tol_mode: str = "uniform", max_iter: int = 100000, max_total: int = 1000000):
    """Alg. 1.  Returns (u_h, u_tilde, stats) with stats[l] = (iters, relres, calls, stagnated)."""
    f, g1, g2 = _node(f, n_finest), _node(g1, n_finest), _faces(g2, n_finest)
    uh = np.empty_like(f)
    ut = np.empty_like(f)
    nl = 0
    n = n_coarsest
    while n < n_finest:
        n *= 2
        nl += 1
    stats = np.zeros((nl + 1, 4))
    mode = {"paper": 0, "uniform": 1}[tol_mode]
    rc = _load().orc_excmg(n_finest, n_coarsest, bc_kind, _p(f), _p(g1), _p(g2), float(tol), mode,
                           int(max_iter), int(max_total), _p(uh), _p(ut), _p(stats))
    _check(rc, "excmg")
    return uh, ut, stats


def error_norms(N: int, a, b):
    """(root-mean-square over all nodes, max) norms of a - b, as in Tables 1-5."""
    a, b = _node(a, N), _node(b, N)
    out = np.zeros(2)
    _load().orc_error_norms(N, _p(a), _p(b), _p(out))
    return float(out[0]), float(out[1])


# ---------------------------------------------------------------- 2D variant
# Node arrays of shape (N+1, N+1) indexed [j, i] (x fastest); g2 of shape
# (4, N+1): edges x=0, x=1, y=0, y=1, indexed by the other coordinate.
def _node2(a, N):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != (N + 1, N + 1):
        raise ValueError(f"expected 2D node array of shape {(N + 1,) * 2}, got {a.shape}")
    return a


def _edges2(a, N):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != (4, N + 1):
        raise ValueError(f"expected edges of shape {(4, N + 1)}, got {a.shape}")
    return a


def stencil_apply2d(N: int, bc_kind: int, u, transpose: bool = False) -> np.ndarray:
    """y = A_h u (or A_h^T u) of the 13-point scheme of the 2D problem."""
    u = _node2(u, N)
    y = np.empty_like(u)
    _check(_load().orc2d_stencil_apply(N, bc_kind, int(bool(transpose)), _p(u), _p(y)), "stencil_apply2d")
    return y


def assemble_rhs2d(N: int, bc_kind: int, f, g1, g2) -> np.ndarray:
    f, g1, g2 = _node2(f, N), _node2(g1, N), _edges2(g2, N)
    fh = np.empty_like(f)
    _check(_load().orc2d_assemble_rhs(N, bc_kind, _p(f), _p(g1), _p(g2), _p(fh)), "assemble_rhs2d")
    return fh


def inject2d(Nf: int, stride: int, src) -> np.ndarray:
    src = _node2(src, Nf)
    dst = np.empty((Nf // stride + 1,) * 2)
    _check(_load().orc2d_inject(Nf, stride, _p(src), _p(dst)), "inject2d")
    return dst


def inject_edges2d(Nf: int, stride: int, src) -> np.ndarray:
    src = _edges2(src, Nf)
    dst = np.empty((4, Nf // stride + 1))
    _check(_load().orc2d_inject_edges(Nf, stride, _p(src), _p(dst)), "inject_edges2d")
    return dst


def assemble_dense2d(N: int, bc_kind: int) -> np.ndarray:
    n = (N - 1) ** 2
    A = np.empty((n, n))
    _check(_load().orc2d_assemble_dense(N, bc_kind, _p(A)), "assemble_dense2d")
    return A


def dsolve2d(N: int, bc_kind: int, fh, u_boundary) -> np.ndarray:
    fh = _node2(fh, N)
    u = _node2(u_boundary, N).copy()
    _check(_load().orc2d_dsolve(N, bc_kind, _p(fh), _p(u)), "dsolve2d")
    return u


def residual_norm2d(N: int, bc_kind: int, fh, u) -> float:
    return float(_load().orc2d_residual_norm(N, bc_kind, _p(_node2(fh, N)), _p(_node2(u, N))))


def bicg2d(N: int, bc_kind: int, b, x0, tol: float, bnorm: float | None = None, max_iter: int = 10**6):
    """Alg. 2 (M = I, r*_0 = r_0) on the 2D system; (x, iterations, relres, status)."""
    b = _node2(b, N)
    x = _node2(x0, N).copy()
    if bnorm is None:
        bnorm = float(_load().orc2d_interior_norm2(N, _p(b)))
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    rc = _load().orc2d_bicg(N, bc_kind, _p(b), _p(x), float(tol), float(bnorm), int(max_iter), ctypes.byref(it),
                            ctypes.byref(rr))
    return x, it.value, rr.value, rc


def exp_finite2d(Nf: int, u1, u0) -> np.ndarray:
    u1, u0 = _node2(u1, Nf // 2), _node2(u0, Nf // 4)
    w = np.empty((Nf + 1,) * 2)
    _check(_load().orc2d_exp_finite(Nf, _p(u1), _p(u0), _p(w)), "exp_finite2d")
    return w


def exp_true2d(Nf: int, uh, u2h) -> np.ndarray:
    uh, u2h = _node2(uh, Nf), _node2(u2h, Nf // 2)
    ut = np.empty_like(uh)
    _check(_load().orc2d_exp_true(Nf, _p(uh), _p(u2h), _p(ut)), "exp_true2d")
    return ut


def excmg2d(n_finest: int, n_coarsest: int, bc_kind: int, f, g1, g2, tol: float, tol_mode: str = "uniform",
            max_iter: int = 100000, max_total: int = 1000000):
    """Alg. 1 on the 2D problem; (u_h, u_tilde, stats) as excmg()."""
    f, g1, g2 = _node2(f, n_finest), _node2(g1, n_finest), _edges2(g2, n_finest)
    uh = np.empty_like(f)
    ut = np.empty_like(f)
    nl, n = 0, n_coarsest
    while n < n_finest:
        n *= 2
        nl += 1
    stats = np.zeros((nl + 1, 4))
    rc = _load().orc2d_excmg(n_finest, n_coarsest, bc_kind, _p(f), _p(g1), _p(g2), float(tol),
                             {"paper": 0, "uniform": 1}[tol_mode], int(max_iter), int(max_total), _p(uh), _p(ut),
                             _p(stats))
    _check(rc, "excmg2d")
    return uh, ut, stats
