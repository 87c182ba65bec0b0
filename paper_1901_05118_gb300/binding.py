"""Thin ctypes binding of ``libexcmg.so`` (the C ABI in ``include/excmg.h``).

Argument marshalling only: every step of the solver runs in the CUDA library.
Arrays are torch CUDA tensors (float64, contiguous) passed by data_ptr(); node
arrays have shape (N+1, N+1, N+1) indexed [k, j, i] (x fastest), boundary
data g2 has shape (6, N+1, N+1).  Work is enqueued on torch's current CUDA
stream of the tensors' device.  If the library has not been built, importing
this module raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libexcmg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(LIB_PATH)

EXCMG_OK = 0
STATUS_NAMES = {0: "EXCMG_OK", -1: "EXCMG_ERR_ARG", -2: "EXCMG_ERR_OOM", -3: "EXCMG_ERR_BREAKDOWN",
                -4: "EXCMG_ERR_NOCONV", -5: "EXCMG_ERR_NAN", -6: "EXCMG_ERR_CUDA",
                -7: "EXCMG_ERR_TIMEOUT", -9: "EXCMG_ERR_BUDGET", -10: "EXCMG_ERR_SIZE",
                -11: "EXCMG_ERR_TOO_LARGE"}
TOL_MODES = {"paper": 0, "uniform": 1}
STENCIL_VARIANTS = {"exact": 0, "fp64": 1}
SHADOW_MODES = {"full": 0, "elided": 1}
SCHEDULES = {"separate": 0, "fused": 1}
PRECISIONS = {"fp64": 0, "mixed": 1}
MIXED_INNER_CAP = 500      # iterations of one FP32 correction solve
MIXED_INNER_TOL = 1e-4     # residual reduction asked of one FP32 correction solve
MAX_LEVELS = 16


class ExcmgError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("tol_mode", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("max_total", ctypes.c_int), ("check_every", ctypes.c_int), ("precision", ctypes.c_int),
                ("inner_tol", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("n", ctypes.c_int * MAX_LEVELS),
                ("iters", ctypes.c_int * MAX_LEVELS), ("calls", ctypes.c_int * MAX_LEVELS),
                ("stagnated", ctypes.c_int * MAX_LEVELS), ("relres", ctypes.c_double * MAX_LEVELS),
                ("ms", ctypes.c_double * MAX_LEVELS)]

    def as_list(self):
        return [dict(n=self.n[l], iters=self.iters[l], calls=self.calls[l],
                     stagnated=bool(self.stagnated[l]), relres=self.relres[l], ms=self.ms[l])
                for l in range(self.levels)]


_vp, _i, _d, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
_lib.excmg_ctx_create.argtypes = [_vp, _sz, ctypes.POINTER(_vp)]
_lib.excmg_ctx_destroy.argtypes = [_vp]
_lib.excmg_ctx_bytes.argtypes = [_vp]
_lib.excmg_ctx_bytes.restype = _sz
_lib.excmg_ctx_set_stencil.argtypes = [_vp, _i]
_lib.excmg_ctx_set_shadow_mode.argtypes = [_vp, _i]
_lib.excmg_ctx_set_schedule.argtypes = [_vp, _i]
_lib.excmg_ctx_set_graphs.argtypes = [_vp, _i]
_lib.excmg_launch_count.argtypes = []
_lib.excmg_launch_count.restype = ctypes.c_longlong
_lib.excmg_ctx_profile.argtypes = [_vp, _i]
_lib.excmg_ctx_profile_read.argtypes = [_vp, _i, ctypes.POINTER(_d), ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.POINTER(_d)]
_lib.excmg_last_error.argtypes = [_vp]
_lib.excmg_last_error.restype = ctypes.c_char_p
_lib.excmg_level_create.argtypes = [_vp, _i, _i, ctypes.POINTER(_vp)]
_lib.excmg_level_destroy.argtypes = [_vp]
_lib.stencil_apply.argtypes = [_vp, _i, _vp, _vp]
_lib.bicg_solve.argtypes = [_vp, _vp, _vp, _d, _i, ctypes.POINTER(_i), ctypes.POINTER(_d)]
_lib.bicg_solve_ex.argtypes = [_vp, _vp, _vp, _vp, _d, _i, ctypes.POINTER(_i), ctypes.POINTER(_d)]
_lib.extrapolate_interpolate.argtypes = [_i, _vp, _vp, _vp, _vp]
_lib.extrapolate_interpolate_ex.argtypes = [_vp, _i, _vp, _vp, _vp, _vp]
_lib.midpoint_extrapolate.argtypes = [_i, _vp, _vp, _vp]
_lib.midpoint_extrapolate_ex.argtypes = [_vp, _i, _vp, _vp, _vp]
_lib.excmg_solve.argtypes = [_i, _i, _i, _vp, _vp, _vp, _d, _vp]
_lib.excmg_solve_ex.argtypes = [_vp, _i, _i, _i, _vp, _vp, _vp, ctypes.POINTER(Params), _vp, _vp,
                                ctypes.POINTER(Stats)]
_lib.excmg_assemble_rhs.argtypes = [_vp, _i, _vp, _vp, _vp, _vp]
_lib.excmg_dsolve.argtypes = [_vp, _vp, _vp]

_lib.excmg_batch_create.argtypes = [_vp, _sz, _i, ctypes.POINTER(_vp)]
_lib.excmg_batch_destroy.argtypes = [_vp]
_lib.excmg_batch_last_error.argtypes = [_vp]
_lib.excmg_batch_last_error.restype = ctypes.c_char_p
_lib.excmg_batch_bytes.argtypes = [_vp]
_lib.excmg_batch_bytes.restype = _sz
_lib.excmg_batch_instance_bytes.argtypes = [_i, _i, _i]
_lib.excmg_batch_instance_bytes.restype = _sz
_lib.excmg_batch_submit.argtypes = [_vp, _i, _i, _i, _vp, _vp, _vp, ctypes.POINTER(Params), _vp,
                                    ctypes.POINTER(_i)]
_lib.excmg_batch_step.argtypes = [_vp, ctypes.POINTER(_i)]
_lib.excmg_batch_query.argtypes = [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(Stats),
                                   ctypes.POINTER(_d)]
_lib.excmg_batch_launches.argtypes = [_vp]
_lib.excmg_batch_launches.restype = ctypes.c_longlong


class BatchProfile(ctypes.Structure):
    _fields_ = [("group_launches", ctypes.c_longlong), ("rounds", ctypes.c_longlong),
                ("member_rounds", ctypes.c_longlong), ("member_iters", ctypes.c_longlong),
                ("group_ms", ctypes.c_double), ("host_s", ctypes.c_double), ("wait_s", ctypes.c_double)]


_lib.excmg_batch_get_profile.argtypes = [_vp, ctypes.POINTER(BatchProfile)]
_lib.excmg_selftest_wait_timeout.argtypes = [_i, ctypes.c_longlong]
_lib.excmg_selftest_wait_timeout.restype = _i
_lib.excmg2d_stencil_apply.argtypes = [_vp, _i, _i, _i, _vp, _vp]
_lib.excmg2d_bicg_solve.argtypes = [_vp, _i, _i, _vp, _vp, _d, _i, ctypes.POINTER(_i), ctypes.POINTER(_d)]
_lib.excmg2d_extrapolate_interpolate.argtypes = [_vp, _i, _vp, _vp, _vp, _vp]
_lib.excmg2d_midpoint_extrapolate.argtypes = [_vp, _i, _vp, _vp, _vp]
_lib.excmg2d_solve.argtypes = [_vp, _i, _i, _i, _vp, _vp, _vp, ctypes.POINTER(Params), _vp, _vp,
                               ctypes.POINTER(Stats)]
for _name in ("excmg2d_stencil_apply", "excmg2d_bicg_solve", "excmg2d_extrapolate_interpolate",
              "excmg2d_midpoint_extrapolate", "excmg2d_solve"):
    getattr(_lib, _name).restype = _i

for _name in ("excmg_batch_create", "excmg_batch_destroy", "excmg_batch_submit", "excmg_batch_step",
              "excmg_batch_query"):
    getattr(_lib, _name).restype = _i

for _name in ("excmg_ctx_create", "excmg_ctx_destroy", "excmg_ctx_set_stencil", "excmg_ctx_set_shadow_mode",
              "excmg_ctx_set_schedule", "excmg_ctx_set_graphs", "excmg_ctx_profile",
              "excmg_ctx_profile_read", "excmg_level_create", "excmg_level_destroy",
              "stencil_apply", "bicg_solve", "bicg_solve_ex", "extrapolate_interpolate", "extrapolate_interpolate_ex",
              "midpoint_extrapolate", "midpoint_extrapolate_ex", "excmg_solve", "excmg_solve_ex",
              "excmg_assemble_rhs", "excmg_dsolve"):
    getattr(_lib, _name).restype = _i


def lib():
    return _lib


def launch_count() -> int:
    """Kernel launches the library has made in this process."""
    return int(_lib.excmg_launch_count())


def selftest_wait_timeout(which: str, limit: int) -> int:
    """Make a bounded device wait run out on purpose ('barrier': the grid
    barrier of the cooperative kernels, limit in polls).  Returns the library
    status (-7, EXCMG_ERR_TIMEOUT, when it gave up)."""
    return int(_lib.excmg_selftest_wait_timeout({"barrier": 0}[which], int(limit)))


# ----------------------------------------------------------------- checks
def _node(t: torch.Tensor, n: int, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != (n + 1) ** 3:
        raise ValueError(f"{name} must be a contiguous float64 tensor with (N+1)^3 = {(n + 1) ** 3} elements")
    return t.data_ptr()


def _faces(t: torch.Tensor, n: int, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != 6 * (n + 1) ** 2:
        raise ValueError(f"{name} must be a contiguous float64 tensor with 6 (N+1)^2 elements")
    return t.data_ptr()


def _new_node(n: int, like: torch.Tensor) -> torch.Tensor:
    return torch.empty((n + 1,) * 3, dtype=torch.float64, device=like.device)


# --------------------------------------------------------------- contexts
class Context:
    """A library context bound to one CUDA stream (default: torch's current)."""

    def __init__(self, device=None, stream=None, hbm_budget_bytes: int = 0):
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index)
        with torch.cuda.device(dev):
            s = stream if stream is not None else torch.cuda.current_stream(dev)
            self.stream = s
            self.device = dev
            h = _vp()
            rc = _lib.excmg_ctx_create(_vp(s.cuda_stream), int(hbm_budget_bytes), ctypes.byref(h))
            if rc != EXCMG_OK:
                raise ExcmgError(rc, "excmg_ctx_create failed")
            self.handle = h

    def check(self, rc: int, what: str):
        if rc != EXCMG_OK:
            msg = _lib.excmg_last_error(self.handle)
            raise ExcmgError(rc, f"{what}: {msg.decode() if msg else ''}")

    def set_stencil(self, variant: str):
        """'exact' (integer accumulation, default) or 'fp64' arithmetic for the operator."""
        self.check(_lib.excmg_ctx_set_stencil(self.handle, STENCIL_VARIANTS[variant]), "excmg_ctx_set_stencil")

    def set_shadow_mode(self, mode: str):
        """'full' (default: Alg. 2 with r*, p*, A^T p* in memory) or 'elided'
        (a labelled variant, not the paper's algorithm as printed: the shadow
        sequence, bit for bit the primal one with the exact operator, is not
        stored; results are the same bits)."""
        self.check(_lib.excmg_ctx_set_shadow_mode(self.handle, SHADOW_MODES[mode]), "excmg_ctx_set_shadow_mode")

    def set_schedule(self, schedule: str):
        """'separate' (default: operator pair, update, direction update) or
        'fused' (direction update folded into the operator launch, staged
        input rows; measured slower on GB300)."""
        self.check(_lib.excmg_ctx_set_schedule(self.handle, SCHEDULES[schedule]), "excmg_ctx_set_schedule")

    def set_graphs(self, enable: bool):
        """Replay full batches of launched Bi-CG iterations from CUDA graphs
        (default on; the same bits either way)."""
        self.check(_lib.excmg_ctx_set_graphs(self.handle, int(bool(enable))), "excmg_ctx_set_graphs")

    def profile(self, enable: bool = True):
        """Time every operator launch inside Bi-CG (CUDA events on this context's stream)."""
        self.check(_lib.excmg_ctx_profile(self.handle, int(bool(enable))), "excmg_ctx_profile")

    def profile_read(self, n: int):
        """(total ms, launches, algorithmic bytes) of the operator launches on
        grids with n intervals since profile()."""
        ms = ctypes.c_double(0.0)
        cnt = ctypes.c_longlong(0)
        nbytes = ctypes.c_double(0.0)
        self.check(_lib.excmg_ctx_profile_read(self.handle, int(n), ctypes.byref(ms), ctypes.byref(cnt),
                                               ctypes.byref(nbytes)), "excmg_ctx_profile_read")
        return ms.value, cnt.value, nbytes.value

    @property
    def bytes(self) -> int:
        return int(_lib.excmg_ctx_bytes(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            with torch.cuda.device(self.device):
                _lib.excmg_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_ctx_lock = threading.Lock()
_ctx_cache: dict = {}


def default_context(device=None) -> Context:
    """One cached context per (device, current stream)."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index)
    key = (dev.index, torch.cuda.current_stream(dev).cuda_stream)
    with _ctx_lock:
        c = _ctx_cache.get(key)
        if c is None:
            c = Context(dev)
            _ctx_cache[key] = c
        return c


class Level:
    """One grid (N intervals, bc_kind) on a context."""

    def __init__(self, n: int, bc_kind: int, ctx: Context | None = None):
        self.ctx = ctx or default_context()
        self.n = int(n)
        self.bc_kind = int(bc_kind)
        h = _vp()
        self.ctx.check(_lib.excmg_level_create(self.ctx.handle, self.n, self.bc_kind, ctypes.byref(h)),
                       "excmg_level_create")
        self.handle = h

    def __del__(self):
        try:
            if getattr(self, "handle", None):
                _lib.excmg_level_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


# ------------------------------------------------------------- the hot path
def stencil_apply(level: Level, u: torch.Tensor, y: torch.Tensor | None = None,
                  transpose: bool = False) -> torch.Tensor:
    """y = A_h u (or A_h^T u) on the level's interior nodes; y's boundary is zero."""
    n = level.n
    pu = _node(u, n, "u")
    if y is None:
        y = _new_node(n, u)
    py = _node(y, n, "y")
    level.ctx.check(_lib.stencil_apply(level.handle, int(bool(transpose)), _vp(pu), _vp(py)), "stencil_apply")
    return y


def bicg_solve(level: Level, b: torch.Tensor, x: torch.Tensor, tol: float, max_iter: int = 100000,
               shadow: torch.Tensor | None = None):
    """Alg. 2 (M = I; r*_0 = shadow, or r_0) on A_h x = b in place; returns (iters, relres, status)."""
    n = level.n
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    if shadow is None:
        rc = _lib.bicg_solve(level.handle, _vp(_node(b, n, "b")), _vp(_node(x, n, "x")), float(tol),
                             int(max_iter), ctypes.byref(it), ctypes.byref(rr))
    else:
        rc = _lib.bicg_solve_ex(level.handle, _vp(_node(b, n, "b")), _vp(_node(x, n, "x")),
                                _vp(_node(shadow, n, "shadow")), float(tol), int(max_iter), ctypes.byref(it),
                                ctypes.byref(rr))
    if rc not in (EXCMG_OK, -4):
        level.ctx.check(rc, "bicg_solve")
    return it.value, rr.value, rc


def extrapolate_interpolate(n_fine: int, u_2h: torch.Tensor, u_4h: torch.Tensor,
                            w_h: torch.Tensor | None = None, ctx: Context | None = None,
                            g1_fine: torch.Tensor | None = None) -> torch.Tensor:
    """EXP_finite: third-order guess on the n_fine grid from u_2h and u_4h.
    With g1_fine (a fine-grid node array) its boundary entries overwrite
    w_h's boundary nodes; without it they keep the interpolated values."""
    ctx = ctx or default_context(u_2h.device)
    p2 = _node(u_2h, n_fine // 2, "u_2h")
    p4 = _node(u_4h, n_fine // 4, "u_4h")
    pg = _vp(_node(g1_fine, n_fine, "g1_fine")) if g1_fine is not None else _vp(0)
    if w_h is None:
        w_h = _new_node(n_fine, u_2h)
    ctx.check(_lib.extrapolate_interpolate_ex(ctx.handle, int(n_fine), _vp(p2), _vp(p4), pg,
                                              _vp(_node(w_h, n_fine, "w_h"))), "extrapolate_interpolate")
    return w_h


def midpoint_extrapolate(n_fine: int, u_h: torch.Tensor, u_2h: torch.Tensor,
                         u_tilde: torch.Tensor | None = None, ctx: Context | None = None) -> torch.Tensor:
    """EXP_true: u~ = u_h + (1/3) multilinear interpolation of (u_h - u_2h)."""
    ctx = ctx or default_context(u_h.device)
    ph = _node(u_h, n_fine, "u_h")
    p2 = _node(u_2h, n_fine // 2, "u_2h")
    if u_tilde is None:
        u_tilde = _new_node(n_fine, u_h)
    ctx.check(_lib.midpoint_extrapolate_ex(ctx.handle, int(n_fine), _vp(ph), _vp(p2),
                                           _vp(_node(u_tilde, n_fine, "u_tilde"))), "midpoint_extrapolate")
    return u_tilde


def excmg_assemble_rhs(level: Level, n_src: int, f: torch.Tensor, g1: torch.Tensor, g2: torch.Tensor,
                       fh: torch.Tensor | None = None) -> torch.Tensor:
    if fh is None:
        fh = _new_node(level.n, f)
    level.ctx.check(_lib.excmg_assemble_rhs(level.handle, int(n_src), _vp(_node(f, n_src, "f")),
                                            _vp(_node(g1, n_src, "g1")), _vp(_faces(g2, n_src, "g2")),
                                            _vp(_node(fh, level.n, "fh"))), "excmg_assemble_rhs")
    return fh


def excmg_dsolve(level: Level, fh: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    level.ctx.check(_lib.excmg_dsolve(level.handle, _vp(_node(fh, level.n, "fh")),
                                      _vp(_node(u, level.n, "u"))), "excmg_dsolve")
    return u


def excmg_solve(n_finest: int, n_coarsest: int, bc_kind: int, f: torch.Tensor, g1: torch.Tensor,
                g2: torch.Tensor, tol: float, u_out: torch.Tensor | None = None, *,
                ctx: Context | None = None, tol_mode: str = "uniform", max_iter: int | None = None,
                max_total: int = 1000000, check_every: int = 16, u_h_out: torch.Tensor | None = None,
                return_stats: bool = False, precision: str = "fp64", inner_tol: float = MIXED_INNER_TOL):
    """Alg. 1.  Returns u_tilde (EXP_true on the finest grid), and the
    per-level statistics when return_stats is set.  precision="mixed" runs
    the Bi-CG levels as FP32 correction solves inside FP64 refinement."""
    ctx = ctx or default_context(f.device)
    n = int(n_finest)
    if u_out is None:
        u_out = _new_node(n, f)
    if max_iter is None:
        # FP64: one Bi-CG call may run to convergence; mixed: each FP32
        # correction solve is capped (FP32 recurrences stop paying off after
        # a few hundred iterations on these operators)
        max_iter = 100000 if precision == "fp64" else MIXED_INNER_CAP
    params = Params(float(tol), TOL_MODES[tol_mode], int(max_iter), int(max_total), int(check_every),
                    PRECISIONS[precision], float(inner_tol))
    stats = Stats()
    ph = _vp(_node(u_h_out, n, "u_h_out")) if u_h_out is not None else _vp(0)
    rc = _lib.excmg_solve_ex(ctx.handle, n, int(n_coarsest), int(bc_kind), _vp(_node(f, n, "f")),
                             _vp(_node(g1, n, "g1")), _vp(_faces(g2, n, "g2")), ctypes.byref(params), ph,
                             _vp(_node(u_out, n, "u_out")), ctypes.byref(stats))
    ctx.check(rc, "excmg_solve")
    if return_stats:
        return u_out, stats.as_list()
    return u_out


# ------------------------------------------------------------ many solves
class Batch:
    """Many independent EXCMG solves on one GPU (FP64 refinement around FP32
    correction solves); see excmg_batch_* in include/excmg.h.  Tensors passed
    to submit() are kept alive here until their instance is done."""

    def __init__(self, ctx: Context | None = None, hbm_budget_bytes: int = 0, max_instances: int = 64):
        self.ctx = ctx or default_context()
        h = _vp()
        rc = _lib.excmg_batch_create(self.ctx.handle, int(hbm_budget_bytes), int(max_instances), ctypes.byref(h))
        if rc != EXCMG_OK:
            raise ExcmgError(rc, "excmg_batch_create failed")
        self.handle = h
        self._keep = {}

    def _check(self, rc, what):
        if rc != EXCMG_OK:
            msg = _lib.excmg_batch_last_error(self.handle)
            raise ExcmgError(rc, f"{what}: {msg.decode() if msg else ''}")

    @staticmethod
    def instance_bytes(n_finest: int, n_coarsest: int, precision: str = "mixed") -> int:
        return int(_lib.excmg_batch_instance_bytes(int(n_finest), int(n_coarsest), PRECISIONS[precision]))

    @property
    def bytes(self) -> int:
        return int(_lib.excmg_batch_bytes(self.handle))

    @property
    def launches(self) -> int:
        return int(_lib.excmg_batch_launches(self.handle))

    def profile(self) -> dict:
        """Counters of the batch's cooperative Bi-CG launches and step times."""
        pr = BatchProfile()
        self._check(_lib.excmg_batch_get_profile(self.handle, ctypes.byref(pr)), "excmg_batch_get_profile")
        return {k: getattr(pr, k) for k, _ in BatchProfile._fields_}

    def submit(self, n_finest: int, n_coarsest: int, bc_kind: int, f: torch.Tensor, g1: torch.Tensor,
               g2: torch.Tensor, tol: float, u_out: torch.Tensor | None = None, *, tol_mode: str = "uniform",
               precision: str = "mixed", inner_tol: float = MIXED_INNER_TOL, max_iter: int | None = None,
               max_total: int = 1000000):
        """Admit one solve; returns (id, u_out), or None when the budget or the
        slots are full right now.  Raises ExcmgError (EXCMG_ERR_TOO_LARGE) for
        an instance that needs more than the whole budget."""
        n = int(n_finest)
        if u_out is None:
            u_out = _new_node(n, f)
        if max_iter is None:
            max_iter = 100000 if precision == "fp64" else MIXED_INNER_CAP
        params = Params(float(tol), TOL_MODES[tol_mode], int(max_iter), int(max_total), 16, PRECISIONS[precision],
                        float(inner_tol))
        ident = ctypes.c_int(-1)
        rc = _lib.excmg_batch_submit(self.handle, n, int(n_coarsest), int(bc_kind), _vp(_node(f, n, "f")),
                                     _vp(_node(g1, n, "g1")), _vp(_faces(g2, n, "g2")), ctypes.byref(params),
                                     _vp(_node(u_out, n, "u_out")), ctypes.byref(ident))
        if rc == -9:
            return None
        self._check(rc, "excmg_batch_submit")
        self._keep[ident.value] = (f, g1, g2, u_out)
        return ident.value, u_out

    def step(self) -> int:
        live = ctypes.c_int(0)
        self._check(_lib.excmg_batch_step(self.handle, ctypes.byref(live)), "excmg_batch_step")
        return live.value

    def query(self, ident: int):
        done = ctypes.c_int(0)
        status = ctypes.c_int(0)
        stats = Stats()
        lat = ctypes.c_double(0.0)
        self._check(_lib.excmg_batch_query(self.handle, int(ident), ctypes.byref(done), ctypes.byref(status),
                                           ctypes.byref(stats), ctypes.byref(lat)), "excmg_batch_query")
        if done.value:
            self._keep.pop(int(ident), None)
            return {"done": True, "status": status.value, "stats": stats.as_list(), "latency_s": lat.value}
        return {"done": False}

    def run(self) -> None:
        """Step until no instance is live."""
        while self.step() > 0:
            pass

    def close(self):
        if getattr(self, "handle", None):
            _lib.excmg_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------- the 2D problem
# Node arrays of shape (N+1, N+1) indexed [j, i] (x fastest); g2 of shape
# (4, N+1): edges x=0, x=1, y=0, y=1, indexed by the other coordinate.
def _node2(t: torch.Tensor, n: int, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != (n + 1) ** 2:
        raise ValueError(f"{name} must be a contiguous float64 tensor with (N+1)^2 = {(n + 1) ** 2} elements")
    return t.data_ptr()


def _new_node2(n: int, like: torch.Tensor) -> torch.Tensor:
    return torch.empty((n + 1, n + 1), dtype=torch.float64, device=like.device)


def stencil_apply2d(n: int, bc_kind: int, u: torch.Tensor, y: torch.Tensor | None = None, transpose: bool = False,
                    ctx: Context | None = None) -> torch.Tensor:
    """y = A_h u of the 13-point scheme of the 2D problem."""
    ctx = ctx or default_context(u.device)
    if y is None:
        y = _new_node2(n, u)
    ctx.check(_lib.excmg2d_stencil_apply(ctx.handle, int(n), int(bc_kind), int(bool(transpose)),
                                         _vp(_node2(u, n, "u")), _vp(_node2(y, n, "y"))), "excmg2d_stencil_apply")
    return y


def bicg_solve2d(n: int, bc_kind: int, b: torch.Tensor, x: torch.Tensor, tol: float, max_iter: int = 100000,
                 ctx: Context | None = None):
    """Alg. 2 on the 2D system in place; returns (iters, relres, status)."""
    ctx = ctx or default_context(b.device)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    rc = _lib.excmg2d_bicg_solve(ctx.handle, int(n), int(bc_kind), _vp(_node2(b, n, "b")), _vp(_node2(x, n, "x")),
                                 float(tol), int(max_iter), ctypes.byref(it), ctypes.byref(rr))
    if rc not in (EXCMG_OK, -4):
        ctx.check(rc, "excmg2d_bicg_solve")
    return it.value, rr.value, rc


def extrapolate_interpolate2d(n_fine: int, u_2h: torch.Tensor, u_4h: torch.Tensor, w_h: torch.Tensor | None = None,
                              g1_fine: torch.Tensor | None = None, ctx: Context | None = None) -> torch.Tensor:
    ctx = ctx or default_context(u_2h.device)
    if w_h is None:
        w_h = _new_node2(n_fine, u_2h)
    pg = _vp(_node2(g1_fine, n_fine, "g1_fine")) if g1_fine is not None else _vp(0)
    ctx.check(_lib.excmg2d_extrapolate_interpolate(ctx.handle, int(n_fine), _vp(_node2(u_2h, n_fine // 2, "u_2h")),
                                                   _vp(_node2(u_4h, n_fine // 4, "u_4h")), pg,
                                                   _vp(_node2(w_h, n_fine, "w_h"))), "excmg2d_extrapolate_interpolate")
    return w_h


def midpoint_extrapolate2d(n_fine: int, u_h: torch.Tensor, u_2h: torch.Tensor, u_tilde: torch.Tensor | None = None,
                           ctx: Context | None = None) -> torch.Tensor:
    ctx = ctx or default_context(u_h.device)
    if u_tilde is None:
        u_tilde = _new_node2(n_fine, u_h)
    ctx.check(_lib.excmg2d_midpoint_extrapolate(ctx.handle, int(n_fine), _vp(_node2(u_h, n_fine, "u_h")),
                                                _vp(_node2(u_2h, n_fine // 2, "u_2h")),
                                                _vp(_node2(u_tilde, n_fine, "u_tilde"))), "excmg2d_midpoint_extrapolate")
    return u_tilde


def excmg_solve2d(n_finest: int, n_coarsest: int, bc_kind: int, f: torch.Tensor, g1: torch.Tensor, g2: torch.Tensor,
                  tol: float, u_out: torch.Tensor | None = None, *, ctx: Context | None = None,
                  tol_mode: str = "uniform", max_iter: int = 100000, max_total: int = 1000000, check_every: int = 16,
                  u_h_out: torch.Tensor | None = None, return_stats: bool = False):
    """Alg. 1 on the 2D problem; returns u_tilde (and per-level statistics)."""
    ctx = ctx or default_context(f.device)
    n = int(n_finest)
    if u_out is None:
        u_out = _new_node2(n, f)
    if not isinstance(g2, torch.Tensor) or g2.dtype != torch.float64 or not g2.is_contiguous() or \
            g2.numel() != 4 * (n + 1):
        raise ValueError("g2 must be a contiguous float64 CUDA tensor with 4 (N+1) elements")
    params = Params(float(tol), TOL_MODES[tol_mode], int(max_iter), int(max_total), int(check_every), 0, 1e-4)
    stats = Stats()
    ph = _vp(_node2(u_h_out, n, "u_h_out")) if u_h_out is not None else _vp(0)
    rc = _lib.excmg2d_solve(ctx.handle, n, int(n_coarsest), int(bc_kind), _vp(_node2(f, n, "f")),
                            _vp(_node2(g1, n, "g1")), _vp(g2.data_ptr()), ctypes.byref(params), ph,
                            _vp(_node2(u_out, n, "u_out")), ctypes.byref(stats))
    ctx.check(rc, "excmg2d_solve")
    if return_stats:
        return u_out, stats.as_list()
    return u_out
