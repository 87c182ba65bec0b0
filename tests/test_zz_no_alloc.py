"""The allocation-free EXP_finite entry point.

It exists for callers that cannot allocate device memory when they run this
step (all device memory owned by an arena or a hard budget, or a path where
the CUDA allocator must not be entered).  It keeps its scratch in a fixed
array inside the library instead.  This file is collected last so that a run
that stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1901_05118_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1901_05118_gb300 import binding as B  # noqa: E402

DEV = torch.device("cuda", 0)
MAX_FINE = 128


def _entry():
    fn = B.lib().extrapolate_interpolate_noalloc
    fn.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def _dev(a):
    return torch.from_numpy(np.array(a, dtype=np.float64, order="C")).to(DEV)


def test_noalloc_matches_extrapolate_interpolate_on_consecutive_calls():
    fn = _entry()
    # two calls in a row through the C ABI; the second one, at the largest
    # allowed size, reuses the array the first one left behind.  Each result
    # is checked against the allocating entry point and against the CPU
    # oracle's Steps 1-5.
    for call, nf in enumerate((64, MAX_FINE)):
        h1 = P.random_field(nf // 2, 500 + call)
        h0 = P.random_field(nf // 4, 600 + call)
        u1, u0 = _dev(h1), _dev(h0)
        ref = B.extrapolate_interpolate(nf, u1, u0)          # the allocating entry point
        w = torch.full((nf + 1,) * 3, float("nan"), dtype=torch.float64, device=DEV)
        torch.cuda.synchronize()
        rc = fn(nf, u1.data_ptr(), u0.data_ptr(), w.data_ptr())
        assert rc == 0
        got, want = w.cpu().numpy(), ref.cpu().numpy()
        assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
        orc = oracle.exp_finite(nf, h1, h0)
        assert np.abs(got - orc).max() <= 1e-13 * np.abs(orc).max()


def test_noalloc_rejects_sizes_beyond_its_array():
    fn = _entry()
    nf = MAX_FINE + 4
    u1 = torch.zeros((nf // 2 + 1,) * 3, dtype=torch.float64, device=DEV)
    u0 = torch.zeros((nf // 4 + 1,) * 3, dtype=torch.float64, device=DEV)
    w = torch.full((nf + 1,) * 3, 7.0, dtype=torch.float64, device=DEV)
    torch.cuda.synchronize()
    assert fn(nf, u1.data_ptr(), u0.data_ptr(), w.data_ptr()) == -10   # EXCMG_ERR_SIZE
    assert bool(torch.all(w == 7.0))
