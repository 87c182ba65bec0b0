"""The 2D problem (eq. (bvp2d)) through the C ABI against the 2D CPU oracle.

Tolerances as for 3D: one operator application within 1e-12 relative in the
max norm, transfers 1e-13, Bi-CG iterates after a fixed number of steps and
whole solves 1e-9."""
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


def dev(a):
    return torch.from_numpy(np.array(a, dtype=np.float64, order="C")).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_max(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


@pytest.mark.parametrize("n", [4, 9, 33, 64, 100])
@pytest.mark.parametrize("bc_kind", [1, 2])
@pytest.mark.parametrize("transpose", [False, True])
def test_stencil2d_random(n, bc_kind, transpose):
    u = P.random_field_2d(n, 21 + n)
    y = host(B.stencil_apply2d(n, bc_kind, dev(u), transpose=transpose))
    ref = oracle.stencil_apply2d(n, bc_kind, u, transpose=transpose)
    assert rel_max(y, ref) <= 1e-12


def test_stencil2d_smooth_and_nonfinite():
    n = 48
    u = P.exp_sum_2d().exact(n)
    y = host(B.stencil_apply2d(n, 1, dev(u)))
    ref = oracle.stencil_apply2d(n, 1, u)
    assert np.abs(y - ref).max() <= 1e-12 * 64 * np.abs(u).max()
    u[10, 10] = np.nan
    y = host(B.stencil_apply2d(n, 1, dev(u)))
    assert np.isnan(y[10, 10])


@pytest.mark.parametrize("nf", [8, 20, 64])
def test_transfers2d(nf):
    u1 = P.random_field_2d(nf // 2, 31 + nf)
    u0 = P.random_field_2d(nf // 4, 32 + nf)
    w = host(B.extrapolate_interpolate2d(nf, dev(u1), dev(u0)))
    assert rel_max(w, oracle.exp_finite2d(nf, u1, u0)) <= 1e-13
    g1 = P.random_field_2d(nf, 33 + nf)
    wb = host(B.extrapolate_interpolate2d(nf, dev(u1), dev(u0), g1_fine=dev(g1)))
    inner = (slice(1, nf), slice(1, nf))
    assert rel_max(wb[inner], w[inner]) == 0.0
    mask = np.ones_like(wb, dtype=bool)
    mask[inner] = False
    np.testing.assert_array_equal(wb[mask], g1[mask])
    uh = P.random_field_2d(nf, 34 + nf)
    ut = host(B.midpoint_extrapolate2d(nf, dev(uh), dev(u1)))
    assert rel_max(ut, oracle.exp_true2d(nf, uh, u1)) <= 1e-13


@pytest.mark.parametrize("n,bc_kind", [(40, 1), (67, 2)])
def test_bicg2d_fixed_iterations(n, bc_kind):
    b = P.random_field_2d(n, 41)
    x0 = P.random_field_2d(n, 42) * 0.1
    x = dev(x0)
    it, rel, rc = B.bicg_solve2d(n, bc_kind, dev(b), x, 0.0, 20)
    xr, itr, relr, rcr = oracle.bicg2d(n, bc_kind, b, x0, 0.0, max_iter=20)
    assert it == itr == 20
    assert rel == pytest.approx(relr, rel=1e-8)
    assert rel_max(host(x), xr) <= 1e-10



@pytest.mark.parametrize("bc_kind", [1, 2])
@pytest.mark.parametrize("name", ["sin_pi_2d", "exp_sum_2d"])
def test_excmg2d_matches_oracle(bc_kind, name):
    n, nc = 64, 4
    prob = getattr(P, name)()
    f, g1, g2 = prob.data(n, bc_kind)
    uh = torch.empty((n + 1, n + 1), dtype=torch.float64, device=DEV)
    ut, stats = B.excmg_solve2d(n, nc, bc_kind, dev(f), dev(g1), dev(g2), 1e-10, u_h_out=uh, return_stats=True)
    ref_h, ref_t, ref_stats = oracle.excmg2d(n, nc, bc_kind, f, g1, g2, 1e-10)
    assert rel_max(host(uh), ref_h) <= 1e-9
    assert rel_max(host(ut), ref_t) <= 1e-9
    # Iteration counts are compared only where every stopping decision is
    # clear of the tolerance (the capped test below): on these 2D systems the
    # Bi-CG residual is not monotone and grazes 1e-10 for dozens of steps, so
    # a rounding difference of 1e-16 moves the stop by many iterations (a CPU
    # emulation of the 128^2 level with the exactly rounded operator stops at
    # 1952 steps, the oracle at 817: the minimum relative residual near step
    # 817 is 1.00005e-10 in one run and 0.99960e-10 in the other, and the
    # next crossing comes at step 1952).
    for s in stats:
        assert s["relres"] <= 1e-10 or s["stagnated"]
    for l in range(len(stats)):
        assert ref_stats[l, 1] <= 1e-10 or ref_stats[l, 3]


@pytest.mark.parametrize("bc_kind", [1, 2])
def test_excmg2d_128_matches_oracle_to_the_algebraic_error(bc_kind):
    """At 128^2 a level takes up to ~2000 Bi-CG steps on a matrix with
    condition number ~4e7, so two FP64 runs whose operator rounds differently
    reach different solutions with the same residual bound; their distance is
    bounded by the algebraic error (cond * tol), which lies far below the
    discretisation error.  Both meet the tolerance on every level, and u_h,
    u~ agree to 1e-3 of the discretisation error of the oracle's u_h."""
    n, nc = 128, 8
    prob = P.sin_pi_2d()
    f, g1, g2 = prob.data(n, bc_kind)
    uh = torch.empty((n + 1, n + 1), dtype=torch.float64, device=DEV)
    ut, stats = B.excmg_solve2d(n, nc, bc_kind, dev(f), dev(g1), dev(g2), 1e-10, u_h_out=uh, return_stats=True)
    ref_h, ref_t, ref_stats = oracle.excmg2d(n, nc, bc_kind, f, g1, g2, 1e-10)
    disc = np.abs(ref_h - prob.exact(n)).max()
    assert np.abs(host(uh) - ref_h).max() <= 1e-3 * disc
    assert np.abs(host(ut) - ref_t).max() <= 1e-3 * disc
    for l, s in enumerate(stats):
        assert s["relres"] <= 1e-10 or s["stagnated"]
        assert ref_stats[l, 1] <= 1e-10 or ref_stats[l, 3]


def test_excmg2d_capped_iterations_match_oracle():
    """With few Bi-CG steps per call, every stopping decision is the same on
    both sides: counts of iterations, calls and stagnation flags agree."""
    n, nc = 128, 4
    prob = P.exp_sum_2d()
    f, g1, g2 = prob.data(n, 2)
    uh = torch.empty((n + 1, n + 1), dtype=torch.float64, device=DEV)
    ut, stats = B.excmg_solve2d(n, nc, 2, dev(f), dev(g1), dev(g2), 1e-12, u_h_out=uh, return_stats=True,
                                max_iter=12, max_total=48)
    ref_h, ref_t, ref_stats = oracle.excmg2d(n, nc, 2, f, g1, g2, 1e-12, max_iter=12, max_total=48)
    assert [s["iters"] for s in stats] == [int(v) for v in ref_stats[:, 0]]
    assert [s["calls"] for s in stats] == [int(v) for v in ref_stats[:, 2]]
    assert [int(s["stagnated"]) for s in stats] == [int(v) for v in ref_stats[:, 3]]
    assert rel_max(host(uh), ref_h) <= 1e-9
    assert rel_max(host(ut), ref_t) <= 1e-9


def test_excmg2d_second_order():
    """Every level meets the tolerance and the error of u_h against the exact
    solution falls like h^2 from 256 to 512 (the oracle measures 2.513e-5 at
    256 with this tolerance; the algebraic error left by a relative residual
    of 1e-10 moves it by about 0.1 %)."""
    prob = P.sin_pi_2d()
    err = {}
    for n in (256, 512):
        f, g1, g2 = (dev(a) for a in prob.data(n, 1))
        uh = torch.empty((n + 1, n + 1), dtype=torch.float64, device=DEV)
        _, stats = B.excmg_solve2d(n, 8, 1, f, g1, g2, 1e-10, u_h_out=uh, return_stats=True)
        for s in stats[2:]:
            assert s["relres"] <= 1e-10 or s["stagnated"]
        err[n] = float((uh - dev(prob.exact(n))).abs().max())
    assert err[256] == pytest.approx(2.513e-5, rel=5e-3)
    assert 3.8 <= err[256] / err[512] <= 4.2
