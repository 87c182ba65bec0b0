"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: a single operator application must match within 1e-12 relative
in the max norm; on smooth inputs (where A u is tiny next to its terms) the
yardstick is 1e-12 * max |A||u|, i.e. 1e-12 * 144 max|u|.  Transfers are
evaluated to rounding (1e-13 relative).  Full solves must match within 1e-9
relative in the max norm.
"""
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
    d = np.abs(a - b).max()
    s = np.abs(b).max()
    return d / s if s > 0 else d


# ------------------------------------------------------------ operator
VARIANTS = ["exact", "fp64"]


def level(n, bc_kind, variant="exact", schedule="separate"):
    ctx = B.Context()
    ctx.set_stencil(variant)
    ctx.set_schedule(schedule)
    return B.Level(n, bc_kind, ctx)


SCHEDULES = ["separate", "fused"]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n", [4, 5, 8, 33, 64])
@pytest.mark.parametrize("bc_kind", [1, 2])
@pytest.mark.parametrize("transpose", [False, True])
def test_stencil_random(n, bc_kind, transpose, variant):
    u = P.random_field(n, 100 + n)   # boundary entries non-zero: must be ignored
    lvl = level(n, bc_kind, variant)
    y = host(B.stencil_apply(lvl, dev(u), transpose=transpose))
    ref = oracle.stencil_apply(n, bc_kind, u, transpose=transpose)
    assert rel_max(y, ref) <= 1e-12
    mask = np.ones_like(y, dtype=bool)
    mask[1:-1, 1:-1, 1:-1] = False
    assert np.all(y[mask] == 0.0)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n,bc_kind", [(48, 1), (48, 2)])
def test_stencil_smooth(n, bc_kind, variant):
    u = P.exp_sum().exact(n)
    lvl = level(n, bc_kind, variant)
    y = host(B.stencil_apply(lvl, dev(u)))
    ref = oracle.stencil_apply(n, bc_kind, u)
    assert np.abs(y - ref).max() <= 1e-12 * 144 * np.abs(u).max()


def test_stencil_full_size_512():
    """The workload's size (512 intervals: 511^3 unknowns), both kinds, both
    arithmetic variants, and A^T."""
    n = 512
    u = P.random_field(n, 7)
    du = dev(u)
    for bc in (1, 2):
        ref = oracle.stencil_apply(n, bc, u)
        for variant in VARIANTS:
            lvl = level(n, bc, variant)
            y = host(B.stencil_apply(lvl, du))
            assert rel_max(y, ref) <= 1e-12
        yt = host(B.stencil_apply(level(n, bc), du, transpose=True))
        assert rel_max(yt, ref) <= 1e-12


def test_stencil_exact_variant_is_order_free():
    """The integer variant sums exactly, so A u and the mirrored-tap gather
    A^T u agree bit for bit (A_h is symmetric)."""
    n = 40
    u = dev(P.random_field(n, 77))
    lvl = level(n, 1)
    assert torch.equal(B.stencil_apply(lvl, u), B.stencil_apply(lvl, u, transpose=True))


def test_stencil_wide_dynamic_range():
    """Inputs spanning 1e-300 .. 1e300 (and zeros) stay within the error
    bound relative to the largest magnitude each block reads."""
    n = 24
    rng = np.random.Generator(np.random.PCG64(5))
    u = rng.uniform(-1, 1, (n + 1,) * 3) * 10.0 ** rng.integers(-300, 300, (n + 1,) * 3)
    u[rng.uniform(size=u.shape) < 0.2] = 0.0
    ref = oracle.stencil_apply(n, 2, u)
    y = host(B.stencil_apply(level(n, 2), dev(u)))
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(u).max()
    tiny = P.random_field(n, 8) * 1e-310   # subnormal inputs
    ref = oracle.stencil_apply(n, 1, tiny)
    y = host(B.stencil_apply(level(n, 1), dev(tiny)))
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(tiny).max() + 1e-323


def test_stencil_nonfinite_propagates():
    n = 16
    u = P.random_field(n, 9)
    u[8, 8, 8] = np.nan
    y = host(B.stencil_apply(level(n, 1), dev(u)))
    assert np.isnan(y[8, 8, 8])


# ----------------------------------------------------- right-hand side
@pytest.mark.parametrize("n,stride", [(4, 1), (8, 2), (13, 1), (16, 4)])
@pytest.mark.parametrize("bc_kind", [1, 2])
def test_assemble_rhs(n, stride, bc_kind):
    ns = n * stride
    prob = P.paper_problem2()
    f, g1, g2 = prob.data(ns, bc_kind)
    lvl = B.Level(n, bc_kind)
    fh = host(B.excmg_assemble_rhs(lvl, ns, dev(f), dev(g1), dev(g2)))
    ref = oracle.assemble_rhs(n, bc_kind, oracle.inject_nodes(ns, stride, f), oracle.inject_nodes(ns, stride, g1),
                              oracle.inject_faces(ns, stride, g2))
    assert np.abs(fh - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())


# ---------------------------------------------------------- transfers
@pytest.mark.parametrize("nf", [8, 16, 40])
def test_extrapolate_interpolate(nf):
    u1 = P.random_field(nf // 2, 1 + nf)
    u0 = P.random_field(nf // 4, 2 + nf)
    w = host(B.extrapolate_interpolate(nf, dev(u1), dev(u0)))
    ref = oracle.exp_finite(nf, u1, u0)
    assert rel_max(w, ref) <= 1e-13


@pytest.mark.parametrize("nf", [8, 40])
def test_extrapolate_interpolate_takes_boundary_from_g1(nf):
    """With g1_fine, w_h's boundary nodes hold g1's boundary values (Alg. 1
    sets the Dirichlet data before Bi-CG); interior nodes are Steps 1-5."""
    u1 = P.random_field(nf // 2, 11 + nf)
    u0 = P.random_field(nf // 4, 12 + nf)
    g1 = P.random_field(nf, 13 + nf)
    w = host(B.extrapolate_interpolate(nf, dev(u1), dev(u0), g1_fine=dev(g1)))
    ref = oracle.exp_finite(nf, u1, u0)
    inner = (slice(1, nf), slice(1, nf), slice(1, nf))
    assert rel_max(w[inner], ref[inner]) <= 1e-13
    mask = np.ones_like(w, dtype=bool)
    mask[inner] = False
    np.testing.assert_array_equal(w[mask], g1[mask])


@pytest.mark.parametrize("nf", [4, 10, 64])
def test_midpoint_extrapolate(nf):
    uh = P.random_field(nf, 3 + nf)
    u2 = P.random_field(nf // 2, 4 + nf)
    ut = host(B.midpoint_extrapolate(nf, dev(uh), dev(u2)))
    ref = oracle.exp_true(nf, uh, u2)
    assert rel_max(ut, ref) <= 1e-13


# ------------------------------------------------------------ DSOLVE
@pytest.mark.parametrize("n", [4, 8, 16])
@pytest.mark.parametrize("bc_kind", [1, 2])
def test_dsolve(n, bc_kind):
    fh = P.random_field(n, 9)
    fh[0] = fh[-1] = 0.0
    lvl = B.Level(n, bc_kind)
    u = torch.zeros((n + 1,) * 3, dtype=torch.float64, device=DEV)
    got = host(B.excmg_dsolve(lvl, dev(fh), u))
    ref = oracle.dsolve(n, bc_kind, fh, np.zeros_like(fh))
    assert rel_max(got, ref) <= 1e-10


# ------------------------------------------------------------- Bi-CG
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n,bc_kind", [(12, 1), (17, 2), (40, 1)])
def test_bicg(n, bc_kind, variant):
    b = P.random_field(n, 31)
    x0 = P.random_field(n, 32) * 0.1
    lvl = level(n, bc_kind, variant)
    x = dev(x0)
    it, rel, rc = B.bicg_solve(lvl, dev(b), x, 1e-12, 5000)
    xr, itr, relr, rcr = oracle.bicg(n, bc_kind, b, x0, 1e-12)
    assert rc == 0 and rcr == 0
    # iteration counts are not pinned (rounding shifts them over hundreds of steps)
    assert abs(it - itr) <= max(3, 0.05 * itr)
    assert rel <= 1e-12
    assert rel_max(host(x), xr) <= 1e-9


def test_bicg_is_deterministic():
    """The reductions add their partial sums in a fixed order, so two runs
    on the same input give the same iterate bit for bit."""
    n = 24
    b = dev(P.random_field(n, 41))
    x1 = torch.zeros((n + 1,) * 3, dtype=torch.float64, device=DEV)
    x2 = torch.zeros_like(x1)
    lvl = level(n, 1)
    r1 = B.bicg_solve(lvl, b, x1, 1e-11, 2000)
    r2 = B.bicg_solve(lvl, b, x2, 1e-11, 2000)
    assert r1 == r2 and torch.equal(x1, x2)


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("n,bc_kind", [(138, 1), (133, 2)])
def test_bicg_large_grid_fixed_iterations(n, bc_kind, schedule):
    """Grids above 64^3 run the launched kernels (ragged tiles in x, y and z
    here), in both schedules (the fused one forms p, p* inside the operator
    launch from staged rows): 20 iterations of Alg. 2 against the oracle's
    20, iterates entry by entry."""
    b = P.random_field(n, 81)
    x0 = P.random_field(n, 82) * 0.1
    lvl = level(n, bc_kind, schedule=schedule)
    x = dev(x0)
    it, rel, rc = B.bicg_solve(lvl, dev(b), x, 0.0, 20)
    xr, itr, relr, rcr = oracle.bicg(n, bc_kind, b, x0, 0.0, max_iter=20)
    assert it == itr == 20
    assert rel == pytest.approx(relr, rel=1e-8)
    assert rel_max(host(x), xr) <= 1e-10


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_bicg_large_grid_is_deterministic(schedule):
    n = 144
    b = dev(P.random_field(n, 83))
    x1 = torch.zeros((n + 1,) * 3, dtype=torch.float64, device=DEV)
    x2 = torch.zeros_like(x1)
    lvl = level(n, 1, schedule=schedule)
    r1 = B.bicg_solve(lvl, b, x1, 0.0, 37)
    r2 = B.bicg_solve(lvl, b, x2, 0.0, 37)
    assert r1 == r2 and torch.equal(x1, x2)


# ---------------------------------------------------------- full solve
@pytest.mark.parametrize("name,bc_kind,variant", [("sin_pi", 1, "exact"), ("exp_sum", 1, "exact"),
                                                   ("exp_sum", 2, "exact"), ("paper_p4", 1, "exact"),
                                                   ("sin_pi", 1, "fp64"), ("exp_sum", 2, "fp64")])
def test_excmg_solve_matches_oracle(name, bc_kind, variant):
    """The small workload: 4^3 .. 32^3, tol 1e-10 on every level."""
    n, nc = 32, 4
    prob = P.by_name(name)
    f, g1, g2 = prob.data(n, bc_kind)
    uh = torch.empty((n + 1,) * 3, dtype=torch.float64, device=DEV)
    ctx = B.Context()
    ctx.set_stencil(variant)
    ut, stats = B.excmg_solve(n, nc, bc_kind, dev(f), dev(g1), dev(g2), 1e-10, u_h_out=uh, return_stats=True,
                              ctx=ctx)
    ref_h, ref_t, ref_stats = oracle.excmg(n, nc, bc_kind, f, g1, g2, 1e-10)
    assert rel_max(host(uh), ref_h) <= 1e-9
    assert rel_max(host(ut), ref_t) <= 1e-9
    for l, s in enumerate(stats):
        assert s["relres"] <= 1e-10 or s["stagnated"]
        # iteration counts are not pinned by the paper; rounding differences
        # shift them slightly over hundreds of iterations
        assert abs(s["iters"] - ref_stats[l, 0]) <= max(3, 0.05 * ref_stats[l, 0])


_ORACLE_128 = {}
# (tolerance schedule, tol, Bi-CG cap per call of the WHILE loop, cap per
# level).  The small per-call cap makes the loop restart Bi-CG several times
# per level and end levels on the stagnation rule.  In the paper's schedule
# the 32^3 level (eps / 100) is held to 60 iterations: stopping decisions
# taken after hundreds of Bi-CG steps can fall one iteration apart between
# two correct FP64 runs (their rounding differs), while decisions after a
# few dozen steps, and a cap, are the same on both sides; the 64^3 level
# still runs to its paper tolerance eps / 10.
CASES_128 = [("uniform", 1e-6, 100000, 400), ("paper", 1e-6, 100000, 60), ("uniform", 1e-8, 8, 400)]


def _oracle_128(bc_kind, case):
    """The oracle's solve of the 128^3 case, computed once per session."""
    key = (bc_kind, case)
    if key not in _ORACLE_128:
        tol_mode, tol, max_iter, max_total = case
        f, g1, g2 = P.exp_sum().data(128, bc_kind)
        _ORACLE_128[key] = oracle.excmg(128, 8, bc_kind, f, g1, g2, tol, tol_mode=tol_mode, max_iter=max_iter,
                                        max_total=max_total)
    return _ORACLE_128[key]


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("case", CASES_128)
@pytest.mark.parametrize("bc_kind", [1, 2])
def test_excmg_solve_128_matches_oracle(bc_kind, case, schedule):
    """Alg. 1 on 8^3 .. 128^3 (u = e^(x+y+z)): the 32^3 and 64^3 levels run
    the cooperative kernels and the 128^3 level the launched operator /
    update / direction-update kernels (in both operator schedules), inside
    the WHILE loop with its restarts, stagnation rule and EXP_finite
    hand-offs, under both tolerance schedules (Alg. 1 and uniform).  Every level
    takes the oracle's Bi-CG iterations and calls and ends the same way; u_h
    and u~ match the oracle's entry by entry."""
    tol_mode, tol, max_iter, max_total = case
    n, nc = 128, 8
    f, g1, g2 = P.exp_sum().data(n, bc_kind)
    ctx = B.Context()
    ctx.set_schedule(schedule)
    uh = torch.empty((n + 1,) * 3, dtype=torch.float64, device=DEV)
    ut, stats = B.excmg_solve(n, nc, bc_kind, dev(f), dev(g1), dev(g2), tol, tol_mode=tol_mode, max_iter=max_iter,
                              max_total=max_total, u_h_out=uh, return_stats=True, ctx=ctx)
    ref_h, ref_t, ref_stats = _oracle_128(bc_kind, case)
    assert [s["iters"] for s in stats] == [int(v) for v in ref_stats[:, 0]]
    assert [s["calls"] for s in stats] == [int(v) for v in ref_stats[:, 2]]
    assert [int(s["stagnated"]) for s in stats] == [int(v) for v in ref_stats[:, 3]]
    assert rel_max(host(uh), ref_h) <= 1e-9
    assert rel_max(host(ut), ref_t) <= 1e-9
    L = len(stats) - 2
    for l, st in enumerate(stats[2:], start=2):
        eps_i = tol * (10.0 ** (l - 1 - L) if tol_mode == "paper" else 1.0)
        assert st["relres"] <= eps_i or st["stagnated"] or st["iters"] == max_total
        assert st["relres"] == pytest.approx(ref_stats[l, 1], rel=1e-6)


def test_excmg_exact_for_triquadratic():
    prob = P.polynomial([0.5, -0.3, 0.8], [1.0, 0.2, -0.6], [0.1, 0.7, 0.3])
    n = 32
    f, g1, g2 = prob.data(n, 1)
    uh = torch.empty((n + 1,) * 3, dtype=torch.float64, device=DEV)
    ut, stats = B.excmg_solve(n, 4, 1, dev(f), dev(g1), dev(g2), 1e-12, u_h_out=uh, return_stats=True)
    ue = prob.exact(n)
    assert np.abs(host(uh) - ue).max() <= 1e-11
    assert np.abs(host(ut) - ue).max() <= 1e-11
    assert all(s["iters"] == 0 for s in stats)


def test_excmg_paper_table_rows_64():
    """Tables 1-2 rows at 32^3 and 64^3 through the GPU path (8^3, 16^3 solved
    directly as in the paper)."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))["problems"]
    for name in ("paper_p1", "paper_p2"):
        prob = P.by_name(name)
        n = 64
        f, g1, g2 = prob.data(n, 1)
        uh = torch.empty((n + 1,) * 3, dtype=torch.float64, device=DEV)
        B.excmg_solve(n, 8, 1, dev(f), dev(g1), dev(g2), 1e-11, u_h_out=uh)
        e = host(uh) - prob.exact(n)
        l2 = np.sqrt((e ** 2).mean())
        linf = np.abs(e).max()
        assert l2 == pytest.approx(gold[name]["rows"]["64"]["l2"], rel=0.006)
        assert linf == pytest.approx(gold[name]["rows"]["64"]["linf"], rel=0.006)


def test_excmg_paper_table_rows_128_256():
    """Table 1 (Test Problem 1, first kind) at 128^3 and 256^3 through the GPU
    path: error norms of u_h within 5 % of the printed ones.  The paper's
    solves stopped early (8 Bi-CG iterations at 256^3) at a tolerance it does
    not state, so its last digits carry an algebraic error of the size of
    ||w_h - u_h|| (5 % at 256^3); ours do not change between tolerances 1e-7
    and 1e-13.  P1's f_h is small, and the true relative residual has an FP64
    floor near 1e-8 at 256^3: tol 1e-7 stays above it."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))["problems"]
    prob = P.by_name("paper_p1")
    for n in (128, 256):
        f, g1, g2 = prob.data(n, 1)
        uh = torch.empty((n + 1,) * 3, dtype=torch.float64, device=DEV)
        B.excmg_solve(n, 8, 1, dev(f), dev(g1), dev(g2), 1e-7, u_h_out=uh)
        e = host(uh) - prob.exact(n)
        assert np.sqrt((e ** 2).mean()) == pytest.approx(gold["paper_p1"]["rows"][str(n)]["l2"], rel=0.05)
        assert np.abs(e).max() == pytest.approx(gold["paper_p1"]["rows"][str(n)]["linf"], rel=0.05)


@pytest.mark.parametrize("bc_kind", [1, 2])
def test_excmg_full_size_converges(bc_kind):
    """The full-size workload (u = e^(x+y+z), 512^3, coarsest 8^3, tol 1e-10):
    every Bi-CG level meets the tolerance without stagnating; the finest
    u_h's residual, formed again through the public calls (RHS assembly and
    stencil_apply, both checked against the oracle elsewhere), meets it too;
    and u_h is close to the exact solution.  The error's convergence order
    is asserted only for first-kind data (error falls about 3x from 256^3):
    with second-kind data the O(h^2) error at 512^3 (a few 1e-9) lies below
    the algebraic error that tol 1e-10 leaves (measured 6e-8)."""
    prob = P.exp_sum()
    l2 = {}
    for n in (256, 512):
        f, g1, g2 = (dev(a) for a in prob.data(n, bc_kind))
        uh = torch.empty((n + 1,) * 3, dtype=torch.float64, device=DEV)
        _, stats = B.excmg_solve(n, 8, bc_kind, f, g1, g2, 1e-10, u_h_out=uh, return_stats=True)
        for s in stats[2:]:
            assert s["relres"] <= 1e-10 and not s["stagnated"]
        lvl = B.Level(n, bc_kind)
        fh = B.excmg_assemble_rhs(lvl, n, f, g1, g2)
        r = fh - B.stencil_apply(lvl, uh)
        assert float(r.norm() / fh.norm()) <= 1.001e-10
        del f, g1, g2, fh, r
        ue = torch.from_numpy(prob.exact(n)).to(DEV)
        l2[n] = float((uh - ue).pow(2).mean().sqrt())
        assert float((uh - ue).abs().max()) <= 1e-6 * float(ue.abs().max())
        del uh, ue
    if bc_kind == 1:
        assert l2[256] / l2[512] >= 2.5


# ------------------------------------------------------------ errors
def test_bad_arguments_raise():
    lvl = B.Level(8, 1)
    u = torch.zeros(9 ** 3, dtype=torch.float64, device=DEV)
    with pytest.raises(B.ExcmgError):
        B.stencil_apply(lvl, u, u)
    with pytest.raises(ValueError):
        B.stencil_apply(lvl, torch.zeros(10, dtype=torch.float64, device=DEV))
    f = torch.zeros((17,) * 3, dtype=torch.float64, device=DEV)
    g2 = torch.zeros((6, 17, 17), dtype=torch.float64, device=DEV)
    with pytest.raises(B.ExcmgError):
        B.excmg_solve(16, 3, 1, f, f, g2, 1e-8)   # coarsest below 4
    with pytest.raises(B.ExcmgError):
        B.excmg_solve(16, 8, 1, f, f, g2, 1e-8)   # L = 0
    with pytest.raises(B.ExcmgError):
        B.excmg_solve(16, 4, 3, f, f, g2, 1e-8)   # bc_kind


# ------------------------------------------- FP32 inner + FP64 refinement
@pytest.mark.parametrize("bc_kind", [1, 2])
def test_mixed_precision_solve(bc_kind):
    """FP32 correction solves inside FP64 refinement reach the same FP64
    residual tolerance on every level, and the result's distance from the
    oracle's FP64 solution is negligible next to the discretisation error."""
    n, nc = 32, 4
    prob = P.sin2pi_plus_poly()
    f, g1, g2 = prob.data(n, bc_kind)
    uh = torch.empty((n + 1,) * 3, dtype=torch.float64, device=DEV)
    ut, stats = B.excmg_solve(n, nc, bc_kind, dev(f), dev(g1), dev(g2), 1e-10, u_h_out=uh,
                              return_stats=True, precision="mixed", inner_tol=1e-4)
    ref_h, ref_t, _ = oracle.excmg(n, nc, bc_kind, f, g1, g2, 1e-10)
    ue = prob.exact(n)
    disc = np.abs(ref_h - ue).max()
    assert np.abs(host(uh) - ref_h).max() <= 1e-3 * disc
    assert np.abs(host(ut) - ref_t).max() <= 1e-3 * disc
    for s in stats[2:]:
        assert s["relres"] <= 1e-10 or s["stagnated"]
        assert s["calls"] >= 1


def test_mixed_precision_exact_polynomial():
    prob = P.polynomial([0.5, -0.3, 0.8], [1.0, 0.2, -0.6], [0.1, 0.7, 0.3])
    n = 32
    f, g1, g2 = prob.data(n, 1)
    ut = B.excmg_solve(n, 4, 1, dev(f), dev(g1), dev(g2), 1e-12, precision="mixed")
    assert np.abs(host(ut) - prob.exact(n)).max() <= 1e-11


def chosen_shadow(b, n, kind):
    """r*_0 for the tests of Alg. 2 with r*_0 != r_0 (x_0 = 0, so r_0 = b):
    an unrelated random field, or r_0 perturbed by 1 % entry by entry.  The
    perturbed one keeps the two-sided recurrences far from breakdown, so
    rounding differences stay small and iterates can be compared tightly;
    with an unrelated field the iteration count swings by tens of percent
    with rounding alone."""
    noise = P.random_field(n, 52)
    return noise if kind == "random" else b * (1.0 + 0.01 * noise)


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_bicg_with_chosen_shadow_zmarch_fixed_iterations(schedule):
    """Alg. 2 with r*_0 != r_0 in the cooperative kernel's z-march on 60^3
    (the fused schedule stages the rows and folds the direction update in):
    40 iterations on both sides, iterates compared entry by entry.  (A
    tolerance-driven run needs thousands of iterations on such grids, far too
    slow for the oracle.)"""
    n, bc_kind = 60, 2
    b = P.random_field(n, 51)
    shadow = chosen_shadow(b, n, "perturbed")
    lvl = level(n, bc_kind, schedule=schedule)
    x = torch.zeros((n + 1,) * 3, dtype=torch.float64, device=DEV)
    it, rel, rc = B.bicg_solve(lvl, dev(b), x, 0.0, 40, shadow=dev(shadow))
    xr, itr, relr, rcr = oracle.bicg(n, bc_kind, b, np.zeros_like(b), 0.0, max_iter=40, shadow=shadow)
    assert it == itr == 40
    assert rel == pytest.approx(relr, rel=1e-8)
    assert rel_max(host(x), xr) <= 1e-10


@pytest.mark.parametrize("n,bc_kind,kind", [(20, 1, "random")])
def test_bicg_with_chosen_shadow(n, bc_kind, kind):
    """Alg. 2 with r*_0 != r_0 to convergence: the shadow sequence now
    differs from the primal one, so A^T p* is applied to a different vector
    (per-node operator of the cooperative kernel on 20^3)."""
    b = P.random_field(n, 51)
    shadow = chosen_shadow(b, n, kind)
    lvl = level(n, bc_kind)
    x = torch.zeros((n + 1,) * 3, dtype=torch.float64, device=DEV)
    it, rel, rc = B.bicg_solve(lvl, dev(b), x, 1e-11, 20000, shadow=dev(shadow))
    xr, itr, relr, rcr = oracle.bicg(n, bc_kind, b, np.zeros_like(b), 1e-11, shadow=shadow)
    assert rc == 0 and rcr == 0 and rel <= 1e-11
    assert abs(it - itr) <= max(3, 0.05 * itr)
    assert rel_max(host(x), xr) <= 1e-8


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_bicg_with_chosen_shadow_large_grid_fixed_iterations(schedule):
    """The launched (non-cooperative) kernels with a differing shadow, both
    schedules: 20 iterations of Alg. 2 on both sides, iterates compared
    entry by entry."""
    n, bc_kind = 132, 2
    b = P.random_field(n, 71)
    shadow = chosen_shadow(b, n, "perturbed")
    lvl = level(n, bc_kind, schedule=schedule)
    x = torch.zeros((n + 1,) * 3, dtype=torch.float64, device=DEV)
    it, rel, rc = B.bicg_solve(lvl, dev(b), x, 0.0, 20, shadow=dev(shadow))
    xr, itr, relr, rcr = oracle.bicg(n, bc_kind, b, np.zeros_like(b), 0.0, max_iter=20, shadow=shadow)
    assert it == itr == 20
    assert rel == pytest.approx(relr, rel=1e-8)
    assert rel_max(host(x), xr) <= 1e-10
