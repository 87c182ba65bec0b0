"""Failure detection through the C ABI, with every failure made on the host
or by a bounded wait that runs out: no test faults, traps or hangs the GPU.

Each case checks the status the library returns and that the context keeps
working afterwards (a later call on it succeeds)."""
import numpy as np
import pytest

from paper_1901_05118_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1901_05118_gb300 import binding as B  # noqa: E402

DEV = torch.device("cuda", 0)
ERR_BREAKDOWN, ERR_NOCONV, ERR_NAN, ERR_TIMEOUT, ERR_BUDGET, ERR_TOO_LARGE = -3, -4, -5, -7, -9, -11


def dev(a):
    return torch.from_numpy(np.array(a, dtype=np.float64, order="C")).to(DEV)


def still_works(ctx, n=16):
    """A small operator application on the same context succeeds."""
    lvl = B.Level(n, 1, ctx)
    y = B.stencil_apply(lvl, dev(P.random_field(n, 5)))
    torch.cuda.synchronize()
    assert bool(torch.isfinite(y).all())


@pytest.mark.parametrize("where", ["interior", "boundary_data"])
def test_nonfinite_input_reports_nan(where):
    n, nc = 32, 4
    f, g1, g2 = (a.copy() for a in P.exp_sum().data(n, 1))
    if where == "interior":
        f[n // 2, n // 3, n // 4] = np.nan      # a right-hand side value
    else:
        g2[0, n // 2, n // 2] = np.inf           # a normal derivative on a face
    ctx = B.Context()
    with pytest.raises(B.ExcmgError) as exc:
        B.excmg_solve(n, nc, 1, dev(f), dev(g1), dev(g2), 1e-10, ctx=ctx)
    assert exc.value.status == ERR_NAN
    still_works(ctx)


@pytest.mark.parametrize("n", [16, 48, 80])   # per-node cooperative, z-march cooperative, launched kernels
def test_orthogonal_shadow_breaks_down(n):
    """r*_0 with (r*_0, r_0) = 0 exactly (disjoint supports, x_0 = 0): rho_0 = 0,
    the breakdown of Alg. 2."""
    ctx = B.Context()
    lvl = B.Level(n, 2, ctx)
    b = np.zeros((n + 1,) * 3)
    shadow = np.zeros_like(b)
    b[1:n // 2, 1:-1, 1:-1] = P.random_field(n, 3)[1:n // 2, 1:-1, 1:-1]
    shadow[n // 2:-1, 1:-1, 1:-1] = P.random_field(n, 4)[n // 2:-1, 1:-1, 1:-1]
    x = torch.zeros((n + 1,) * 3, dtype=torch.float64, device=DEV)
    with pytest.raises(B.ExcmgError) as exc:
        B.bicg_solve(lvl, dev(b), x, 1e-10, 50, shadow=dev(shadow))
    assert exc.value.status == ERR_BREAKDOWN
    still_works(ctx)


@pytest.mark.parametrize("n", [16, 48, 80])
def test_iteration_cap_reports_noconv(n):
    ctx = B.Context()
    lvl = B.Level(n, 1, ctx)
    x = torch.zeros((n + 1,) * 3, dtype=torch.float64, device=DEV)
    it, rel, rc = B.bicg_solve(lvl, dev(P.random_field(n, 8)), x, 1e-14, 1)
    assert rc == ERR_NOCONV and it == 1 and rel > 1e-14


def test_budget_smaller_than_the_levels():
    n, nc = 32, 4
    f, g1, g2 = P.exp_sum().data(n, 1)
    ctx = B.Context(hbm_budget_bytes=1 << 20)   # a cap (0 would mean none), far below the level buffers
    with pytest.raises(B.ExcmgError) as exc:
        B.excmg_solve(n, nc, 1, dev(f), dev(g1), dev(g2), 1e-10, ctx=ctx)
    assert exc.value.status == ERR_BUDGET
    assert ctx.bytes <= 1 << 20


def test_batch_refuses_an_instance_larger_than_its_budget():
    n, nc = 64, 8
    f, g1, g2 = P.exp_sum().data(n, 1)
    need = B.Batch.instance_bytes(n, nc, "fp64")
    batch = B.Batch(hbm_budget_bytes=need // 2, max_instances=4)
    with pytest.raises(B.ExcmgError) as exc:
        batch.submit(n, nc, 1, dev(f), dev(g1), dev(g2), 1e-8, precision="fp64")
    assert exc.value.status == ERR_TOO_LARGE
    assert batch.bytes == 0
    batch.close()


def test_bounded_waits_give_up():
    """The grid barrier of the cooperative kernels, waiting for an arrival
    nothing makes, gives up after 20000 polls and reports EXCMG_ERR_TIMEOUT;
    the GPU stays usable."""
    assert B.selftest_wait_timeout("barrier", 20000) == ERR_TIMEOUT
    assert B.selftest_wait_timeout("barrier", 20000) == ERR_TIMEOUT   # and again: nothing left behind
    still_works(B.Context())
