"""Host logic of the solve server, on CPU with a fake engine."""
import numpy as np
import pytest

from paper_1901_05118_gb300 import problems as P
from paper_1901_05118_gb300 import serving as S


def test_size_grid_and_rounding():
    g = S.size_grid(32, 256)
    assert g[0] == 32 and g[-1] == 256
    assert all(any(v == c << k for c in S.SIZE_BASES for k in range(3, 10)) for v in g)
    assert S.round_size(33) == 32 and S.round_size(250) == 256 and S.round_size(45) == 48
    for n in g:
        nc = S.coarsest_for(n)
        assert 4 <= nc <= 8 and n % nc == 0
        ratio = n // nc
        assert ratio >= 4 and ratio & (ratio - 1) == 0     # two direct grids + >= 1 Bi-CG grid


def test_requests_are_seeded_poisson():
    a = S.make_requests(2000, rate=50.0, seed=1)
    b = S.make_requests(2000, rate=50.0, seed=1)
    assert [(r.t_arrival, r.n, r.bc) for r in a] == [(r.t_arrival, r.n, r.bc) for r in b]
    gaps = np.diff([0.0] + [r.t_arrival for r in a])
    assert abs(gaps.mean() - 1 / 50.0) < 0.1 / 50.0
    assert {r.bc for r in a} == {1, 2}
    sizes = np.array([r.n for r in a])
    assert sizes.min() >= 32 and sizes.max() <= 256


class FakeEngine:
    """Admits up to `slots` solves; each finishes after `work` steps."""

    def __init__(self, slots, work):
        self.slots, self.work, self.live, self.done, self.next = slots, work, {}, set(), 0

    def submit(self, n, nc, bc, f, g1, g2, tol, out, **kw):
        if len(self.live) >= self.slots:
            return None
        i = self.next
        self.next += 1
        self.live[i] = self.work
        return i, out

    def step(self):
        for i in list(self.live):
            self.live[i] -= 1
            if self.live[i] == 0:
                del self.live[i]
                self.done.add(i)
        return len(self.live)

    def query(self, i):
        return {"done": i in self.done, "status": 0}


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001
        return self.t


class FakePool:
    def get(self, n, bc, ps):
        return None, None, None


def test_serve_admits_as_slots_free_and_reports_latency():
    reqs = S.make_requests(50, rate=2000.0, seed=3)   # all arrive almost at once
    clock = FakeClock()
    eng = FakeEngine(slots=4, work=3)
    recs, summ = S.serve(eng, reqs, FakePool(), 1e-8, clock=clock, sleep=lambda s: None)
    assert summ["requests"] == 50 and summ["failed"] == 0
    assert max(len(eng.live), 0) == 0
    assert summ["p99_s"] >= summ["p50_s"] > 0
    assert sorted(r["rid"] for r in recs) == list(range(50))


class PickyEngine(FakeEngine):
    """Never admits grids of `never` intervals: returns None for them (as a
    full engine does), or raises like excmg_batch_submit's
    EXCMG_ERR_TOO_LARGE when `raise_status` is set."""

    def __init__(self, slots, work, never, raise_status=None):
        super().__init__(slots, work)
        self.never, self.raise_status = never, raise_status

    def submit(self, n, nc, bc, f, g1, g2, tol, out, **kw):
        if n == self.never:
            if self.raise_status is not None:
                err = RuntimeError("instance larger than the whole budget")
                err.status = self.raise_status
                raise err
            return None
        return super().submit(n, nc, bc, f, g1, g2, tol, out, **kw)


@pytest.mark.parametrize("raise_status", [None, -11])
def test_serve_rejects_a_request_that_can_never_be_admitted(raise_status):
    # the loop must end (it used to spin forever with nothing live), serve
    # every other request and record the refused ones as rejected
    reqs = S.make_requests(60, rate=2000.0, seed=3)
    big = max(r.n for r in reqs)
    n_big = sum(1 for r in reqs if r.n == big)
    assert 0 < n_big < len(reqs)
    eng = PickyEngine(slots=4, work=2, never=big, raise_status=raise_status)
    recs, summ = S.serve(eng, reqs, FakePool(), 1e-8, clock=FakeClock(), sleep=lambda s: None)
    assert summ["requests"] == 60 and summ["rejected"] == n_big
    rejected = [r for r in recs if r.get("rejected")]
    assert {r["n"] for r in rejected} == {big}
    assert all(r["status"] == (raise_status if raise_status is not None else S.REJECTED) for r in rejected)
    assert all(r["status"] == 0 for r in recs if not r.get("rejected"))


def test_random_sines_torch_matches_numpy():
    torch = pytest.importorskip("torch")
    for bc in (1, 2):
        f, g1, g2 = P.random_sines(1003).data(12, bc)
        tf, tg1, tg2 = P.random_sines_torch(1003, 12, bc, "cpu")
        np.testing.assert_allclose(tf.numpy(), f, rtol=1e-12, atol=1e-9)
        np.testing.assert_allclose(tg1.numpy(), g1, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(tg2.numpy(), g2, rtol=1e-12, atol=1e-12)
