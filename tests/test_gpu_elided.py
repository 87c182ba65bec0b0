"""Shadow-elided Bi-CG (a labelled variant, not Alg. 2 as printed): with
r*_0 = r_0 and the exact integer operator the shadow sequence of Alg. 2 is
the primal one bit for bit, so the elided mode, which stores neither r*, p*
nor A^T p*, must give the same bits as the full mode on every path (per-node
and z-march cooperative kernels, launched kernels above 128^3) and in whole
solves."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1901_05118_gb300 import binding as B
    from paper_1901_05118_gb300 import problems as P

DEV = torch.device("cuda", 0)


def ctx(mode, schedule="separate"):
    c = B.Context()
    c.set_shadow_mode(mode)
    c.set_schedule(schedule)
    return c


@pytest.mark.parametrize("schedule", ["separate", "fused"])
@pytest.mark.parametrize("n,bc_kind,tol,max_iter", [(24, 1, 1e-11, 5000), (56, 2, 0.0, 300),
                                                     (136, 1, 0.0, 60), (133, 2, 0.0, 45)])
def test_elided_bicg_is_bit_identical(n, bc_kind, tol, max_iter, schedule):
    b = torch.from_numpy(P.random_field(n, 91)).to(DEV)
    x0 = torch.from_numpy(P.random_field(n, 92) * 0.1).to(DEV)
    out = {}
    for mode in ("full", "elided"):
        lvl = B.Level(n, bc_kind, ctx(mode, schedule))
        x = x0.clone()
        it, rel, rc = B.bicg_solve(lvl, b, x, tol, max_iter)
        torch.cuda.synchronize()
        out[mode] = (it, rel, rc, x)
    (itf, relf, rcf, xf), (ite, rele, rce, xe) = out["full"], out["elided"]
    assert (itf, relf, rcf) == (ite, rele, rce)
    if tol > 0:
        assert rcf == 0
    assert torch.equal(xf, xe)


@pytest.mark.parametrize("n,bc_kind", [(128, 1), (256, 2)])
def test_elided_solve_is_bit_identical(n, bc_kind):
    prob = P.exp_sum()
    f, g1, g2 = (torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in prob.data(n, bc_kind))
    res = {}
    for mode in ("full", "elided"):
        res[mode] = B.excmg_solve(n, 8, bc_kind, f, g1, g2, 1e-10, ctx=ctx(mode), return_stats=True)
    torch.cuda.synchronize()
    (uf, sf), (ue, se) = res["full"], res["elided"]
    assert [s["iters"] for s in sf] == [s["iters"] for s in se]
    assert torch.equal(uf, ue)


@pytest.mark.parametrize("schedule", ["separate", "fused"])
@pytest.mark.parametrize("mode", ["full", "elided"])
def test_graph_replay_is_bit_identical(schedule, mode):
    """Batches of launched Bi-CG iterations replayed from CUDA graphs give the
    same bits as the same launches made directly (80 iterations: the first
    batch of 16 launched directly, the next four replayed from the graph)."""
    n = 136
    b = torch.from_numpy(P.random_field(n, 93)).to(DEV)
    x0 = torch.from_numpy(P.random_field(n, 94) * 0.1).to(DEV)
    out = {}
    for graphs in (False, True):
        c = ctx(mode, schedule)
        c.set_graphs(graphs)
        lvl = B.Level(n, 1, c)
        x = x0.clone()
        it, rel, rc = B.bicg_solve(lvl, b, x, 0.0, 80)
        assert it == 80
        out[graphs] = (x, rel)
    assert out[True][1] == out[False][1]
    assert torch.equal(out[True][0], out[False][0])
