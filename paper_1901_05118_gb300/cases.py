"""Small, fixed GPU cases for profiling single kernels of the library.

    python -m paper_1901_05118_gb300.cases stencil --n 256 --variant exact --reps 3
    python -m paper_1901_05118_gb300.cases bicg --n 256 --iters 4 [--schedule fused]
    python -m paper_1901_05118_gb300.cases solve --n 64 --nc 8
    python -m paper_1901_05118_gb300.cases issue-rates

Each case allocates a few hundred MB at most (inputs still larger than L2 at
n = 256) and runs a handful of launches, so a profiler capture ends quickly.
"""
from __future__ import annotations

import argparse
import os
import subprocess
import sys


def issue_rates():
    """Compile and run issue_rates.cu (FP64 / FP32 / integer issue rates)."""
    here = os.path.dirname(os.path.abspath(__file__))
    exe = os.path.join(here, "_build", "issue_rates")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                           os.path.join(here, "issue_rates.cu")])
    sys.exit(subprocess.call([exe]))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["stencil", "bicg", "solve", "issue-rates"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--nc", type=int, default=8)
    ap.add_argument("--bc", type=int, default=1)
    ap.add_argument("--variant", choices=["exact", "fp64"], default="exact")
    ap.add_argument("--schedule", choices=["separate", "fused"], default="separate")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--iters", type=int, default=4)
    a = ap.parse_args(argv)
    if a.case == "issue-rates":
        issue_rates()
    import torch

    from . import binding as B
    from . import problems

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ctx = B.Context(dev)
    ctx.set_stencil(a.variant)
    ctx.set_schedule(a.schedule)
    n = a.n
    gen = torch.Generator(device=dev)
    gen.manual_seed(0)
    if a.case == "stencil":
        u = torch.rand((n + 1,) * 3, dtype=torch.float64, device=dev, generator=gen)
        y = torch.empty_like(u)
        lvl = B.Level(n, a.bc, ctx)
        for _ in range(a.reps):
            B.stencil_apply(lvl, u, y)
    elif a.case == "bicg":
        b = torch.rand((n + 1,) * 3, dtype=torch.float64, device=dev, generator=gen)
        x = torch.zeros_like(b)
        lvl = B.Level(n, a.bc, ctx)
        B.bicg_solve(lvl, b, x, 0.0, a.iters)
    else:
        prob = problems.exp_sum()
        f, g1, g2 = (torch.from_numpy(v).to(dev) for v in prob.data(n, a.bc))
        B.excmg_solve(n, a.nc, a.bc, f, g1, g2, 1e-10, ctx=ctx)
    torch.cuda.synchronize()
    print("ok")


if __name__ == "__main__":
    main()
