"""Record the CPU oracle's own per-level Bi-CG counts for the 512^3 workload.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``).  Runs the oracle's
Alg. 1 on the benchmark workload -- u = e^(x+y+z), f = 9u, first- and
second-kind data, finest grid 512^3, coarsest 8^3, Bi-CG tolerance 1e-10 on
every level -- and writes, per kind of boundary data, the iterations, Bi-CG
calls, stagnation flags and final relative residuals of every level, with
the wall time of the whole solve and the threads it used, to
``oracle/excmg_512_counts.json``.  Nothing but ``oracle`` and the seeded
input generators is called.  The counts do not depend on the thread count
(the oracle's sums keep their order) or on the host (plain IEEE double
arithmetic without contraction).

    python -m oracle.work_units [--n 512] [--threads K]

It needs about 12 GB of host memory at 512^3 and a few minutes on a
multi-core host.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "excmg_512_counts.json")


def main(argv=None):
    import oracle
    from paper_1901_05118_gb300 import problems

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--nc", type=int, default=8)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--threads", type=int, default=len(os.sched_getaffinity(0)))
    ap.add_argument("--out", default=OUT)
    a = ap.parse_args(argv)
    used = oracle.set_threads(a.threads)
    prob = problems.exp_sum()
    record = {"workload": (f"EXCMG, u = exp(x+y+z), {a.n}^3 intervals, coarsest {a.nc}^3, Bi-CG tol {a.tol:g} on "
                           "every level"),
              "n_finest": a.n, "n_coarsest": a.nc, "tol": a.tol, "threads": used,
              "host": {"machine": platform.machine(), "cpus": os.cpu_count()}, "kinds": {}}
    for bc in (1, 2):
        f = prob.rhs(a.n)
        g1 = prob.exact(a.n)
        g2 = prob.boundary_g2(a.n, bc)
        t0 = time.perf_counter()
        _, _, st = oracle.excmg(a.n, a.nc, bc, f, g1, g2, a.tol)
        wall = time.perf_counter() - t0
        del f, g1, g2
        levels = [{"n": a.nc << l, "iters": int(st[l, 0]), "relres": float(st[l, 1]), "calls": int(st[l, 2]),
                   "stagnated": bool(st[l, 3])} for l in range(st.shape[0])]
        wu = sum(lv["iters"] * ((lv["n"] - 1) / (a.n - 1)) ** 3 for lv in levels)
        record["kinds"][str(bc)] = {"levels": levels, "work_units": wu, "solve_s": wall}
        print(json.dumps({"bc": bc, "solve_s": round(wall, 1), "iters": [lv["iters"] for lv in levels]}),
              flush=True)
    with open(a.out, "w") as fh:
        json.dump(record, fh, indent=1)
    print(a.out)


if __name__ == "__main__":
    main()
