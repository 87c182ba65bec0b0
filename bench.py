"""Benchmark of the EXCMG solve on GB300.

Workload (default): the plain FP64 EXCMG solve on the 512^3-interval grid
(511^3 = 133,432,831 unknowns), coarsest grid 8^3 (7 nested levels, 8^3 and
16^3 solved directly), manufactured u = exp(x+y+z), f = 9u, Bi-CG relative
residual tolerance 1e-10 on every level.  One step = two solves: first-kind
and second-kind boundary data.  Inputs are synthetic closed forms; every
input array is larger than the 129 MB L2, so no flush is needed.

Printed: one JSON line (rank 0).  ``value`` = seconds per solve with the
inputs resident in HBM; ``e2e`` = the same through the C ABI with pinned host
buffers, host->device copies of f, g1, g2 and the device->host copy of the
solution inside the timed region.  ``roofline`` is the operator kernel on the
finest grid, timed live (CUDA events around each of its launches inside
Bi-CG).  ``cpu_baseline`` times the CPU oracle on a bounded sample.

Multi-GPU: the solve does not shard here; ``--gpus N`` under torchrun runs N
independent replicas (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "EXCMG solve s @512³ FP64 vs FP32+refine; stencil HBM GB/s % peak; p99 latency"
# The CPU oracle's own per-level Bi-CG counts on the default workload, written
# by `python -m oracle.work_units` (a run of the oracle's whole 512^3 solve).
# DRAM bytes (read + write) per launch measured by ncu on 255^3 unknowns
# (python bench.py --case bicg --n 256 --iters 4 [--schedule separate]; the
# summaries under profiles/ give the full capture commands)
TRAFFIC_255 = {"stencil_pair_kernel": 288.93e6 + 220.17e6, "stencil_pair_dir_kernel": 582.57e6 + 489.67e6}
ORACLE_COUNTS = os.path.join(ROOT, "oracle", "excmg_512_counts.json")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--nc", type=int, default=8)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--stencil", choices=["exact", "fp64"], default="exact")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the FP32-inner / FP64-refinement leg")
    ap.add_argument("--mixed-steps", type=int, default=2)
    ap.add_argument("--mixed-tols", default="",
                    help="comma-separated FP64 residual tolerances for a sweep of the precision leg")
    ap.add_argument("--mixed-inner", default="",
                    help="comma-separated inner_tol:cap pairs of the FP32 correction solves to sweep at --tol")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-instance batched leg")
    ap.add_argument("--batch-mixed", action="store_true",
                    help="batched leg: also the mixed-precision form (about 90 s more)")
    ap.add_argument("--no-serve", action="store_true", help="skip the request-stream leg")
    ap.add_argument("--serve-requests", type=int, default=120)
    ap.add_argument("--serve-max-s", type=float, default=90.0,
                    help="request stream: arrivals spread over at most this many seconds (0: 0.8x capacity only)")
    ap.add_argument("--no-elided", action="store_true", help="skip the shadow-elided variant leg")
    ap.add_argument("--schedule", choices=["separate", "fused"], default="fused",
                    help="Bi-CG operator schedule of the timed solves on grids above 64^3")
    ap.add_argument("--serve-precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--oracle-report", action="store_true",
                    help="time the CPU oracle on the small workload and one 512^3 operator application, then exit")
    ap.add_argument("--case", choices=["stencil", "bicg", "solve", "batch"],
                    help="run one small fixed case for a profiler capture (sizes from --n / --nc) and exit")
    ap.add_argument("--bc", type=int, default=1, help="--case: kind of boundary data")
    ap.add_argument("--iters", type=int, default=4, help="--case bicg: Bi-CG iterations")
    ap.add_argument("--reps", type=int, default=3, help="--case stencil: operator applications")
    ap.add_argument("--shadow", choices=["full", "elided"], default="full", help="--case bicg: shadow mode")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64", help="--case solve: precision")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest of every rank's x (a timing): the job takes as long as its
    slowest replica."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def seconds_per_solve(ms_per_step_max: float, solves_per_step: int, world: int) -> float:
    """Whole-job seconds per solve: every replica runs solves_per_step solves
    per step, so the job finishes world * solves_per_step solves per step."""
    return ms_per_step_max / 1e3 / (solves_per_step * world)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- CPU oracle
def host_threads() -> int:
    """Host CPUs this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


class OracleSampler:
    """The CPU oracle (oracle/, plain C, FP64) timed on bounded samples of the
    workload and scaled to one whole solve with the oracle's own counts.

    A whole oracle solve of the 512^3 workload takes minutes, so one timed
    sample is: on every Bi-CG level N = 4 nc .. min(n, 256), one Bi-CG
    iteration of the oracle (the time of a k-iteration call minus that of a
    0-iteration call on the level's own right-hand side, over at least
    0.2 s), times the oracle's iterations on that level; plus each level's
    fixed work of Alg. 1 (assembly of f_h, EXP_finite, the true residuals of
    the WHILE loop), timed once on min(N, 128).  Levels above the timed size
    take the timed size's seconds scaled by their unknowns (the oracle's
    loops are linear in them).  The counts are the oracle's own from a whole
    run (oracle/excmg_512_counts.json); without that file for this workload
    there is no value."""

    ITER_MAX_N = 256
    FIXED_MAX_N = 128

    def __init__(self, n: int, nc: int, threads: int):
        import oracle
        from paper_1901_05118_gb300 import problems

        self.oracle, self.n, self.nc = oracle, n, nc
        self.threads = oracle.set_threads(threads)
        self.prob = problems.exp_sum()
        self.counts = None
        try:
            rec = json.load(open(ORACLE_COUNTS))
            if rec["n_finest"] == n and rec["n_coarsest"] == nc:
                self.counts = {int(k): v for k, v in rec["kinds"].items()}
        except (OSError, ValueError, KeyError):
            pass
        self.levels = []
        N = 4 * nc
        while N <= n:
            self.levels.append(N)
            N *= 2
        self.data = {}
        self.fixed = {}

    def _level(self, N, bc):
        key = (N, bc)
        if key not in self.data:
            f, g1, g2 = self.prob.data(N, bc)
            self.data[key] = (self.oracle.assemble_rhs(N, bc, f, g1, g2), np.ascontiguousarray(g1))
        return self.data[key]

    @staticmethod
    def _scale(N, M):
        """Unknowns of level N over those of level M."""
        return ((N - 1) / (M - 1)) ** 3

    def iteration_s(self, N, bc):
        """Seconds per oracle Bi-CG iteration on level N: (time of a k-iteration
        call - time of a 0-iteration call) / k, k grown until the difference
        is at least 0.2 s (at most 256 iterations); above ITER_MAX_N, that
        size's time scaled by the unknowns."""
        if N > self.ITER_MAX_N:
            return self.iteration_s(self.ITER_MAX_N, bc) * self._scale(N, self.ITER_MAX_N)
        key = ("it", N, bc)
        if key in self.fixed:
            return self.fixed[key]
        fh, g1 = self._level(N, bc)
        t0 = time.perf_counter()
        self.oracle.bicg(N, bc, fh, g1, 0.0, max_iter=0)
        setup = time.perf_counter() - t0
        k = 1
        while True:
            t0 = time.perf_counter()
            self.oracle.bicg(N, bc, fh, g1, 0.0, max_iter=k)
            run = time.perf_counter() - t0 - setup
            if run >= 0.2 or k >= 256:
                self.fixed[key] = max(run / k, 1e-9)
                return self.fixed[key]
            k *= 4

    def fixed_s(self, N, bc, calls):
        """Alg. 1's work on level N besides the Bi-CG iterations (timed once,
        on min(N, FIXED_MAX_N) and scaled by the unknowns)."""
        if N > self.FIXED_MAX_N:
            M = self.FIXED_MAX_N
            setup, resid = self._fixed_parts(M, bc)
            return (setup + (calls + 1) * resid) * self._scale(N, M)
        setup, resid = self._fixed_parts(N, bc)
        return setup + (calls + 1) * resid

    def _fixed_parts(self, N, bc):
        key = (N, bc)
        if key not in self.fixed:
            o = self.oracle
            f, g1, g2 = self.prob.data(N, bc)
            u1 = np.ascontiguousarray(self.prob.exact(N // 2))
            u0 = np.ascontiguousarray(self.prob.exact(N // 4))
            t0 = time.perf_counter()
            fh = o.assemble_rhs(N, bc, f, g1, g2)
            w = o.exp_finite(N, u1, u0)
            t1 = time.perf_counter()
            o.residual_norm(N, bc, fh, w)
            t2 = time.perf_counter()
            self.fixed[key] = (t1 - t0, t2 - t1)
        return self.fixed[key]

    def solve_s(self, bc):
        """Seconds of one oracle solve of the workload with kind bc, and the
        per-level breakdown; (None, None) without the oracle's counts."""
        if self.counts is None:
            return None, None
        # iteration times are taken afresh by every call (the fixed work,
        # timed once, is kept)
        for key in [k for k in self.fixed if k[0] == "it"]:
            del self.fixed[key]
        lv = {L["n"]: L for L in self.counts[bc]["levels"]}
        total, parts = 0.0, []
        for N in self.levels:
            t_it = self.iteration_s(N, bc)
            t_fx = self.fixed_s(N, bc, lv[N]["calls"])
            total += lv[N]["iters"] * t_it + t_fx
            parts.append({"n": N, "iters": lv[N]["iters"], "iteration_s": round(t_it, 4), "fixed_s": round(t_fx, 3)})
        return total, parts

    def describe(self):
        return (f"oracle (plain C, FP64) on {self.threads} host threads: per Bi-CG level N = "
                f"{self.levels[0]}..{self.levels[-1]}, timed Bi-CG iterations (at least 0.2 s of them; levels above "
                f"{self.ITER_MAX_N}^3 scaled by their unknowns from {self.ITER_MAX_N}^3) x the oracle's own iterations "
                f"on that level (oracle/excmg_512_counts.json, from a whole oracle solve), plus each level's "
                f"assembly, EXP_finite and true residuals timed once on min(N, {self.FIXED_MAX_N})^3 and scaled by the "
                f"unknowns; the direct solves of the two coarsest grids are not counted")


def run_reference(args):
    """The reference arm: the CPU oracle, timed as OracleSampler says, on the
    same workload and metric.  Each step samples one kind of boundary data
    (alternating); `value` is the mean over the timed steps of the oracle's
    seconds per solve, `ms_per_step` the wall time a timed step took."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    sampler = OracleSampler(args.n, args.nc, host_threads())
    if sampler.counts is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no oracle counts for {args.n}^3 / {args.nc}^3 "
                          "(run python -m oracle.work_units)"}), flush=True)
        return
    values, walls, parts = [], [], {}
    for s_ in range(args.warmup + args.steps):
        bc = 1 + s_ % 2
        t0 = time.perf_counter()
        v, part = sampler.solve_s(bc)
        wall = time.perf_counter() - t0
        if s_ >= args.warmup:
            values.append(v)
            walls.append(wall)
            parts[str(bc)] = part
    value = statistics.mean(values)
    info = {"kind": "oracle", "cores": sampler.threads, "host_cpus": os.cpu_count(), "value": value, "unit": "s",
            "sample": sampler.describe(), "levels": parts,
            "oracle_whole_solve_s_recorded": {k: v["solve_s"] for k, v in sampler.counts.items()}}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(walls) * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args), "cpu_baseline": info,
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(args):
    """The oracle on the host cores, one sample of each kind of boundary data
    (OracleSampler), as seconds per solve."""
    sampler = OracleSampler(args.n, args.nc, host_threads())
    if sampler.counts is None:
        return {"kind": "oracle", "value": None, "unavailable": "no oracle counts for this workload"}
    t0 = time.perf_counter()
    per_kind = {bc: sampler.solve_s(bc) for bc in (1, 2)}
    return {"kind": "oracle", "value": statistics.mean(v for v, _ in per_kind.values()), "unit": "s",
            "cores": sampler.threads, "host_cpus": os.cpu_count(), "sample": sampler.describe(),
            "sample_wall_s": time.perf_counter() - t0,
            "levels": {str(bc): part for bc, (_, part) in per_kind.items()},
            "oracle_whole_solve_s_recorded": {k: v["solve_s"] for k, v in sampler.counts.items()}}


def config(args):
    return {"workload": (f"EXCMG FP64, {args.n}^3 intervals ({args.n - 1}^3 unknowns), coarsest {args.nc}^3, "
                         f"u=exp(x+y+z), first- and second-kind data, Bi-CG tol {args.tol:g} per level"),
            "n_finest": args.n, "n_coarsest": args.nc, "levels": int(np.log2(args.n // args.nc)) + 1,
            "solves_per_step": 2, "tol": args.tol, "stencil": args.stencil, "schedule": args.schedule,
            "l2_flush": "inputs larger than L2 (each node array 1.08 GB)", "parallelism": "replicas"}


# --------------------------------------------------------------- GPU arm
def _cpulist(text):
    cpus = set()
    for part in text.strip().split(","):
        if not part:
            continue
        lo, _, hi = part.partition("-")
        cpus.update(range(int(lo), int(hi or lo) + 1))
    return cpus


def bind_host_to_gpu_numa(dev_index):
    """Run this process on the CPUs of the GPU's NUMA node, so that the pinned
    host buffers of the end-to-end leg (placed by first touch) sit next to the
    GPU's host link, as `numactl --cpunodebind` would.  Returns what was done,
    or None where the system does not say which node that is."""
    import torch

    try:
        p = torch.cuda.get_device_properties(dev_index)
        bdf = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        node = int(open(f"/sys/bus/pci/devices/{bdf}/numa_node").read())
        if node < 0:
            return None
        cpus = _cpulist(open(f"/sys/devices/system/node/node{node}/cpulist").read())
        cpus &= os.sched_getaffinity(0)
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return {"numa_node": node, "cpus": len(cpus)}
    except (OSError, ValueError, AttributeError):
        return None


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    from paper_1901_05118_gb300 import binding as B, problems

    host_binding = bind_host_to_gpu_numa(local)
    n, nc = args.n, args.nc
    prob = problems.exp_sum()
    bcs = (1, 2)
    host = {}
    f = prob.rhs(n)
    g1 = prob.exact(n)
    host["f"] = torch.from_numpy(f).pin_memory()
    host["g1"] = torch.from_numpy(g1).pin_memory()
    for bc in bcs:
        host[f"g2_{bc}"] = torch.from_numpy(prob.boundary_g2(n, bc)).pin_memory()
    del f, g1
    d = {k: v.to(dev, non_blocking=False) for k, v in host.items()}
    u_out = torch.empty((n + 1,) * 3, dtype=torch.float64, device=dev)
    u_host = torch.empty((n + 1,) * 3, dtype=torch.float64).pin_memory()
    ctx = B.Context(dev)
    ctx.set_stencil(args.stencil)
    ctx.set_schedule(args.schedule)
    stream = torch.cuda.current_stream(dev)

    def solve(bc, stats=False):
        return B.excmg_solve(n, nc, bc, d["f"], d["g1"], d[f"g2_{bc}"], args.tol, u_out, ctx=ctx,
                             return_stats=stats)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # warm-up (also builds the DSOLVE inverses held by the context)
    for _ in range(args.warmup):
        for bc in bcs:
            solve(bc)
    stats = {bc: solve(bc, stats=True)[1] for bc in bcs}

    # ---- device-resident timing
    ctx.profile(True)
    launches0 = B.launch_count()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            for bc in bcs:
                solve(bc)
        e1.record(stream)
        barrier()
    ms_total = e0.elapsed_time(e1)
    launches = B.launch_count() - launches0
    st_ms, st_cnt, st_bytes = ctx.profile_read(n)
    ctx.profile(False)
    ms_step = max_over_ranks(ms_total / args.steps, world, dev)
    value = seconds_per_solve(ms_step, len(bcs), world)

    # ---- end to end through the C ABI, host buffers.  Every solve copies its
    # inputs (f, g1, g2) from pinned host memory and reads u back; the copies
    # run on their own streams into two device buffer sets, so the inputs of
    # solve i+1 and the result of solve i-1 move while solve i computes (the
    # solve call itself returns when its work is done).
    e2e = None
    if not args.no_e2e:
        h2d = sum(host[k].numel() * 8 for k in ("f", "g1")) + host["g2_1"].numel() * 8
        d2h = u_host.numel() * 8
        sets = [d, {k: torch.empty_like(v) for k, v in d.items()}]
        outs = [u_out, torch.empty_like(u_out)]
        u_hosts = [u_host, torch.empty_like(u_host).pin_memory()]
        s_h2d, s_d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        order = [bc for _ in range(args.steps) for bc in bcs]
        ns = len(order)

        def e2e_solve(bc, k):
            return B.excmg_solve(n, nc, bc, sets[k]["f"], sets[k]["g1"], sets[k][f"g2_{bc}"], args.tol, outs[k],
                                 ctx=ctx)

        barrier()
        ev = lambda: torch.cuda.Event(enable_timing=True)
        h2d_start = [ev() for _ in range(ns)]
        d2h_start = [ev() for _ in range(ns)]
        inputs_ready = [ev() for _ in range(ns)]
        result_read = [ev() for _ in range(ns)]
        solve_start = [ev() for _ in range(ns)]
        solve_done = [ev() for _ in range(ns)]
        e2, e3 = ev(), ev()
        e2.record(stream)

        def sliced_copy(dst, src):
            # 64 MB slices: the solve's own small state reads share the copy
            # engines and slip in between slices instead of waiting a whole
            # gigabyte copy out
            dv, sv = dst.view(-1), src.view(-1)
            step = 1 << 23
            for a in range(0, dv.numel(), step):
                dv[a:a + step].copy_(sv[a:a + step], non_blocking=True)

        def prefetch(i):
            k = i % 2
            with torch.cuda.stream(s_h2d):
                s_h2d.wait_stream(stream)          # set k's previous solve has finished
                h2d_start[i].record(s_h2d)
                for key in ("f", "g1", f"g2_{order[i]}"):
                    sliced_copy(sets[k][key], host[key])
                inputs_ready[i].record(s_h2d)

        prefetch(0)
        for i, bc in enumerate(order):
            k = i % 2
            stream.wait_event(inputs_ready[i])
            if i >= 2:
                stream.wait_event(result_read[i - 2])   # outs[k] has been read back
            solve_start[i].record(stream)
            if i + 1 < ns:
                prefetch(i + 1)
            e2e_solve(bc, k)
            solve_done[i].record(stream)
            with torch.cuda.stream(s_d2h):
                s_d2h.wait_event(solve_done[i])
                d2h_start[i].record(s_d2h)
                sliced_copy(u_hosts[k], outs[k])
                result_read[i].record(s_d2h)
        stream.wait_event(result_read[ns - 1])
        e3.record(stream)
        barrier()
        ms_e2e = max_over_ranks(e2.elapsed_time(e3) / args.steps, world, dev)
        e2e = {"value": seconds_per_solve(ms_e2e, len(bcs), world), "unit": "s",
               "h2d_bytes_per_step": h2d * len(bcs), "d2h_bytes_per_step": d2h * len(bcs),
               "pipeline": "inputs of the next solve and the result of the previous one copied on two "
                           "streams into two device buffer sets while a solve runs",
               "per_solve_ms": {"h2d": statistics.mean(h2d_start[i].elapsed_time(inputs_ready[i]) for i in range(ns)),
                                "solve": statistics.mean(solve_start[i].elapsed_time(solve_done[i]) for i in range(ns)),
                                "d2h": statistics.mean(d2h_start[i].elapsed_time(result_read[i]) for i in range(ns))},
               "host_binding": host_binding}

    # ---- roofline of the operator kernel on the finest grid
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    # algorithmic bytes per launch as the library counts them: 8 B per unknown
    # for every field read or written (the fused launch that also forms the
    # directions: r, r*, p_old, p*_old in; p, p*, A p, A^T p* out)
    avg_ms = st_ms / st_cnt if st_cnt else float("nan")
    bytes_per_launch = st_bytes / st_cnt if st_cnt else None
    achieved = st_bytes / (st_ms * 1e-3) / 1e9 if st_cnt else None
    per_unknown = bytes_per_launch / (n - 1) ** 3 if bytes_per_launch else 0.0
    if args.stencil != "exact":
        kernel = f"stencil_f64_kernel: A p or A^T p* on the {n}^3 grid"
    elif per_unknown > 48.0:
        kernel = f"stencil_pair_dir_kernel (fused schedule): p, p* formed, A p, A^T p*, sigma on the {n}^3 grid"
    else:
        kernel = f"stencil_pair_kernel: A p, A^T p*, sigma (operator pair) on the {n}^3 grid"
    # DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the kernel
    # from one ncu capture on 255^3 unknowns, scaled to this launch by the
    # unknowns it processes (traffic grows in proportion); None for a kernel
    # without a capture of its current code
    traffic = None
    captured = TRAFFIC_255.get(kernel.split(" ")[0]) if args.stencil == "exact" else None
    if captured:
        traffic = captured / 255 ** 3 * (n - 1) ** 3
    roofline = {"kernel": kernel, "bound": "hbm",
                "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": (achieved / hbm_peak) if achieved else None, "traffic": traffic,
                "launches": st_cnt, "avg_ms": avg_ms, "bytes_per_launch": bytes_per_launch,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}

    elided = None
    if not args.no_elided:
        elided = elided_leg(args, B, lambda bc: solve(bc), d, dev, stream, barrier, world)

    mixed = None
    if not args.no_mixed:
        mixed = precision_leg(args, B, problems, ctx, dev, stream, barrier, world)

    batched = None
    if not args.no_batch:
        batched = batched_leg(args, B, problems, ctx, dev)
    served = None
    if not args.no_serve:
        served = serving_leg(args, B, ctx, dev)

    wu = {bc: sum(s["iters"] * (s["n"] / n) ** 3 for s in stats[bc] if s["iters"]) for bc in bcs}
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(args),
            "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "clocks": clk.summary(),
            "levels": {str(bc): [{"n": s["n"], "iters": s["iters"], "ms": round(s["ms"], 3),
                                  "relres": s["relres"]} for s in stats[bc]] for bc in bcs},
            "work_units": {str(bc): round(w, 2) for bc, w in wu.items()}, "shadow_elided_leg": elided,
            "precision_leg": mixed, "batched_leg": batched, "serving_leg": served}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def elided_leg(args, B, solve_full, d, dev, stream, barrier, world):
    """The headline workload with the shadow-elided Bi-CG, a labelled
    variant that is not the paper's Alg. 2 as printed: r*, p* and A^T p*
    (bit for bit r, p and A p here) are not stored.  Reports seconds per solve
    and whether every result equals the full mode's bit for bit."""
    import torch

    n, nc, bcs = args.n, args.nc, (1, 2)
    ctx_e = B.Context(dev)
    ctx_e.set_stencil(args.stencil)
    ctx_e.set_shadow_mode("elided")
    u_e = torch.empty((n + 1,) * 3, dtype=torch.float64, device=dev)
    same = True
    for bc in bcs:
        u_full = solve_full(bc).clone()
        B.excmg_solve(n, nc, bc, d["f"], d["g1"], d[f"g2_{bc}"], args.tol, u_e, ctx=ctx_e)   # warm-up
        same = same and bool(torch.equal(u_full, u_e))
        del u_full
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        for bc in bcs:
            B.excmg_solve(n, nc, bc, d["f"], d["g1"], d[f"g2_{bc}"], args.tol, u_e, ctx=ctx_e)
    e1.record(stream)
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    return {"label": "non-paper variant: shadow sequence of Alg. 2 not stored (equal to the primal one bit for bit)",
            "value": seconds_per_solve(ms, len(bcs), world), "unit": "s", "bitwise_equal_to_full": same}


def precision_leg(args, B, problems, ctx, dev, stream, barrier, world):
    """FP64 versus FP32-inner / FP64-refinement on the same 512^3 problem:
    u = sin(2 pi x) sin(2 pi y) sin(2 pi z) + x^2 y^2 z^2, both kinds of data,
    refinement to the same FP64 relative residual tol on every level.
    Reports seconds per solve of each, the max error of each against the
    exact solution (the discretisation error) and their distance from each
    other; with --mixed-tols, the same for every tolerance of the sweep."""
    import torch

    n, nc = args.n, args.nc
    prob = problems.sin2pi_plus_poly()
    f = torch.from_numpy(prob.rhs(n)).to(dev)
    ue = torch.from_numpy(prob.exact(n)).to(dev)
    g2s = {bc: torch.from_numpy(prob.boundary_g2(n, bc)).to(dev) for bc in (1, 2)}

    def one(tol, inner=None):
        res = {}
        for prec in (("mixed",) if inner else ("fp64", "mixed")):
            kw = {}
            if inner and prec == "mixed":
                kw = {"inner_tol": inner[0], "max_iter": inner[1]}
            times, errs, outs = [], [], {}
            for bc in (1, 2):
                u = torch.empty_like(f)
                run = lambda: B.excmg_solve(n, nc, bc, f, ue, g2s[bc], tol, u, ctx=ctx, precision=prec,
                                            return_stats=True, max_total=20000, **kw)
                _, st = run()   # warm-up
                barrier()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.mixed_steps):
                    _, st = run()
                e1.record(stream)
                barrier()
                times.append(e0.elapsed_time(e1) / args.mixed_steps / 1e3)
                errs.append(float((u - ue).abs().max()))
                outs[bc] = u.clone()
                res.setdefault("levels_" + prec, {})[str(bc)] = [(s["n"], s["iters"], s["calls"]) for s in st]
            res[prec] = (sum(times) / len(times), errs, outs)
        if inner:
            tmx, emx, _ = res["mixed"]
            return {"tol": tol, "inner_tol": inner[0], "inner_cap": inner[1],
                    "mixed_s": max_over_ranks(tmx, world, dev), "err_vs_exact_linf_mixed": emx,
                    "levels_mixed": res["levels_mixed"]}
        t64, e64, o64 = res["fp64"]
        tmx, emx, omx = res["mixed"]
        return {"tol": tol, "fp64_s": max_over_ranks(t64, world, dev), "mixed_s": max_over_ranks(tmx, world, dev),
                "speedup": t64 / tmx, "err_vs_exact_linf_fp64": e64, "err_vs_exact_linf_mixed": emx,
                "mixed_minus_fp64_linf": [float((omx[bc] - o64[bc]).abs().max()) for bc in (1, 2)],
                "levels_fp64": res["levels_fp64"], "levels_mixed": res["levels_mixed"]}

    out = {"workload": (f"{n}^3, coarsest {nc}^3, u = sin(2 pi x)sin(2 pi y)sin(2 pi z) + x^2y^2z^2, "
                        f"first- and second-kind data, FP64 residual tol {args.tol:g} per level"),
           "inner_tol": B.MIXED_INNER_TOL, "inner_cap": B.MIXED_INNER_CAP}
    out.update(one(args.tol))
    if args.mixed_tols:
        out["sweep"] = [one(float(t)) for t in args.mixed_tols.split(",") if t.strip()]
    if args.mixed_inner:
        pairs = [p.split(":") for p in args.mixed_inner.split(",") if p.strip()]
        out["inner_sweep"] = [one(args.tol, (float(a), int(b))) for a, b in pairs]
    return out


def batched_leg(args, B, problems, ctx, dev):
    """64 independent solves, finest grids drawn (seeded) from 32..128 with
    coarsest 8/6/8/6/8, mixed kinds of boundary data, u = four random sines,
    tol 1e-10, in FP64 (and with --batch-mixed also with FP32 correction
    solves in FP64 refinement).  All submitted at once to the batch engine;
    compared with the same 64 solved one by one."""
    import torch

    rng = np.random.Generator(np.random.PCG64(0))
    sizes = [int(v) for v in rng.choice([32, 48, 64, 96, 128], 64)]
    coarse = {32: 8, 48: 6, 64: 8, 96: 6, 128: 8}
    kinds = [int(v) for v in rng.integers(1, 3, 64)]
    tol = 1e-10
    inputs = [problems.random_sines_torch(2000 + i, sizes[i], kinds[i], dev) for i in range(64)]

    def run_batch(idx, precision):
        batch = B.Batch(ctx, max_instances=len(idx))
        outs = {}
        for i in idx:
            f, g1, g2 = inputs[i]
            ident, u = batch.submit(sizes[i], coarse[sizes[i]], kinds[i], f, g1, g2, tol, precision=precision)
            outs[i] = (ident, u)
        steps = 0
        while batch.step() > 0:
            steps += 1
        res = {i: (batch.query(ident), u) for i, (ident, u) in outs.items()}
        launches = batch.launches
        prof = batch.profile()
        batch.close()
        return res, steps + 1, launches, prof

    # warm-up: one instance of every (coarsest, kind) builds the DSOLVE inverses
    seen, warm = set(), []
    for i in range(64):
        key = (coarse[sizes[i]], kinds[i])
        if key not in seen:
            seen.add(key)
            warm.append(i)
    out = {"workload": "64 instances, n from {32,48,64,96,128} (PCG64 seed 0), coarsest 8/6/8/6/8, kinds mixed, "
                       "u = 4 random sines, tol 1e-10 per level"}
    for precision in (("fp64", "mixed") if args.batch_mixed else ("fp64",)):
        # untimed: the DSOLVE inverses, then one whole pass so that the
        # context's grid-size tuner has settled every level group
        run_batch(warm, precision)
        run_batch(list(range(64)), precision)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        res, steps, launches, prof = run_batch(list(range(64)), precision)
        torch.cuda.synchronize(dev)
        t_batch = time.perf_counter() - t0
        t0 = time.perf_counter()
        seq = {}
        for i in range(64):
            f, g1, g2 = inputs[i]
            seq[i] = B.excmg_solve(sizes[i], coarse[sizes[i]], kinds[i], f, g1, g2, tol, ctx=ctx, precision=precision)
        torch.cuda.synchronize(dev)
        t_seq = time.perf_counter() - t0
        diff = max(float((res[i][1] - seq[i]).abs().max() / seq[i].abs().max()) for i in range(64))
        out[precision] = {"batched_s": t_batch, "solves_per_s": 64 / t_batch, "engine_steps": steps,
                          "launches": launches, "engine_profile": prof,
                          "sequential_s": t_seq, "speedup_vs_sequential": t_seq / t_batch,
                          "max_rel_diff_vs_sequential": diff,
                          "all_ok": all(res[i][0]["done"] and res[i][0]["status"] == 0 for i in range(64))}
    return out


def serving_leg(args, B, ctx, dev):
    """Poisson request stream (sizes log-uniform in 32..256 rounded to
    c*2^k, kinds uniform, random-sine problems, tol 1e-8) through the batch
    engine at 0.8x its measured capacity; p50 / p99 latency and solves/s."""
    import torch

    from paper_1901_05118_gb300 import serving as S

    tol = 1e-8
    prec = {"precision": args.serve_precision}
    pool = S.InputPool(dev)
    new_out = lambda n: torch.empty((n + 1,) * 3, dtype=torch.float64, device=dev)
    # capacity: a closed burst of 64 requests from the same distribution
    burst = S.make_requests(64, rate=1e9, seed=11)
    pool.warm(burst)
    warm, seen = [], set()
    for r in burst:
        if (r.nc, r.bc) not in seen:
            seen.add((r.nc, r.bc))
            warm.append(r)
    S.serve(B.Batch(ctx, max_instances=256), warm, pool, tol, new_output=new_out, submit_kwargs=prec)
    # one untimed burst settles the context's grid-size tuner
    S.serve(B.Batch(ctx, max_instances=256), burst, pool, tol, new_output=new_out, submit_kwargs=prec)
    torch.cuda.synchronize(dev)
    _, cap = S.serve(B.Batch(ctx, max_instances=256), burst, pool, tol, new_output=new_out, submit_kwargs=prec)
    # 0.8x capacity, but the stream lasts at most about --serve-max-s seconds
    rate = 0.8 * cap["solves_per_s"]
    if args.serve_max_s > 0:
        rate = max(rate, args.serve_requests / args.serve_max_s)
    reqs = S.make_requests(args.serve_requests, rate=rate, seed=1)
    pool.warm(reqs)
    torch.cuda.synchronize(dev)
    budget = 64 * (1 << 30)
    recs, summ = S.serve(B.Batch(ctx, hbm_budget_bytes=budget, max_instances=256), reqs, pool, tol,
                         new_output=new_out, submit_kwargs=prec, keep_outputs=False)
    summ.update({"capacity_solves_per_s": cap["solves_per_s"], "rate_per_s": rate, "hbm_budget_bytes": budget,
                 "precision": args.serve_precision,
                 "workload": (f"{args.serve_requests} requests, Poisson at "
                              + (f"max(0.8x capacity, requests / {args.serve_max_s:g} s), " if args.serve_max_s > 0
                                 else "0.8x capacity, ")
                              + "n log-uniform in "
                              "[32, 256] rounded to c*2^k (c = 4..7), kinds uniform, 4 random-sine problems "
                              "per (n, kind), tol 1e-8")})
    return summ


def oracle_report():
    """CPU-baseline figures of the oracle on this host (single-threaded C):
    the whole small workload (32^3, coarsest 4, first kind, u = sin pi x sin
    pi y sin pi z, tol 1e-10 per level) and one operator application on 512^3."""
    import oracle
    from paper_1901_05118_gb300 import problems

    prob = problems.sin_pi()
    f, g1, g2 = prob.data(32, 1)
    t0 = time.perf_counter()
    _, _, st = oracle.excmg(32, 4, 1, f, g1, g2, 1e-10)
    t_small = time.perf_counter() - t0
    u = problems.random_field(512, 7)
    t0 = time.perf_counter()
    oracle.stencil_apply(512, 1, u)
    t_op = time.perf_counter() - t0
    print(json.dumps({"oracle_small_workload_s": t_small, "levels": st[:, 0].astype(int).tolist(),
                      "oracle_stencil_512_s": t_op, "oracle_stencil_512_GBs": 16 * 511 ** 3 / t_op / 1e9,
                      "cores": 1, "host_cpus": os.cpu_count()}), flush=True)


def profile_case(args):
    """A small, fixed GPU case for profiling single kernels: `stencil` (reps
    operator applications), `bicg` (iters Bi-CG iterations from x = 0 on a
    random right-hand side), `solve` (one EXCMG solve of u = e^(x+y+z)) or
    `batch` (16 solves of one size in the batch engine).
    At n = 256 the inputs are still larger than L2 and a capture of a few
    launches ends quickly."""
    import torch

    from paper_1901_05118_gb300 import binding as B, problems

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ctx = B.Context(dev)
    ctx.set_stencil(args.stencil)
    ctx.set_schedule(args.schedule)
    ctx.set_shadow_mode(args.shadow)
    n = args.n
    gen = torch.Generator(device=dev)
    gen.manual_seed(0)
    if args.case == "stencil":
        u = torch.rand((n + 1,) * 3, dtype=torch.float64, device=dev, generator=gen)
        y = torch.empty_like(u)
        lvl = B.Level(n, args.bc, ctx)
        for _ in range(args.reps):
            B.stencil_apply(lvl, u, y)
    elif args.case == "bicg":
        b = torch.rand((n + 1,) * 3, dtype=torch.float64, device=dev, generator=gen)
        x = torch.zeros_like(b)
        lvl = B.Level(n, args.bc, ctx)
        B.bicg_solve(lvl, b, x, 0.0, args.iters)
    elif args.case == "batch":
        # 16 instances of one size (random sines, alternating kinds) in the batch engine
        batch = B.Batch(ctx, max_instances=16)
        for i in range(16):
            f, g1, g2 = problems.random_sines_torch(5000 + i, n, 1 + i % 2, dev)
            batch.submit(n, args.nc, 1 + i % 2, f, g1, g2, args.tol, precision=args.precision)
        batch.run()
        batch.close()
    else:
        f, g1, g2 = (torch.from_numpy(v).to(dev) for v in problems.exp_sum().data(n, args.bc))
        B.excmg_solve(n, args.nc, args.bc, f, g1, g2, args.tol, ctx=ctx, precision=args.precision)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "n": n, "ok": True}), flush=True)


def main():
    args = parse()
    if args.case:
        profile_case(args)
        return
    if args.oracle_report:
        oracle_report()
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
