"""Continuous-batching EXCMG solve server on one GPU.

Requests (grid size, kind of boundary data, manufactured problem) arrive as a
Poisson stream.  Each arrival waits in a queue until the batch engine
(``binding.Batch``, C ABI ``excmg_batch_*``) admits it against its
device-memory budget; admitted solves run together -- their FP32 correction
solves in one cooperative launch per engine step -- and leave as soon as they
finish, which frees budget for the queue.  Latency = completion time minus
arrival time (queueing included).
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np

SIZE_BASES = (4, 5, 6, 7)
REJECTED = -9   # status recorded for a request the engine refuses while idle (EXCMG_ERR_BUDGET)


def size_grid(lo: int = 32, hi: int = 256):
    """Sizes c * 2^k (c in 4..7, k >= 3) within [lo, hi], ascending."""
    out = set()
    for c in SIZE_BASES:
        k = 3
        while c << k <= hi:
            if c << k >= lo:
                out.add(c << k)
            k += 1
    return sorted(out)


def round_size(n: float, lo: int = 32, hi: int = 256) -> int:
    """The grid size of size_grid(lo, hi) nearest to n (log distance)."""
    g = size_grid(lo, hi)
    return min(g, key=lambda v: abs(math.log(v) - math.log(n)))


def coarsest_for(n: int) -> int:
    """Coarsest grid of Alg. 1 for n = c * 2^k: c for c in 5..7, 8 for c = 4
    (two direct-solve grids, at least one Bi-CG grid)."""
    c = n
    while c > 7:
        c //= 2
    if c == 4 or c * 2 == 8:
        return 8
    return c


@dataclass(order=True)
class Request:
    t_arrival: float
    rid: int = field(compare=False)
    n: int = field(compare=False)
    nc: int = field(compare=False)
    bc: int = field(compare=False)
    problem_seed: int = field(compare=False)


def make_requests(count: int, rate: float, seed: int, lo: int = 32, hi: int = 256, n_problems: int = 4):
    """Seeded Poisson stream: exponential inter-arrival times of mean 1/rate,
    sizes log-uniform in [lo, hi] rounded to size_grid, kind of boundary data
    uniform over {1, 2}, one of n_problems random-sine problems."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for rid in range(count):
        t += float(rng.exponential(1.0 / rate))
        n = round_size(float(np.exp(rng.uniform(np.log(lo), np.log(hi)))), lo, hi)
        bc = int(rng.integers(1, 3))
        ps = int(rng.integers(0, n_problems))
        out.append(Request(t, rid, n, coarsest_for(n), bc, ps))
    return out


class InputPool:
    """Device-resident inputs (f, g1, g2) per (n, bc, problem seed), built once."""

    def __init__(self, device, base_seed: int = 1000):
        self.device = device
        self.base_seed = base_seed
        self.cache = {}

    def get(self, n: int, bc: int, ps: int):
        key = (n, bc, ps)
        if key not in self.cache:
            from .problems import random_sines_torch
            self.cache[key] = random_sines_torch(self.base_seed + ps, n, bc, self.device)
        return self.cache[key]

    def warm(self, requests):
        for r in requests:
            self.get(r.n, r.bc, r.problem_seed)


def serve(engine, requests, pool, tol: float, clock=time.perf_counter, new_output=None, sleep=time.sleep,
          submit_kwargs=None, keep_outputs: bool = True):
    """Run the request stream through `engine` (a binding.Batch or anything
    with submit/step/query; submit_kwargs go to every submit).  Returns
    per-request records (with each result when keep_outputs) and a
    summary."""
    submit_kwargs = submit_kwargs or {}
    pending = collections.deque(sorted(requests))
    queued = collections.deque()
    live = {}
    records = []
    t0 = clock()
    steps = 0
    while pending or queued or live:
        now = clock() - t0
        while pending and pending[0].t_arrival <= now:
            queued.append(pending.popleft())
        while queued:
            r = queued[0]
            f, g1, g2 = pool.get(r.n, r.bc, r.problem_seed)
            out = new_output(r.n) if new_output else None
            try:
                sub = engine.submit(r.n, r.nc, r.bc, f, g1, g2, tol, out, **submit_kwargs)
            except Exception as exc:          # e.g. larger than the whole budget
                sub = exc
            if sub is None and live:
                break            # budget or slots full: wait for completions
            if sub is None or isinstance(sub, Exception):
                # refused with nothing running: it can never be admitted
                status = getattr(sub, "status", REJECTED)
                queued.popleft()
                records.append({"rid": r.rid, "n": r.n, "bc": r.bc, "status": status, "latency_s": 0.0,
                                "arrival_s": r.t_arrival, "engine_latency_s": None, "output": None,
                                "rejected": True})
                continue
            live[sub[0]] = (r, sub[1])
            queued.popleft()
        if live:
            engine.step()
            steps += 1
            t_now = clock() - t0
            for ident in list(live):
                q = engine.query(ident)
                if q["done"]:
                    r, u = live.pop(ident)
                    records.append({"rid": r.rid, "n": r.n, "bc": r.bc, "status": q["status"],
                                    "latency_s": t_now - r.t_arrival, "arrival_s": r.t_arrival,
                                    "engine_latency_s": q.get("latency_s"), "output": u if keep_outputs else None})
        elif pending:
            sleep(max(0.0, min(0.01, pending[0].t_arrival - (clock() - t0))))
    wall = clock() - t0
    solved = [rec for rec in records if not rec.get("rejected")]
    lat = np.array([rec["latency_s"] for rec in solved]) if solved else np.zeros(1)
    summary = {"requests": len(records), "rejected": len(records) - len(solved), "wall_s": wall,
               "solves_per_s": len(solved) / wall if wall > 0 else 0.0,
               "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
               "mean_s": float(lat.mean()), "steps": steps,
               "failed": sum(1 for rec in records if rec["status"] != 0)}
    if hasattr(engine, "profile"):
        summary["engine_profile"] = engine.profile()
    return records, summary
