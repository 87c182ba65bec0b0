"""Host-side helpers of bench.py that need no GPU."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def test_cpulist_parses_ranges_and_singles():
    assert bench._cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench._cpulist("5") == {5}
    assert bench._cpulist("") == set()


def test_config_names_the_workload():
    args = bench.parse([])
    cfg = bench.config(args)
    assert cfg["n_finest"] == 512 and cfg["n_coarsest"] == 8 and cfg["levels"] == 7
    assert cfg["schedule"] == "fused" and cfg["stencil"] == "exact"
    assert "512^3" in cfg["workload"]


def test_oracle_sampler_bounded_and_scaled(monkeypatch):
    """The oracle sample times iterations only up to 256^3 and fixed work only
    on 128^3; larger levels take those times scaled by their unknowns, and the
    whole-solve figure is the oracle's own per-level counts times them."""
    s = bench.OracleSampler(512, 8, 1)
    assert s.counts is not None and s.levels == [32, 64, 128, 256, 512]
    timed = []

    def fake_iteration(N, bc):
        timed.append(N)
        return 1e-3 * ((N - 1) / 31) ** 3

    monkeypatch.setattr(s, "_fixed_parts", lambda N, bc: (0.5 * ((N - 1) / 127) ** 3, 0.1 * ((N - 1) / 127) ** 3))
    real = bench.OracleSampler.iteration_s

    def iteration_s(N, bc):
        if N > s.ITER_MAX_N:
            return real(s, N, bc)        # scales the 256^3 figure
        return fake_iteration(N, bc)

    monkeypatch.setattr(s, "iteration_s", iteration_s)
    total, parts = s.solve_s(1)
    assert max(timed) == 256 and 512 not in timed
    lv = {L["n"]: L for L in s.counts[1]["levels"]}
    want = 0.0
    for N in s.levels:
        it = 1e-3 * ((N - 1) / 31) ** 3
        scale = ((N - 1) / 127) ** 3
        want += lv[N]["iters"] * it + (0.5 + (lv[N]["calls"] + 1) * 0.1) * scale
    assert abs(total - want) <= 1e-9 * want
    assert [p["n"] for p in parts] == s.levels
