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
