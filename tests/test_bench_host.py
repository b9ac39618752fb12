"""Host helpers of bench.py (no GPU): per-workload defaults, and the DRAM
traffic of the sweep, which is reported only while the sweep source matches
the source the ncu figures were taken on."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_workload_defaults():
    for wl, (n, steps) in bench.WORKLOAD_DEFAULTS.items():
        a = bench.parse_args(["--workload", wl])
        assert (a.n, a.steps) == (n, steps)
    a = bench.parse_args(["--steps", "7", "--n", "64"])
    assert (a.workload, a.n, a.steps, a.warmup, a.gpus) == ("turb", 64, 7, 3, 1)


def test_traffic_follows_the_source_hash(monkeypatch):
    zones = 1000
    h = bench.kernel_source_hash()
    monkeypatch.setattr(bench, "SWEEP_TRAFFIC", {"src": h, "fp64": 100.0, "fp32": 40.0})
    assert bench.sweep_traffic("fp64", zones) == 100.0 * zones
    assert bench.sweep_traffic("fp32", zones) == 40.0 * zones
    monkeypatch.setattr(bench, "SWEEP_TRAFFIC", {"src": "0" * 16, "fp64": 100.0, "fp32": 40.0})
    assert bench.sweep_traffic("fp64", zones) is None
    assert bench.hbm_gbs(None, 1.0) is None
    assert bench.hbm_gbs(2e9, 1.0) == 2000.0

