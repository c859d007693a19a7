"""bench.py's host-side bookkeeping, without a GPU: the split of serving
latencies into the first second and the steady state."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_latency_split_first_second_and_steady():
    arrival = np.concatenate([np.linspace(0, 0.999, 1000), np.linspace(1.0, 4.999, 4000)])
    lat = np.concatenate([np.full(1000, 5e-3), np.full(4000, 50e-6)])   # a bad first second
    out = bench.latency_split(arrival, lat)
    assert out["first_second"]["requests"] == 1000 and out["steady"]["requests"] == 4000
    assert out["first_second"]["p99_us"] == 5000.0 and out["steady"]["p99_us"] == 50.0
    assert out["steady"]["p50_us"] <= out["steady"]["p99_us"] <= out["steady"]["p999_us"]


def test_latency_split_short_run_has_no_steady_state():
    arrival = np.linspace(0, 0.7, 100)
    out = bench.latency_split(arrival, np.full(100, 1e-4))
    assert out["steady"] is None and out["first_second"]["requests"] == 100
