"""bench.py's JSON lines on a GPU: the keys and units each arm promises, on
small, quick settings (the numbers themselves are not checked here)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, timeout=600):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                         text=True, timeout=timeout)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_default_line_keys():
    d = run_bench("--steps", "4", "--warmup", "3", "--pages", "65536", "--no-serving", "--no-batching",
                  "--e2e-pages", "65536", "--cpu-seconds", "1")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks",
              "gpu_launches"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 4 and d["warmup"] == 3 and d["gpu_launches"] == 8
    assert d["unit"] == "GB/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["workload"].startswith("profiling case") and "L2" in d["config"]["l2"]
    r = d["roofline"]
    assert r["bound"] == "alu" and r["peak"] > 0 and 0 < r["frac"] == pytest.approx(r["achieved"] / r["peak"], 1e-3)
    assert r["traffic"] is None                      # the committed capture is of the 1 GiB launch only
    e = d["e2e"]
    assert e["unit"] == "GB/s" and e["value"] > 0 and e["round_trip_ok"] is True
    assert e["h2d_bytes_per_step"] == e["d2h_bytes_per_step"] == 2 * 65536 * 4096
    assert e["link"]["bound_gbs"] > 0 and 0 < e["frac_of_link"]
    ip = e["in_place"]                               # the same passes in place over the host link
    assert ip["value"] > 0 and ip["round_trip_ok"] is True and ip["h2d_bytes_per_step"] == 0
    assert ip["link_bytes_per_step_each_way"] == 2 * 65536 * 4096
    c = d["cpu_baseline"]
    assert c["kind"] == "oracle" and c["cores"] >= 1 and c["value"] > 0 and c["sample"]
    assert set(d["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}
    assert d["clocks"]["samples"] >= 20 and d["clocks"]["sm_mhz"] > 0


def test_default_line_batching_and_serving_summaries():
    """The default line's batching and serving summaries, on a reduced batching
    workload and a small working set (keys only)."""
    d = run_bench("--steps", "3", "--warmup", "3", "--pages", "65536", "--no-e2e", "--no-cpu", "--batching-scale",
                  "0.05", "--serve-pages", "65536", "--serve-seconds", "1.5", "--serve-rates", "10000,141000",
                  "--one-per-launch-cap", "5000", timeout=900)
    b = d["batching"]
    assert b["unit"] == "pages/s" and b["fed"]["identical_to_one_launch_per_request"] is True
    assert b["graph_launched"]["identical_to_one_launch_per_request"] is True
    assert b["one_launch_per_request"]["pages_per_s"] > 0 and b["speedup_vs_one_launch_per_request"] > 0
    rows = d["serving"]["rows"]
    assert {(r["offered_pages_per_s"], r["mode"]) for r in rows} == {
        (rate, m) for rate in (1e4, 1.41e5) for m in ("continuous", "one_per_launch", "resident")}
    for r in rows:
        assert r["first_second"]["p99_us"] > 0 and r["p99_us_by_second"]
        if r["mode"] == "one_per_launch":
            assert r["requests"] <= 5000
    assert len(d["serving"]["vs_one_per_launch"]) == 4


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--steps", "3", "--warmup", "3")
    assert d["impl"] == "reference" and d["unit"] == "GB/s" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert f" {d['config']['pages']} pages" in d["cpu_baseline"]["sample"]    # the pages actually timed


def test_small_workload_line():
    d = run_bench("--workload", "small", "--steps", "50", "--warmup", "3")
    assert d["unit"] == "us" and d["higher_is_better"] is False and d["round_trip_ok"] is True
    assert d["pages_changed_by_one_encrypt"] == 256
    for form in ("host_list", "device_list"):
        assert 0 < d["forms"][form]["back_to_back_us"] <= d["forms"][form]["call_to_sync_us_p50"]
