#!/usr/bin/env python3
"""Benchmark of the B300 page cipher (MemShield Sec. 4.4 hot path).

Default workload (one JSON line on rank 0): the bulk device-resident
configuration -- 1 GiB = 262,144 pages x 4 KiB of SplitMix64(seed 2) bytes in
HBM, page ids 0..262143, key = SplitMix64(seed 1)[0:32].  One step is one
encrypt launch plus one decrypt launch over the whole buffer, through the
C-ABI device-list entry points.  The buffer (1 GiB) is larger than the L2
(126 MB), so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``value`` is page bytes processed per second (encrypt and decrypt bytes both
count) over all ranks; ``e2e`` is the same metric through ms_crypt_host with
the pages in pinned HOST memory (host<->device copies inside the timed
region); ``roofline`` relates the page kernel's average launch time to the
integer-ALU peak; ``cpu_baseline`` times the CPU oracle on the host cores on
a bounded sample of the same buffer.  Under torchrun (N > 1) every rank runs
an independent replica on its own GPU (the pages shard with no exchange).
``--impl reference`` times the CPU oracle itself on this workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PAGE = 4096
L2_BYTES = 126 * 10**6
BULK_PAGES = 262144
OPS_PER_BLOCK = 992            # 80 quarter rounds x 12 + 16 feed-forward adds + 16 data XORs
INT32_LANES_PER_SM = 128       # 4 schedulers x 32 lanes issue one int32 op each per clock
ALU_PIPE_LANES_PER_SM = 64     # xor / funnel-shift / byte-permute pipe, measured at half the issue width
ALU_PIPE_OPS_PER_BLOCK = 656   # 320 + 16 xors and 320 rotations per block must use that pipe
WORKLOAD = ("bulk: 1 GiB = 262,144 x 4 KiB pages resident in HBM (SplitMix64 seed 2), page ids "
            "0..262143, key = SplitMix64(seed 1)[0:32], ChaCha20; one encrypt launch + one decrypt "
            "launch per step")


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_2004_09252_b300", "csrc", "ms_cipher.cuh"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the bulk page kernel from the committed ncu summary,
    or None when the kernel source changed since the capture."""
    p = os.path.join(ROOT, "profiles", "k_pages_bulk_1gib.md")
    if not os.path.exists(p):
        return None
    text = open(p).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.e+]+)", text)
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    if not m or not h or h.group(1) != kernel_source_hash():
        return None
    return float(m.group(1))


# ------------------------------------------------------------------ clocks
REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
           0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown", 0x2: "applications_clocks_setting",
           0x1: "gpu_idle", 0x10: "sync_boost"}


class ClockSampler:
    """Samples the SM clock and the clock-event reasons while the GPU is under
    load: NVML when the binding is importable, else an ``nvidia-smi -lms``
    child whose lines are read as they arrive.  Every sample carries its
    host time, so the summary can say how many fell inside the timed region
    (``mark_start``/``mark_end``) and how many in the loaded window around it."""

    def __init__(self, torch_dev: int, period_s: float = 0.025):
        self.samples = []            # (monotonic time, sm MHz, reason bits)
        self.max_mhz = None
        self.period = period_s
        self._stop = threading.Event()
        self._t = None
        self.err = None
        self.t_start = self.t_end = None
        self.lock = threading.Lock()
        try:
            import pynvml
            pynvml.nvmlInit()
            import torch
            props = torch.cuda.get_device_properties(torch_dev)
            h = None
            try:
                bus = "%08x:%02x:%02x.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
                h = pynvml.nvmlDeviceGetHandleByPciBusId(bus)
            except Exception:
                h = pynvml.nvmlDeviceGetHandleByIndex(torch_dev)
            self.nvml, self.h = pynvml, h
            self.max_mhz = pynvml.nvmlDeviceGetMaxClockInfo(h, pynvml.NVML_CLOCK_SM)
        except Exception as e:  # no NVML binding: fall back to nvidia-smi sampling
            self.nvml, self.h, self.err = None, None, f"{type(e).__name__}: {e}"
        self.smi = None
        self.smi_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(torch_dev)).split(",")[0] or "0"

    def _add(self, mhz, reasons):
        with self.lock:
            self.samples.append((time.monotonic(), float(mhz), int(reasons)))

    def _run_nvml(self):
        n = self.nvml
        while not self._stop.is_set():
            try:
                mhz = n.nvmlDeviceGetClockInfo(self.h, n.NVML_CLOCK_SM)
                try:
                    r = n.nvmlDeviceGetCurrentClocksEventReasons(self.h)
                except AttributeError:
                    r = n.nvmlDeviceGetCurrentClocksThrottleReasons(self.h)
                self._add(mhz, r)
            except Exception:
                pass
            time.sleep(self.period)

    def _run_smi(self):
        for line in self.smi.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 3:
                continue
            try:
                mhz, mx, r = float(parts[0]), float(parts[1]), int(parts[2], 16)
            except ValueError:
                continue
            self.max_mhz = mx
            self._add(mhz, r)

    def __enter__(self):
        if self.nvml:
            self._t = threading.Thread(target=self._run_nvml, daemon=True)
        else:
            import subprocess
            try:
                self.smi = subprocess.Popen(
                    ["nvidia-smi", "-i", self.smi_index, "--query-gpu=clocks.sm,clocks.max.sm,"
                     "clocks_event_reasons.active", "--format=csv,noheader,nounits",
                     "-lms", str(int(self.period * 1000))],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, bufsize=1)
                self._t = threading.Thread(target=self._run_smi, daemon=True)
            except Exception as e:
                self.err = f"{self.err}; nvidia-smi: {e}"
        if self._t:
            self._t.start()
        return self

    def count(self, since=None):
        with self.lock:
            return sum(1 for t, _, _ in self.samples if since is None or t >= since)

    def mark_start(self):
        self.t_start = time.monotonic()

    def mark_end(self):
        self.t_end = time.monotonic()

    def __exit__(self, *a):
        self._stop.set()
        if self.smi:
            self.smi.terminate()
            try:
                self.smi.wait(timeout=10)
            except Exception:
                self.smi.kill()
        if self._t:
            self._t.join(timeout=10)

    def summary(self, loaded_since=None):
        """Median SM clock and the reasons seen over the samples taken since
        ``loaded_since`` (the start of the loaded window), with the count of
        those inside the timed region."""
        with self.lock:
            sel = [x for x in self.samples if loaded_since is None or x[0] >= loaded_since]
        reasons = set()
        for _, _, r in sel:
            for bit, name in REASONS.items():
                if r & bit and name != "gpu_idle":
                    reasons.add(name)
        timed = [x for x in sel if self.t_start is not None and self.t_start <= x[0] <= (self.t_end or 1e300)]
        src = "nvml" if self.nvml else ("nvidia-smi" if self.smi else "none")
        out = {"sm_mhz": statistics.median(m for _, m, _ in sel) if sel else None,
               "sm_max_mhz": self.max_mhz, "reasons": sorted(reasons), "samples": len(sel),
               "samples_in_timed_region": len(timed),
               "sm_mhz_timed_region": statistics.median(m for _, m, _ in timed) if timed else None,
               "window": "the timed steps plus untimed steps of the same launches right before them "
                         "(the GPU under the same load throughout)",
               "source": src}
        if not self.nvml:
            out["nvml_error"] = self.err
        return out


# ----------------------------------------------------------- replicas (N>1)
def aggregate_replicas(elapsed_ms: float, bytes_local: float, world: int, device="cpu"):
    """Whole-job figures over independent replicas: the max elapsed time over
    ranks and all ranks' bytes divided by it (GB/s).  With world == 1 this is
    the local figure; with world > 1 it uses the default process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    b = torch.tensor([bytes_local], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(b, op=dist.ReduceOp.SUM)
    max_ms, total = float(t.item()), float(b.item())
    return max_ms, total / (max_ms / 1e3) / 1e9


# --------------------------------------------------------------- CPU oracle
def cpu_oracle_rate(seconds: float, threads: int):
    """Time the CPU oracle (as it stands) on a bounded sample of the bulk buffer."""
    import numpy as np

    import oracle
    import synth
    oracle.build()
    key = synth.key_bytes(1)
    cal = synth.page_bytes_fast(2, 0, 32)
    ids = np.arange(32, dtype=np.uint64)
    t0 = time.perf_counter()
    oracle.crypt_pages(key, cal, ids, ids, threads=1)
    per_page = (time.perf_counter() - t0) / 32
    n = int(max(threads * 8, min(BULK_PAGES, seconds / per_page * threads)))
    buf = synth.page_bytes_fast(2, 0, n)
    ids = np.arange(n, dtype=np.uint64)
    passes = 0
    t0 = time.perf_counter()
    while True:                      # whole passes until `seconds` of wall time
        oracle.crypt_pages(key, buf, ids, ids, threads=threads)
        passes += 1
        dt = time.perf_counter() - t0
        if dt >= seconds or passes >= 64:
            break
    return passes * n * PAGE / dt / 1e9, n, dt, passes


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ------------------------------------------------------------------- ours
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    from paper_2004_09252_b300 import memshield as ms

    rank, world, local = env_rank()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    key = synth.key_bytes(1)
    n = args.pages
    plain = synth.page_bytes_fast(2, 0, n)
    d = torch.from_numpy(plain).to(f"cuda:{dev}")
    ids = np.arange(n, dtype=np.uint64)
    lst = torch.from_numpy(ms.pages_array(d.data_ptr() + PAGE * ids, ids).view(np.uint8)).to(f"cuda:{dev}")
    ctx = ms.Context(key, device=dev, stream=stream.cuda_stream)
    if args.shape:
        ctx.set_shape(*(int(x) for x in args.shape.split(",")))
    shape = ctx.get_shape()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        ctx.encrypt_pages_dev(lst, n)
        ctx.decrypt_pages_dev(lst, n)
    if ctx.sync() != 0:
        raise RuntimeError("warm-up failed")
    # correctness guard: after warm-up (even number of XORs) the buffer is the plaintext
    if not torch.equal(d[:PAGE * 64], torch.from_numpy(plain[:PAGE * 64]).to(d.device)):
        raise RuntimeError("round trip check failed")

    K = args.steps
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * K + 1)]
    sampler = ClockSampler(dev)
    with sampler:
        # untimed steps of the same launches until the sampler has seen the
        # loaded GPU at least 24 times (a few seconds at most): the timed
        # region of a short run is shorter than one sampling period
        barrier()
        loaded = time.monotonic()
        while sampler.count(loaded) < 24 and time.monotonic() - loaded < 6.0:
            for _ in range(64):
                ctx.encrypt_pages_dev(lst, n)
                ctx.decrypt_pages_dev(lst, n)
            torch.cuda.synchronize()
        barrier()
        sampler.mark_start()
        evs[0].record(stream)
        for k in range(K):
            ctx.encrypt_pages_dev(lst, n)
            evs[2 * k + 1].record(stream)
            ctx.decrypt_pages_dev(lst, n)
            evs[2 * k + 2].record(stream)
        barrier()
        sampler.mark_end()
    rc = ctx.sync()
    if rc != 0:
        raise RuntimeError(f"ms_sync failed: {ms.strerror(rc)}")
    launch_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(2 * K)]
    total_ms, value = aggregate_replicas(evs[0].elapsed_time(evs[-1]), 2.0 * K * n * PAGE, world, d.device)
    avg_launch_s = statistics.mean(launch_ms) / 1e3

    peaks, peaks_kind = load_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    alu_peak = props.multi_processor_count * INT32_LANES_PER_SM * sm_max * 1e6 / 1e12
    ops_launch = n * 64 * OPS_PER_BLOCK
    alu_pipe_peak = (props.multi_processor_count * ALU_PIPE_LANES_PER_SM * sm_max * 1e6
                     * OPS_PER_BLOCK / ALU_PIPE_OPS_PER_BLOCK / 1e12)
    achieved = ops_launch / avg_launch_s / 1e12
    alg_bytes = n * (2 * PAGE + 16)
    traffic = profiled_traffic() if n == BULK_PAGES else None  # the capture is of the 1 GiB launch

    # e2e through the host-page entry point on the host-page workload: a 4 GiB
    # pinned host buffer (seed 4), copies inside the timed region, beside the
    # host link measured in the same run
    e2e = None
    if not args.no_e2e:
        ne = args.e2e_pages
        hbuf = torch.empty(ne * PAGE, dtype=torch.uint8).pin_memory()
        synth.fill_pages(hbuf.data_ptr(), 4, 0, ne)
        head = hbuf[:PAGE * 64].clone()
        link = host_link(hbuf)
        chunk = args.e2e_chunk_mib << 20
        ctx.crypt_host(ms.MS_ENCRYPT, hbuf, 0, ne, chunk, args.e2e_streams)
        ctx.crypt_host(ms.MS_DECRYPT, hbuf, 0, ne, chunk, args.e2e_streams)
        es = max(2, min(5, K))
        barrier()
        t0 = time.perf_counter()
        for _ in range(es):
            ctx.crypt_host(ms.MS_ENCRYPT, hbuf, 0, ne, chunk, args.e2e_streams)
            ctx.crypt_host(ms.MS_DECRYPT, hbuf, 0, ne, chunk, args.e2e_streams)
        barrier()
        el_ms, e2e_gbs = aggregate_replicas((time.perf_counter() - t0) * 1e3, 2.0 * es * ne * PAGE, world,
                                            d.device)
        ok = torch.equal(hbuf[:PAGE * 64], head)
        e2e = {"value": round(e2e_gbs, 3), "unit": "GB/s",
               "h2d_bytes_per_step": 2 * ne * PAGE, "d2h_bytes_per_step": 2 * ne * PAGE,
               "workload": (f"host pages: {ne * PAGE / 2**30:g} GiB pinned host buffer ({ne} pages, SplitMix64 "
                            "seed 4), ids 0.., through ms_crypt_host; a step = one encrypt pass + one decrypt pass"),
               "steps": es, "chunk_bytes": chunk, "streams": args.e2e_streams or 2,
               "host_memory": "pinned", "round_trip_ok": bool(ok),
               "link": link, "frac_of_link": round(e2e_gbs / world / link["bound_gbs"], 3)}
        # the same passes in place over the host link (ms_crypt_host_inplace:
        # the SMs read and write the pinned pages, no copy engine, no device buffer)
        e2e["in_place"] = in_place_result(ms, ctx, hbuf, ne, es, head, link, world, d.device, barrier)
        del hbuf

    ctx.shutdown()
    pipes = ms.probe_int_pipes(dev)  # the op-class rates the ALU-pipe peak below assumes
    line = {
        "metric": "page encrypt GB/s (ChaCha20, 4 KiB pages, device-resident)",
        "value": round(value, 3),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": round(total_ms / K, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic (SplitMix64 seeded page bytes)",
        "config": {"workload": WORKLOAD if n == BULK_PAGES else f"profiling case: {n} pages of the bulk buffer",
                   "pages": n, "page_bytes": PAGE, "rounds": 20,
                   "l2": (f"inputs larger than L2 ({n * PAGE / 2**20:.0f} MiB vs 126 MB), no flush"
                          if n * PAGE > L2_BYTES else f"inputs fit in L2 ({n * PAGE / 2**20:.0f} MiB): "
                                                     "DRAM figures do not apply"),
                   "parallelism": f"replicas{world}",
                   "shape": shape},
        "gpu_launches": 2 * K,
        "roofline": {"bound": "alu", "achieved": round(achieved, 3), "peak": round(alu_peak, 3),
                     "unit": "Tops/s (int32)", "frac": round(achieved / alu_peak, 4), "traffic": traffic,
                     "peak_source": f"{props.multi_processor_count} SMs x {INT32_LANES_PER_SM} int32 lanes x "
                                    f"{sm_max:.0f} MHz ({peaks_kind} max SM clock)",
                     "ops_per_launch": ops_launch, "avg_launch_ms": round(avg_launch_s * 1e3, 5),
                     "alu_pipe": {"peak": round(alu_pipe_peak, 3), "frac": round(achieved / alu_pipe_peak, 4),
                                  "note": f"{props.multi_processor_count} SMs x {ALU_PIPE_LANES_PER_SM} lanes x "
                                          f"{sm_max:.0f} MHz on the xor/rotate pipe, x {OPS_PER_BLOCK}/"
                                          f"{ALU_PIPE_OPS_PER_BLOCK} algorithmic ops per pipe op",
                                  "probe_lanes_per_sm_clk": {r["class"]: r["lanes_per_sm_clk"] for r in pipes}},
                     "hbm": {"achieved_gbs": round(alg_bytes / avg_launch_s / 1e9, 1),
                             "peak_gbs": peaks.get("hbm_gbs"),
                             "frac": round(alg_bytes / avg_launch_s / 1e9 / float(peaks.get("hbm_gbs", 6400.0)), 4),
                             "note": f"{peaks_kind} copy bandwidth"}},
        "clocks": sampler.summary(loaded),
        "e2e": e2e,
    }
    if not args.no_batching and world == 1:
        # the batching workload at full size: one launch per request, graph-launched
        # submits (doubling from 60 to 4000 requests) and the fed form
        br = batching_result(args, ["r60-4000"], [16384])
        fed = next(r for r in br["batched"] if str(r["requests_per_submit"]).startswith("fed"))
        graph = next(r for r in br["batched"] if not str(r["requests_per_submit"]).startswith("fed"))
        keys = ("pages_per_s", "gb_per_s", "gpu_span_ms", "wall_s", "identical_to_one_launch_per_request")
        line["batching"] = {
            "workload": br["config"]["workload"], "unit": "pages/s",
            "one_launch_per_request": br["one_launch_per_request"],
            "graph_launched": dict({k: graph[k] for k in keys}, submits=graph["submits"],
                                   requests_per_submit=graph["requests_per_submit"]),
            "fed": dict({k: fed[k] for k in keys}, publications=fed["publications"]),
            "speedup_vs_one_launch_per_request": br["speedup_vs_one_launch_per_request"],
            "autotune": br["autotune"]}
    if not args.no_serving and world == 1:
        rows, setup_s = serve_rows(args, args.serve_rates, ["continuous", "one_per_launch", "resident"],
                                   args.serve_seconds, one_per_launch_cap=args.one_per_launch_cap,
                                   reps_below=(1e5, args.low_rate_reps))
        keep = ("offered_pages_per_s", "mode", "requests", "arrival_s", "sustained_pages_per_s", "p50_us", "p99_us",
                "p999_us", "reps", "p99_us_each", "first_second", "steady", "p99_us_by_second", "max_submit_lag_ms",
                "max_server_pass_ms")
        one = {r["offered_pages_per_s"]: r for r in rows if r["mode"] == "one_per_launch"}

        def p99(r):  # the steady state where the run has one, else the whole run
            return r["steady"]["p99_us"] if r.get("steady") else r["p99_us"]
        line["serving"] = {
            "workload": SERVE_WORKLOAD.format(n=args.serve_pages, gib=args.serve_pages * PAGE / 2**30,
                                              sec=args.serve_seconds)
            + f"; one launch per request capped at {args.one_per_launch_cap} requests (>= 50k requests)"
            + f"; rates under 100k run {args.low_rate_reps} times (medians; every run in p99_us_each)"
            + (f"; {args.serve_warmup_s:g} s of separate requests replayed untimed before each run"
               if args.serve_warmup_s > 0 else ""),
            "working_set_setup_s": round(setup_s, 1),
            "rows": [{k: r[k] for k in keep} for r in rows],
            "vs_one_per_launch": [{"offered": r["offered_pages_per_s"], "mode": r["mode"],
                                   "steady_p99_us": p99(r), "one_per_launch_p99_us": p99(one[r["offered_pages_per_s"]]),
                                   "beats_one_per_launch": p99(r) <= p99(one[r["offered_pages_per_s"]])}
                                  for r in rows if r["mode"] != "one_per_launch"]}
    if rank == 0 and world == 1 and not args.no_cpu:
        threads = host_cores()
        v, npg, dt, passes = cpu_oracle_rate(args.cpu_seconds, threads)
        v1, npg1, dt1, passes1 = cpu_oracle_rate(max(2.0, args.cpu_seconds / 4), 1)
        line["cpu_baseline"] = {"value": round(v, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                                "sample": f"{npg} pages ({npg * PAGE / 2**20:.0f} MiB) of the bulk buffer, "
                                          f"{passes} encrypt passes in {dt:.1f} s, pages split over "
                                          f"{threads} threads",
                                "single_core": {"value": round(v1, 4), "unit": "GB/s",
                                                "sample": f"{npg1} pages, {passes1} passes in {dt1:.1f} s, 1 thread"}}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


# ------------------------------------------------------ batching (config 3)
def fill_device_pages(d, seed, n_pages, chunk_pages=262144):
    """Write pages 0..n_pages-1 of SplitMix64(seed) into device tensor d, in chunks."""
    import torch

    import synth
    h = torch.empty(min(chunk_pages, n_pages) * PAGE, dtype=torch.uint8).pin_memory()
    for p0 in range(0, n_pages, chunk_pages):
        np_ = min(chunk_pages, n_pages - p0)
        synth.fill_pages(h.data_ptr(), seed, p0, np_)
        d[p0 * PAGE:(p0 + np_) * PAGE].copy_(h[:np_ * PAGE])
    torch.cuda.synchronize()


def run_small(args):
    """256 pages of SplitMix64(seed 0), ids 0..255: latency of one launch (encrypt,
    then decrypt) through the host-list and the device-list entry points; the
    round trip must restore the input.  Too small to fill the GPU: no roofline."""
    import numpy as np
    import torch

    import synth
    from paper_2004_09252_b300 import memshield as ms

    n = 256
    key = synth.key_bytes(1)
    d = torch.empty(n * PAGE, dtype=torch.uint8, device="cuda")
    fill_device_pages(d, 0, n)
    plain = d.clone()
    stream = torch.cuda.current_stream()
    ctx = ms.Context(key, stream=stream)
    ids = np.arange(n, dtype=np.uint64)
    table = ms.pages_array(d.data_ptr() + PAGE * ids, ids)
    d_table = torch.from_numpy(table.view(np.uint8)).cuda()
    lib, h = ms.lib, ctx.handle
    host_fns = (lib.ms_encrypt_pages, lib.ms_decrypt_pages)
    dev_fns = (lib.ms_encrypt_pages_dev, lib.ms_decrypt_pages_dev)
    out = {}
    for form, fns, ptr in (("host_list", host_fns, table.ctypes.data), ("device_list", dev_fns, d_table.data_ptr())):
        for i in range(args.warmup * 2):
            fns[i % 2](h, ptr, n)
        torch.cuda.synchronize()
        dev_us, wall_us = [], []
        for i in range(2 * args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record(stream)
            rc = fns[i % 2](h, ptr, n)
            e1.record(stream)
            if rc or ctx.sync():
                raise RuntimeError(ms.strerror(rc) if rc else "sync failed")
            wall_us.append((time.perf_counter() - t0) * 1e6)
            dev_us.append(e0.elapsed_time(e1) * 1e3)
        # back to back: 2 * steps launches queued without a wait, one event pair around them
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(2 * args.steps):
            fns[i % 2](h, ptr, n)
        e1.record(stream)
        if ctx.sync():
            raise RuntimeError("sync failed")
        b2b = e0.elapsed_time(e1) * 1e3 / (2 * args.steps)
        out[form] = {"back_to_back_us": round(b2b, 2),
                     "device_us_p50": round(float(np.percentile(dev_us, 50)), 2),
                     "device_us_p99": round(float(np.percentile(dev_us, 99)), 2),
                     "call_to_sync_us_p50": round(float(np.percentile(wall_us, 50)), 2),
                     "call_to_sync_us_p99": round(float(np.percentile(wall_us, 99)), 2)}
    # one page per request, waited for on its own ticket (the fault path), on a
    # device page and on a pinned host page the kernel works on in place
    hpg = torch.empty(PAGE * 2, dtype=torch.uint8).pin_memory()
    one = {"device_page": ms.pages_array([d.data_ptr()], [0]),
           "pinned_host_page": ms.pages_array([ms.host_device_address(hpg)], [0])}
    for name, entry in one.items():
        lat = []
        for i in range(2 * (args.warmup + args.steps)):  # an even count: the page ends as it started
            t0 = time.perf_counter()
            ctx.wait(ctx.submit_host(i % 2, entry))
            if i >= 2 * args.warmup:
                lat.append((time.perf_counter() - t0) * 1e6)
        out[f"ticket_{name}"] = {"submit_to_done_us_p50": round(float(np.percentile(lat, 50)), 2),
                                 "submit_to_done_us_p99": round(float(np.percentile(lat, 99)), 2)}
    ok = torch.equal(d, plain)  # an even number of launches in every form
    ctx.encrypt_pages(table)
    ctx.sync_checked()
    changed = int((d.view(n, PAGE) != plain.view(n, PAGE)).any(dim=1).sum())
    ctx.shutdown()
    print(json.dumps({
        "metric": "latency of one launch (256 pages, encrypt or decrypt)",
        "value": out["device_list"]["device_us_p50"], "unit": "us", "higher_is_better": False,
        "config": {"workload": "small: 256 pages x 4 KiB of SplitMix64(seed 0), ids 0..255, key SplitMix64(seed 1)",
                   "pages": n, "launches_per_form": 2 * args.steps},
        "forms": out, "round_trip_ok": ok, "pages_changed_by_one_encrypt": changed,
    }), flush=True)


def run_batching(args):
    """20,000 Zipf(1.2) requests (1..512 pages, seed 3) scattered over an 8 GiB
    device buffer: one launch per request vs the persistent batched form."""
    print(json.dumps(batching_result(args, args.batch_requests, args.feed_chunks)), flush=True)


def batching_result(args, batch_requests, feed_chunks):
    """The batching workload through one launch per request, graph-launched
    batched submits (one row per entry of batch_requests) and the fed form
    (one row per publication size in feed_chunks); every form's 8 GiB result
    is compared with the one-launch-per-request buffer."""
    import numpy as np
    import torch

    import synth
    from paper_2004_09252_b300 import memshield as ms

    n_slots = int(2097152 * args.batching_scale)
    sizes, slots, ops = synth.batching_workload(3, n_requests=int(20000 * args.batching_scale), n_slots=n_slots)
    n_req, total = len(sizes), int(sizes.sum())
    key = synth.key_bytes(1)
    a = torch.empty(n_slots * PAGE, dtype=torch.uint8, device="cuda")
    fill_device_pages(a, 3, n_slots)
    plain = a.clone()
    b = a.clone()
    stream = torch.cuda.current_stream()
    ctx = ms.Context(key, stream=stream)
    tune = None if args.no_autotune else ctx.autotune(65536)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    sl = slots.astype(np.uint64)
    table_a = ms.pages_array(a.data_ptr() + PAGE * sl, sl)
    table_b = ms.pages_array(b.data_ptr() + PAGE * sl, sl)
    lib, h = ms.lib, ctx.handle

    # one launch per request (host list -> staging -> K1), direct ctypes calls
    ptrs = [table_b.ctypes.data + 16 * int(o) for o in offsets[:-1]]
    szs = [int(x) for x in sizes]
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ev0.record(stream)
    for r in range(n_req):
        rc = lib.ms_encrypt_pages(h, ptrs[r], szs[r])
        if rc:
            raise RuntimeError(ms.strerror(rc))
    ev1.record(stream)
    if ctx.sync():
        raise RuntimeError("sync failed")
    t_single = time.perf_counter() - t0
    span_single = ev0.elapsed_time(ev1)

    results = []
    applied = 0
    for breq in batch_requests:
        # a fixed number of requests per submit, or "rA-B": A requests first,
        # doubling on every submit up to B (the first kernel starts sooner, and
        # each fill still overlaps the previous submit's kernel)
        if isinstance(breq, str):
            size, cap = (int(x) for x in breq[1:].split("-"))
        else:
            size = cap = breq
        with ctx.batch(capacity=max(1 << 16, int(total))) as bt:
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            ev0.record(stream)
            first, step = 0, size
            while first < n_req:
                rc, added = bt.add_requests(ops, offsets, table_a, first, min(step, n_req - first))
                first += added
                bt.submit()
                step = min(cap, 2 * step)
            ev1.record(stream)
            if ctx.sync():
                raise RuntimeError("sync failed")
            el = time.perf_counter() - t0
            st = bt.stats()
        applied += 1
        ok = torch.equal(a, b) if applied % 2 == 1 else torch.equal(a, plain)
        results.append({"requests_per_submit": breq, "submits": st["submits"], "graph_launches": st["graph_launches"],
                        "wall_s": round(el, 5), "pages_per_s": round(total / el, 1),
                        "gb_per_s": round(total * PAGE / el / 1e9, 2),
                        "gpu_span_ms": round(ev0.elapsed_time(ev1), 3), "identical_to_one_launch_per_request": ok})
    # the fed form: one persistent kernel drains the queue while the host is still filling it;
    # one untimed run first (the first run in a process pays one-time host costs)
    if feed_chunks:
        with ctx.feed(capacity=int(total), chunk=feed_chunks[0]) as fd:
            fd.open()
            fd.add_requests(ops, offsets, table_a)
            fd.close()
            if ctx.sync():
                raise RuntimeError("sync failed")
        applied += 1
    for chunk in feed_chunks:
        with ctx.feed(capacity=int(total), chunk=chunk) as fd:   # allocation outside the timed span
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            ev0.record(stream)
            fd.open()
            first = 0
            while first < n_req:
                first += fd.add_requests(ops, offsets, table_a, first, min(2000, n_req - first))
            fd.close()
            ev1.record(stream)
            if ctx.sync():
                raise RuntimeError("sync failed")
            el = time.perf_counter() - t0
            st = fd.stats()
        applied += 1
        ok = torch.equal(a, b) if applied % 2 == 1 else torch.equal(a, plain)
        results.append({"requests_per_submit": f"fed, chunk {chunk}", "submits": 1, "graph_launches": 0,
                        "publications": st["publications"], "wall_s": round(el, 5),
                        "pages_per_s": round(total / el, 1), "gb_per_s": round(total * PAGE / el / 1e9, 2),
                        "gpu_span_ms": round(ev0.elapsed_time(ev1), 3), "identical_to_one_launch_per_request": ok})
    ctx.shutdown()
    del a, b, plain
    torch.cuda.empty_cache()
    best = max(results, key=lambda r: r["pages_per_s"])
    single = total / t_single
    return {
        "metric": "batching pages/s (persistent kernel over a device work queue, autotuned: best of graph-launched "
                  "submits and the fed form)",
        "value": best["pages_per_s"], "unit": "pages/s", "higher_is_better": True, "best_form": best["requests_per_submit"],
        "config": {"workload": (f"batching: {n_req} requests, Zipf(1.2) sizes 1..512 (mean 44.08), {total} pages "
                                f"scattered without replacement over a {n_slots * PAGE / 2**30:g} GiB buffer "
                                f"({n_slots} slots), seed 3, ops 50/50 enc/dec"
                                + ("" if args.batching_scale == 1.0 else " (profiling case)")),
                   "pages": total, "requests": n_req},
        "one_launch_per_request": {"wall_s": round(t_single, 5), "pages_per_s": round(single, 1),
                                   "gb_per_s": round(total * PAGE / t_single / 1e9, 2), "launches": n_req,
                                   "gpu_span_ms": round(span_single, 3)},
        "speedup_vs_one_launch_per_request": round(best["pages_per_s"] / single, 2),
        "batched": results, "autotune": tune,
    }


# ---------------------------------------------------- host pages (config 4)
def run_host(args):
    """4 GiB pinned host buffer (seed 4) streamed through the cipher in 2..64 MiB
    chunks on 2 streams; against the measured host-link bandwidth."""
    print(json.dumps(host_result(args, args.chunks_mib)), flush=True)


def host_link(hbuf, probe=1 << 30, reps=5):
    """Pinned host-link rates (GB/s): host->device alone, device->host alone, and
    each direction while both run at once (torch copies = cudaMemcpyAsync)."""
    import torch
    probe = min(probe, hbuf.numel())
    dsrc = torch.empty(probe, dtype=torch.uint8, device="cuda")
    ddst = torch.empty(probe, dtype=torch.uint8, device="cuda")
    hin = hbuf[:probe]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    scratch = torch.empty(probe, dtype=torch.uint8).pin_memory()
    h2d = probe / timed(lambda: ddst.copy_(hin, non_blocking=True)) / 1e9
    d2h = probe / timed(lambda: scratch.copy_(dsrc, non_blocking=True)) / 1e9

    def both():
        with torch.cuda.stream(s1):
            ddst.copy_(hin, non_blocking=True)
        with torch.cuda.stream(s2):
            scratch.copy_(dsrc, non_blocking=True)
    bidir_each = probe / timed(both) / 1e9
    del dsrc, ddst, scratch
    return {"h2d_gbs": round(h2d, 2), "d2h_gbs": round(d2h, 2), "bidirectional_each_gbs": round(bidir_each, 2),
            "bound_gbs": round(min(bidir_each, h2d, d2h), 2),
            "note": "the path moves every page both ways, so its bound is the slower direction while both run"}


def in_place_result(ms, ctx, hbuf, n, steps, head, link, world=1, device=None, barrier=lambda: None):
    """ms_crypt_host_inplace over the whole buffer: `steps` encrypt + decrypt
    passes, host wall time from the first call to the final sync (max over
    ranks when `device` is given)."""
    ctx.crypt_host_inplace(ms.MS_ENCRYPT, hbuf, 0, n)
    ctx.crypt_host_inplace(ms.MS_DECRYPT, hbuf, 0, n)
    ctx.sync_checked()
    barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        ctx.crypt_host_inplace(ms.MS_ENCRYPT, hbuf, 0, n)
        ctx.crypt_host_inplace(ms.MS_DECRYPT, hbuf, 0, n)
    ctx.sync_checked()
    barrier()
    el_ms = (time.perf_counter() - t0) * 1e3
    if device is not None:
        el_ms, gbs = aggregate_replicas(el_ms, 2.0 * steps * n * PAGE, world, device)
    else:
        gbs = 2.0 * steps * n * PAGE / (el_ms * 1e-3) / 1e9
    import torch
    return {"value": round(gbs, 3), "unit": "GB/s", "entry": "ms_crypt_host_inplace", "steps": steps,
            "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
            "link_bytes_per_step_each_way": 2 * n * PAGE,
            "round_trip_ok": bool(torch.equal(hbuf[:PAGE * 64], head)),
            "frac_of_link": round(gbs / world / link["bound_gbs"], 3)}


def host_result(args, chunks_mib):
    """The host-page workload through ms_crypt_host at each chunk size, against
    the measured host link."""
    import torch

    import synth
    from paper_2004_09252_b300 import memshield as ms

    n = 1048576
    key = synth.key_bytes(1)
    hbuf = torch.empty(n * PAGE, dtype=torch.uint8).pin_memory()
    synth.fill_pages(hbuf.data_ptr(), 4, 0, n)
    head = hbuf[:PAGE * 64].clone()
    link = host_link(hbuf)
    link_bound = link["bound_gbs"]

    ctx = ms.Context(key, stream=torch.cuda.current_stream())
    rows = []
    for mib in chunks_mib:
        for ns in (2,) if mib != 16 else (2, 3, 4):
            ctx.crypt_host(ms.MS_ENCRYPT, hbuf, 0, n, mib << 20, ns)       # warm + leaves data encrypted
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.crypt_host(ms.MS_DECRYPT, hbuf, 0, n, mib << 20, ns)
            el = time.perf_counter() - t0
            rows.append({"chunk_mib": mib, "streams": ns, "gb_per_s": round(n * PAGE / el / 1e9, 2),
                         "frac_of_link": round(n * PAGE / el / 1e9 / link_bound, 3)})
    ok = torch.equal(hbuf[:PAGE * 64], head)
    in_place = in_place_result(ms, ctx, hbuf, n, 3, head, link)
    # the one-launch page kernel on the same pinned pages through their device
    # view (ms_crypt_range): a grid of one thread per 4 keystream blocks, the
    # shape that suits HBM, against the bounded grid of ms_crypt_host_inplace
    dev = ms.host_device_address(hbuf)
    t0 = time.perf_counter()
    ctx.crypt_range(ms.MS_ENCRYPT, dev, 0, n)
    ctx.crypt_range(ms.MS_DECRYPT, dev, 0, n)
    ctx.sync_checked()
    el = time.perf_counter() - t0
    in_place["full_grid_one_launch"] = {"value": round(2 * n * PAGE / el / 1e9, 3), "unit": "GB/s",
                                        "entry": "ms_crypt_range on the device view",
                                        "round_trip_ok": bool(torch.equal(hbuf[:PAGE * 64], head))}
    ctx.shutdown()
    best = max(rows, key=lambda r: r["gb_per_s"])
    return {
        "metric": "end-to-end host page GB/s (H2D + cipher + D2H)", "value": best["gb_per_s"], "unit": "GB/s",
        "higher_is_better": True,
        "config": {"workload": "host pages: 4 GiB pinned host buffer (1,048,576 pages, seed 4), ms_crypt_host, "
                               "chunks 2..64 MiB, 2..4 streams", "pages": n},
        "link": link, "frac_of_link": round(best["gb_per_s"] / link_bound, 3), "sweep": rows,
        "round_trip_ok": ok, "in_place": in_place,
    }


# ------------------------------------------------------- serving (config 5)
SERVE_RATES = [1e4, 3.76e4, 1.41e5, 5.32e5, 2e6]


def run_serving(args):
    """Poisson arrivals at 5 page rates; 80 % 1-page decrypts, 20 % 8..64-page
    encrypts over a 16 GiB pinned host working set (seed 5); 256 MiB staging
    budget; continuous batching vs one launch per request."""
    rows, setup_s = serve_rows(args, args.serve_rates, args.serve_modes, args.serve_seconds)
    n = args.serve_pages
    head = "continuous" if "continuous" in args.serve_modes else args.serve_modes[0]
    cont = [r for r in rows if r["mode"] == head]
    one = {r["offered_pages_per_s"]: r for r in rows if r["mode"] == "one_per_launch"}
    if not one:
        one = {r["offered_pages_per_s"]: r for r in cont}
    top = cont[-1]
    print(json.dumps({
        "metric": f"served pages/s and p50/p99 request latency ({head})",
        "value": top["sustained_pages_per_s"], "unit": "pages/s", "higher_is_better": True,
        "config": {"workload": SERVE_WORKLOAD.format(n=n, gib=n * PAGE / 2**30, sec=args.serve_seconds),
                   "rates_pages_per_s": args.serve_rates, "copy_threads": args.copy_threads,
                   "working_set_setup_s": round(setup_s, 1)},
        "p50_us": top["p50_us"], "p99_us": top["p99_us"], "p999_us": top["p999_us"],
        "vs_one_per_launch": [{"offered": r["offered_pages_per_s"],
                               "sustained_ratio": round(r["sustained_pages_per_s"] /
                                                        one[r["offered_pages_per_s"]]["sustained_pages_per_s"], 3),
                               "p99_ratio": round(one[r["offered_pages_per_s"]]["p99_us"] / r["p99_us"], 3)}
                              for r in cont],
        "rows": rows,
    }), flush=True)


SERVE_WORKLOAD = ("serving: {n} pages ({gib:.0f} GiB) pinned host working set (seed 5), Poisson arrivals, 80 % "
                  "1-page decrypts / 20 % U{{8..64}}-page encrypts, 256 MiB staging budget, {sec:g} s per rate")


def resident_multi(args, ms, ctx, ws, n, rate, seconds):
    """The resident form fed by several client threads at once: thread t owns
    pages [t*n/T, (t+1)*n/T) of the working set, its own resident worker set
    (args.resident_workers each) and its own serving workload (seed 5 + t) at
    rate / T.  Returns (all latencies, the longest makespan, pages)."""
    import threading

    import numpy as np

    import synth
    T = args.resident_submitters
    part = n // T
    loads = []
    for t in range(T):
        n_req = max(2000, int(rate / T / 8.0 * seconds))
        arr, _, offs, pages = synth.serving_workload(5 + t, n_req, rate / T, part)
        loads.append((arr, offs, pages.astype(np.uint64) + np.uint64(t * part)))
    res = [ms.Resident(ctx, workers=args.resident_workers) for _ in range(T)]
    out, errors = [None] * T, []

    def client(t):
        try:
            arr, offs, pages = loads[t]
            out[t] = res[t].replay(ws, n, arr, offs, pages, timeout_ms=60000)
        except Exception as e:  # surfaced below
            errors.append(e)
    threads = [threading.Thread(target=client, args=(t,)) for t in range(T)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    for r in res:
        r.destroy()
    if errors:
        raise errors[0]
    lat = np.concatenate([out[t][0] for t in range(T)])
    return lat, max(out[t][1] for t in range(T)), sum(int(loads[t][1][-1]) for t in range(T))


def latency_split(arrival, lat):
    """p50 / p99 / p99.9 (us) of the requests scheduled in the first second of a
    run, and of the rest (the steady state; None when the run is shorter)."""
    import numpy as np
    us = lat * 1e6
    out = {}
    for name, sel in (("first_second", arrival < 1.0), ("steady", arrival >= 1.0)):
        if not sel.any():
            out[name] = None
            continue
        v = us[sel]
        out[name] = {"requests": int(sel.sum()), "p50_us": round(float(np.percentile(v, 50)), 1),
                     "p99_us": round(float(np.percentile(v, 99)), 1),
                     "p999_us": round(float(np.percentile(v, 99.9)), 1)}
    return out


def serve_rows(args, rates, modes, seconds, one_per_launch_cap=None, reps_below=None):
    """Replay the serving workload at each rate in each mode; one row per (rate, mode).
    Each run covers `seconds` of arrivals; one_per_launch_cap (requests) bounds
    the one-launch-per-request runs, which saturate far below the top rates.
    reps_below = (rate, k): rates under `rate` run k times (medians reported),
    where a single spoiled second weighs most."""
    import numpy as np
    import torch

    import synth
    from paper_2004_09252_b300 import memshield as ms

    n = args.serve_pages
    key = synth.key_bytes(1)
    t0 = time.perf_counter()
    ws = torch.empty(n * PAGE, dtype=torch.uint8).pin_memory()
    synth.fill_pages(ws.data_ptr(), 5, 0, n)
    setup_s = time.perf_counter() - t0
    ctx = ms.Context(key)
    ctx.autotune(65536)
    rows = []
    mode_ids = {"continuous": ms.MS_SERVE_CONTINUOUS, "one_per_launch": ms.MS_SERVE_ONE_PER_LAUNCH,
                "zero_copy": ms.MS_SERVE_ZERO_COPY}
    for rate in rates:
        n_full = max(2000, int(rate / 8.0 * seconds))
        w_arrival, w_ops, w_offsets, w_pages = synth.serving_workload(5, n_full, rate, n)
        warm = None
        if args.serve_warmup_s > 0:   # a separate stream of requests (seed 55) at the same rate
            warm = synth.serving_workload(55, max(200, int(rate / 8.0 * args.serve_warmup_s)), rate, n)
        for name in modes:
            n_req = n_full
            if name == "one_per_launch" and one_per_launch_cap:
                n_req = min(n_req, one_per_launch_cap)
            arrival, ops = w_arrival[:n_req], w_ops[:n_req]
            offsets = w_offsets[:n_req + 1]
            pages = w_pages[:int(offsets[-1])]
            reps = []
            n_reps = max(1, args.serve_reps)
            if reps_below and rate < reps_below[0]:
                n_reps = max(n_reps, reps_below[1])
            for _ in range(n_reps):
                if name == "resident" and args.resident_submitters > 1:
                    lat, makespan, total_mt = resident_multi(args, ms, ctx, ws, n, rate, seconds)
                    st = {"waves": total_mt, "max_wave_requests": 1, "conflict_waits": 0, "budget_waits": 0,
                          "gather_ns": 0, "scatter_ns": 0}
                elif name == "resident":
                    with ms.Resident(ctx, workers=args.resident_workers) as res:
                        if warm is not None:
                            res.replay(ws, n, warm[0], warm[2], warm[3], timeout_ms=60000)
                        lat, makespan = res.replay(ws, n, arrival, offsets, pages, timeout_ms=60000)
                        rst = res.stats()
                    st = {"waves": rst["requests"], "max_wave_requests": 1, "conflict_waits": 0, "budget_waits": 0,
                          "gather_ns": 0, "scatter_ns": 0, "submit_lag_ms": round(rst["replay_max_lag_ns"] * 1e-6, 3)}
                else:
                    with ms.Server(ctx, ws, n, mode=mode_ids[name], copy_threads=args.copy_threads,
                                   waves_in_flight=args.waves_in_flight, idle_spin_us=args.idle_spin_us,
                                   max_wave_pages=args.max_wave_pages,
                                   zero_copy_max_pages=args.zero_copy_max_pages) as srv:
                        if warm is not None:
                            srv.replay(warm[0], warm[1], warm[2], warm[3], timeout_ms=600000)
                        st0 = srv.stats()
                        lat, makespan = srv.replay(arrival, ops, offsets, pages, timeout_ms=600000)
                        st = srv.stats()
                        for k in ("waves", "conflict_waits", "budget_waits", "gather_ns", "scatter_ns"):
                            st[k] -= st0[k]
                        st["submit_lag_ms"] = round(st["replay_max_lag_ns"] * 1e-6, 3)
                        st["server_pass_ms"] = round(st["max_pass_ns"] * 1e-6, 3)
                multi = name == "resident" and args.resident_submitters > 1
                total = st["waves"] if multi else int(offsets[-1])
                us = lat * 1e6
                # p99 of the requests scheduled in each second of the run (single-submitter runs)
                by_sec = []
                split = None
                if not multi:
                    sec = np.floor(arrival).astype(np.int64)
                    by_sec = [round(float(np.percentile(us[sec == k], 99)), 1) for k in range(int(sec.max()) + 1)
                              if (sec == k).any()]
                    split = latency_split(arrival, lat)
                reps.append({"sustained_pages_per_s": total / makespan, "p50_us": float(np.percentile(us, 50)),
                             "p99_us": float(np.percentile(us, 99)), "p999_us": float(np.percentile(us, 99.9)),
                             "by_sec": by_sec, "split": split, "st": st})
            # medians over the repetitions (single-run tails are noisy on a shared host)
            med = {k: float(np.median([r[k] for r in reps])) for k in ("sustained_pages_per_s", "p50_us", "p99_us",
                                                                      "p999_us")}
            mid = reps[len(reps) // 2]
            st = mid["st"]

            def split_median(part):  # each latency figure of a part: the median over the repetitions
                vals = [r["split"][part] for r in reps if r["split"] and r["split"][part]]
                if not vals:
                    return None
                return {k: (vals[0][k] if k == "requests" else round(float(np.median([v[k] for v in vals])), 1))
                        for k in vals[0]}
            rows.append({"offered_pages_per_s": rate, "mode": name, "requests": n_req, "pages": total,
                         "arrival_s": round(float(arrival[-1]), 2),
                         "sustained_pages_per_s": round(med["sustained_pages_per_s"], 1),
                         "p50_us": round(med["p50_us"], 1), "p99_us": round(med["p99_us"], 1),
                         "p999_us": round(med["p999_us"], 1), "reps": len(reps),
                         "first_second": split_median("first_second"), "steady": split_median("steady"),
                         "p99_us_each": [round(r["p99_us"], 1) for r in reps],
                         "p99_us_by_second": [r["by_sec"] for r in reps],
                         "max_submit_lag_ms": [r["st"].get("submit_lag_ms") for r in reps],
                         "late_submissions": [r["st"].get("replay_late") for r in reps],
                         "max_server_pass_ms": [r["st"].get("server_pass_ms") for r in reps],
                         "waves": st["waves"], "max_wave_requests": st["max_wave_requests"],
                         "conflict_waits": st["conflict_waits"], "budget_waits": st["budget_waits"],
                         "gather_s": round(st["gather_ns"] * 1e-9, 3), "scatter_s": round(st["scatter_ns"] * 1e-9, 3)})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    ctx.shutdown()
    del ws
    return rows, setup_s


# ------------------------------------------- sliding-window clients (NEXT)
def run_window(args):
    """Clients fault through FIFO windows of clear pages (Sec. 4.3), as in the
    paper's Table 1 (window 4..32 pages) and Table 2 (1, 2, 4 instances), under
    three eviction policies: the paper's (each eviction finished before the
    next fault), asynchronous evictions, and background eviction (the paper's
    proposed improvement)."""
    import numpy as np
    import torch

    import synth
    from paper_2004_09252_b300 import memshield as ms

    per = args.window_client_pages
    max_clients = max(args.window_clients)
    n = per * max_clients
    key = synth.key_bytes(1)
    ws = torch.empty(n * PAGE, dtype=torch.uint8).pin_memory()
    synth.fill_pages(ws.data_ptr(), 6, 0, n)
    ctx = ms.Context(key)
    rows = []
    srv = ms.Server(ctx, ws, n)
    res = ms.Resident(ctx, workers=args.resident_workers) if "resident" in args.window_backends else None
    try:
        for c in range(max_clients):           # client pages start encrypted with the client's PID
            for p0 in range(c * per, (c + 1) * per, 4096):
                srv.wait(srv.submit(ms.MS_ENCRYPT, np.arange(p0, min(p0 + 4096, (c + 1) * per)), domain=1000 + c),
                         20000)
        traces = [synth.window_trace(200 + c, per, args.window_trace) for c in range(max_clients)]
        state = {}
        for backend in args.window_backends:
            for n_cl in args.window_clients:
                for wnd in args.window_sizes:
                    for batch in args.window_batches:
                        for policy in args.window_policies:
                            # sync: the client waits for its own evictions (the paper's server);
                            # async: it does not; background: an evictor keeps window_free slots free
                            free = args.window_free if policy == "background" else 0
                            if batch > wnd + 1 or free >= wnd:
                                continue
                            # clients resume from where the previous run left their windows: re-encrypt them first
                            for c, win in state.items():
                                if win:
                                    srv.wait(srv.submit(ms.MS_ENCRYPT, np.array(win), domain=1000 + c), 20000)
                            state = {}
                            cl = [(1000 + c, c * per, per, traces[c]) for c in range(n_cl)]
                            t0 = time.perf_counter()
                            kw = dict(timeout_ms=20000, background_free=free, sync_evict=policy == "sync")
                            if backend == "ticketed":   # one clone of ctx per client: its PID, its stream
                                st, wins = ctx.run_window_clients(ws, n, wnd, batch, cl, **kw)
                            elif backend == "resident":
                                st, wins = res.run_window_clients(ws, n, wnd, batch, cl, **kw)
                            else:
                                st, wins = srv.run_window_clients(wnd, batch, cl, **kw)
                            el = time.perf_counter() - t0
                            state = {c: wins[c] for c in range(n_cl)}
                            faults = sum(x["faults"] for x in st)
                            rows.append({"backend": backend, "clients": n_cl, "window_pages": wnd,
                                         "evict_batch": batch, "policy": policy, "background_free": free,
                                         "accesses": sum(x["accesses"] for x in st), "faults": faults,
                                         "evictions": sum(x["evictions"] for x in st),
                                         "evict_requests": sum(x["evict_requests"] for x in st),
                                         "background_evictions": sum(x["background_evictions"] for x in st),
                                         "faults_per_s": round(faults / el, 1),
                                         "fault_p50_us": round(float(np.mean([x["fault_p50_us"] for x in st])), 1),
                                         "fault_p99_us": round(float(max(x["fault_p99_us"] for x in st)), 1),
                                         "client_s_max": round(max(x["elapsed_s"] for x in st), 3)})
                            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    finally:
        if res is not None:
            res.destroy()
        srv.destroy()
    ctx.shutdown()
    print(json.dumps({
        "metric": "sliding-window fault service (faults/s, fault latency)", "unit": "faults/s",
        "value": max(r["faults_per_s"] for r in rows), "higher_is_better": True,
        "config": {"workload": f"sliding-window clients: {per} pages per client (seed 6), trace of "
                               f"{args.window_trace} accesses per client (60 % Zipf(1.1) hot set, 40 % sequential "
                               "scan), each client its own PID domain", "client_pages": per},
        "rows": rows}), flush=True)


# ------------------------------------------------------------ pipe rates
def run_pipes(args):
    """Sustained rates of the cipher's 32-bit op classes (ms_probe_int_pipes),
    alone and in 1:1 mixes: the measurement behind the ALU-pipe roofline."""
    import torch

    from paper_2004_09252_b300 import memshield as ms
    dev = torch.cuda.current_device()
    rows = ms.probe_int_pipes(dev)
    props = torch.cuda.get_device_properties(dev)
    print(json.dumps({
        "metric": "int32 lane operations per SM per clock, by op class", "unit": "lanes/SM/clk",
        "value": next(r["lanes_per_sm_clk"] for r in rows if r["class"] == "xor"), "higher_is_better": True,
        "config": {"workload": "4 CTAs x 256 threads per SM, 8 independent chains x 16384 ops per thread",
                   "sms": props.multi_processor_count},
        "rows": rows}), flush=True)


# -------------------------------------------------------------- reference
def run_reference(args):
    """The reference arm: the CPU oracle, as it stands, on the host cores.  A
    step is one encrypt pass plus one decrypt pass over the whole 1 GiB bulk
    buffer when (steps + warmup) such steps fit in about 150 s on this host;
    otherwise over the largest prefix that does, and ``config.pages`` says
    which."""
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import numpy as np

    import oracle
    import synth
    oracle.build()
    threads = host_cores()
    key = synth.key_bytes(1)
    budget = 150.0
    # the first warm-up step runs on the whole buffer and sets the sample: the
    # whole buffer when the remaining steps fit in the budget, else a prefix
    npg = BULK_PAGES
    buf = synth.page_bytes_fast(2, 0, npg)
    ids = np.arange(npg, dtype=np.uint64)
    t0 = time.perf_counter()
    oracle.crypt_pages(key, buf, ids, ids, threads=threads)
    oracle.crypt_pages(key, buf, ids, ids, threads=threads)
    t_step = time.perf_counter() - t0
    left = args.steps + args.warmup - 1
    if left * t_step > budget:
        npg = max(threads * 4, int(BULK_PAGES * budget / (left * t_step)))
        buf = np.ascontiguousarray(buf[:npg * PAGE])
        ids = ids[:npg]
    for _ in range(args.warmup - 1):
        oracle.crypt_pages(key, buf, ids, ids, threads=threads)
        oracle.crypt_pages(key, buf, ids, ids, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.crypt_pages(key, buf, ids, ids, threads=threads)
        oracle.crypt_pages(key, buf, ids, ids, threads=threads)
    dt = time.perf_counter() - t0
    value = 2.0 * args.steps * npg * PAGE / dt / 1e9
    whole = npg == BULK_PAGES
    sample = (f"each step: encrypt + decrypt of {'all' if whole else 'the first'} {npg} pages "
              f"({npg * PAGE / 2**20:.1f} MiB) of the bulk buffer on {threads} threads")
    workload = WORKLOAD if whole else (f"bulk, first {npg} of 262,144 pages (the whole buffer does not fit the "
                                       f"reference arm's time budget on this host): " + WORKLOAD)
    print(json.dumps({
        "impl": "reference", "metric": "page encrypt GB/s (ChaCha20, 4 KiB pages, device-resident)",
        "value": round(value, 4), "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic (SplitMix64 seeded page bytes)",
        "config": {"workload": workload, "pages": npg, "page_bytes": PAGE, "rounds": 20,
                   "l2": "host memory", "parallelism": "cpu"},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--pages", type=int, default=BULK_PAGES,
                    help="pages in the buffer (default: the 1 GiB bulk workload; smaller only for profiling)")
    ap.add_argument("--shape", default="", help="K1 shape override: bpt,tpc,unroll,rot_policy[,hoist]")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving summary in the bulk line")
    ap.add_argument("--no-batching", action="store_true", help="skip the batching summary in the bulk line")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--e2e-chunk-mib", type=int, default=16)
    ap.add_argument("--e2e-pages", type=int, default=1048576, help="host-page e2e buffer (default 4 GiB)")
    ap.add_argument("--e2e-streams", type=int, default=2)
    ap.add_argument("--workload", choices=["bulk", "small", "batching", "host", "serving", "window", "pipes"],
                    default="bulk",
                    help="bulk (default, the contract line); batching / host / serving print their own line")
    ap.add_argument("--serve-pages", type=int, default=4194304, help="working-set pages (default 16 GiB)")
    ap.add_argument("--serve-rates", type=lambda v: [float(x) for x in v.split(",")], default=SERVE_RATES)
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    ap.add_argument("--serve-warmup-s", type=float, default=0.3,
                    help="serving: replay this many seconds of a separate request stream (seed 55) at the same "
                         "rate, untimed, before each measured run")
    ap.add_argument("--low-rate-reps", type=int, default=3,
                    help="default line: repetitions of the rates under 100k pages/s (medians reported)")
    ap.add_argument("--one-per-launch-cap", type=int, default=50000,
                    help="serving: requests per one-launch-per-request run at most (it saturates near 270k pages/s)")
    ap.add_argument("--copy-threads", type=int, default=8)
    ap.add_argument("--serve-reps", type=int, default=1, help="repetitions per serving configuration (medians reported)")
    ap.add_argument("--resident-workers", type=int, default=8)
    ap.add_argument("--resident-submitters", type=int, default=1,
                    help="serving, resident mode: client threads, each with its own worker set and page range")
    ap.add_argument("--batching-scale", type=float, default=1.0, help="fraction of the batching workload (profiling)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--window-client-pages", type=int, default=16384)
    ap.add_argument("--window-trace", type=int, default=50000)
    ap.add_argument("--window-clients", type=lambda v: [int(x) for x in v.split(",")], default=[1, 2, 4])
    ap.add_argument("--window-sizes", type=lambda v: [int(x) for x in v.split(",")], default=[4, 8, 16, 32])
    ap.add_argument("--window-batches", type=lambda v: [int(x) for x in v.split(",")], default=[1, 8])
    ap.add_argument("--window-policies", type=lambda v: v.split(","), default=["sync", "async", "background"],
                    help="eviction policies: sync (the client waits for its evictions, as the paper's server), "
                         "async (it does not), background (an evictor keeps --window-free slots free)")
    ap.add_argument("--window-free", type=int, default=1,
                    help="background eviction threshold: free window slots the evictor keeps")
    ap.add_argument("--window-backends", type=lambda v: v.split(","), default=["server", "resident", "ticketed"],
                    help="serve the window clients through the continuous server, resident workers and/or "
                         "ticketed launches")
    ap.add_argument("--waves-in-flight", type=int, default=0, help="serving pipeline depth (0 = library default)")
    ap.add_argument("--max-wave-pages", type=int, default=0, help="serving wave size cap (0 = library default)")
    ap.add_argument("--zero-copy-max-pages", type=int, default=None,
                    help="continuous serving: waves up to this many pages run in place (default: library's)")
    ap.add_argument("--idle-spin-us", type=int, default=None, help="serving idle poll window (default: library's)")
    ap.add_argument("--serve-modes", type=lambda v: v.split(","), default=["continuous", "one_per_launch"])
    ap.add_argument("--batch-requests", type=lambda v: [x if x.startswith("r") else int(x) for x in v.split(",")],
                    default=[1, 16, 256, 2000, 20000, "r60-4000"],
                    help="requests per submit; rA-B = A first, doubling per submit up to B")
    ap.add_argument("--feed-chunks", type=lambda v: [int(x) for x in v.split(",") if x], default=[16384],
                    help="batching: also run the fed form with these publication sizes (entries)")
    ap.add_argument("--chunks-mib", type=lambda v: [int(x) for x in v.split(",")], default=[2, 4, 8, 16, 32, 64])
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "small":
        run_small(args)
    elif args.workload == "pipes":
        run_pipes(args)
    elif args.workload == "batching":
        run_batching(args)
    elif args.workload == "host":
        run_host(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "window":
        run_window(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
