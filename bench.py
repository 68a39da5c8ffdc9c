"""Benchmark of the GB300 positional population count.

Default workload (the large-array sweep, one GPU): an 8 GiB array of
Bernoulli(0.5) bits (seed 0) resident in HBM; one step counts it for
w = 8, 16, 32 and 64 (four launches of the single-array kernel).  The value
is input GB/s over the timed steps (device time, CUDA events), and the line
also carries:

* per_w: GB/s and fraction of measured HBM peak for each w;
* roofline: the counting kernel's achieved GB/s per launch against the
  measured HBM peak, plus the DRAM traffic per launch from the committed
  ncu summary (null when the kernel source changed since it was taken);
* read_roofline: the roofline read kernels (Section 5's "dummy" kernel,
  direct loads and cp.async.bulk staging) on the same array;
* e2e: the same metric through the host-memory entry point (pinned host
  input, every step's input crosses the CPU-GPU link, counts read back);
* batched: the ragged one-hot batch (200000 uint8 arrays, log-uniform
  1 B .. 4 MiB, about 55 GB), one batched call vs one launch per array;
* plain: the 1 MiB w = 16 configuration, GPU microseconds per call and
  the oracle's time;
* short: microseconds per call for short unaligned arrays, one launch each,
  plain and graph-replayed;
* multi: several counts in one launch (pospopcnt_multi): the plain
  configuration queued 16 counts a launch, and four 1 GiB arrays in one
  launch against four single launches;
* sizes: one count of 1 MiB, 16 MiB, 128 MiB and 1 GiB, launched back to
  back and alone, against the same count as a one-entry multi launch and
  the roofline read kernel (the fixed cost of a launch);
* serving: the continuous-batching server on Poisson request streams at
  0.3 / 0.6 / 0.9 of the large-array rate, GB/s and p50/p99 latency;
* masked: the WHERE-selected count on the 8 GiB array as 32-bit words;
* gather: 100000 separate regions of the array into one counter array;
* counts_ok: the timed counts of every w checked against the CPU oracle's
  count of the whole 8 GiB array (host copy, all host cores), outside the
  timed region;
* cpu_baseline: the CPU oracle on the host cores on a bounded sample;
* sweep: every w at 1 GiB and 8 GiB over Bernoulli(0.01/0.5/0.99) and
  all-ones bits, each cell's counts checked;
* tuned (only with --sections tuned): the autotuner's table against the
  shipped one on the batch, single counts and the serving trace;
* clocks: SM clocks and throttle reasons sampled during the timed region.

``--impl reference`` times the CPU oracle on the same workload instead.
Under torchrun each rank runs an independent replica (weak scaling);
``--shard`` instead splits the one 8 GiB array into per-rank shards (64-byte
boundaries), each rank counts its shard and one all-reduce of the counters
per step completes the count (strong scaling).
"""
from __future__ import annotations

import argparse
import contextlib
import hashlib
import json
import os
import platform
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GIB = 1 << 30
WIDTHS = (8, 16, 32, 64)
METRIC = "pospopcnt input GB/s and % of HBM peak per w; batched vs per-array; p99 us"
WORKLOAD = ("large-array sweep: 8 GiB array of Bernoulli(0.5) bits (seed 0) resident in HBM, "
            "w in {8,16,32,64} per step")


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clocks/throttle sampling in the background (read-only)."""

    FIELDS = ("timestamp", "index", "clocks.sm", "clocks.max.sm", "power.draw",
              "clocks_event_reasons.active", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, period_ms: int = 50):
        self.samples = []
        self.proc = None
        self.index = index
        self.period_ms = period_ms
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self, t0: float, t1: float) -> dict:
        win = [s for (t, s) in self.samples if t0 - 0.06 <= t <= t1 + 0.06]
        if not win and self.samples:
            mid = 0.5 * (t0 + t1)
            win = [min(self.samples, key=lambda x: abs(x[0] - mid))[1]]
        if not win:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        sm = [float(s[2]) for s in win if s[2].replace(".", "").isdigit()]
        smax = [float(s[3]) for s in win if s[3].replace(".", "").isdigit()]
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for s in win:
            for name, val in zip(names, s[6:10]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(win)}


def _kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2412_16370_gb300", "csrc")
    for f in ("pospop_device.cuh", "pospop_stream.cu"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profile_traffic(nbytes: int):
    """DRAM bytes per launch of the counting kernel from the committed ncu summary."""
    import re
    path = os.path.join(ROOT, "profiles", "stream_kernel_1GiB_ncu_full.md")
    try:
        text = open(path).read()
    except OSError:
        return None, "no committed ncu summary"
    m1 = re.search(r"^traffic_per_input_byte:\s*([0-9.]+)", text, re.M)
    m2 = re.search(r"^kernel_source_sha256_16:\s*([0-9a-f]+)", text, re.M)
    if not (m1 and m2):
        return None, "ncu summary lacks the traffic line"
    if m2.group(1) != _kernel_source_hash():
        return None, "kernel changed since the ncu capture"
    return round(float(m1.group(1)) * nbytes), ("dram read+write of a 1 GiB launch (ncu) scaled "
                                                 "to this launch's input bytes")


def _oracle_counts(data_dev, widths, chunk: int = GIB):
    """The CPU oracle's counts of a device buffer (copied back in 1 GiB
    chunks, which start on word boundaries; all host cores), one array per w."""
    import torch
    import oracle
    orc = oracle.load()
    cores = os.cpu_count() or 1
    n = data_dev.numel()
    out = {w: np.zeros(w, dtype=np.uint64) for w in widths}
    host = torch.empty(min(chunk, n), dtype=torch.uint8, pin_memory=True)
    for c0 in range(0, n, chunk):
        h = host[:min(chunk, n - c0)]
        h.copy_(data_dev[c0:c0 + h.numel()])
        a = h.numpy()
        for w in widths:
            orc.bytes_mt(w, a, cores, counts=out[w])
    return out


def _verify_counts(counts, data, launches):
    """The timed counters hold `launches` counts of the array for each w:
    compare them with the oracle's count of the array."""
    t0 = time.perf_counter()
    exp = _oracle_counts(data, WIDTHS)
    got = counts.cpu().numpy().view(np.uint64)
    per_w = {str(w): bool(np.array_equal(got[k, :w], exp[w] * np.uint64(launches)))
             for k, w in enumerate(WIDTHS)}
    return {"all": all(per_w.values()), "per_w": per_w,
            "how": f"timed counters (each the sum of {launches} launches) == {launches} x the CPU "
                   "oracle's count of the whole array (Fig. 2 loop on the host copy, all cores), "
                   "checked after the timed region",
            "oracle_s": round(time.perf_counter() - t0, 1)}


def _cpu_baseline(data_dev, budget_s: float = 12.0, runs: int = 5, sample: int = GIB):
    """The oracle as it stands on a bounded sample of the array (its first
    `sample` bytes, the same sample size as the reference arm's default):
    all host cores and one thread, each the median of `runs` timed passes
    (every pass counts the sample once per w), with the spread of the runs."""
    import torch
    import oracle
    orc = oracle.load()
    cores = os.cpu_count() or 1
    sample = min(sample, data_dev.numel())
    sample -= sample % 64
    host = data_dev[:sample].cpu().numpy()
    orc.bytes_mt(16, host[:16 << 20], cores)          # warm-up
    t0 = time.perf_counter()
    orc.bytes_mt(16, host[:16 << 20], cores)
    rate = (16 << 20) / max(time.perf_counter() - t0, 1e-6)
    one = int(min(sample, max(1 << 20, rate / cores * budget_s / 5 / (runs * len(WIDTHS)))))
    one -= one % 64

    def timed(nbytes, threads):
        t1 = time.perf_counter()
        for w in WIDTHS:
            orc.bytes_mt(w, host[:nbytes], threads)
        return nbytes * len(WIDTHS) / (time.perf_counter() - t1) / 1e9

    all_runs = [timed(sample, cores) for _ in range(runs)]
    all_cores = float(np.median(all_runs))
    one_thread = float(np.median([timed(one, 1) for _ in range(runs)]))
    del torch
    return {"value": round(all_cores, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "runs_GBps": [round(x, 4) for x in all_runs],
            "one_thread_GBps": round(one_thread, 4),
            "cpu_model": _cpu_model(),
            "sample": f"first {sample >> 20} MiB of the 8 GiB array, counted once per w in "
                      f"{{8,16,32,64}} with {cores} threads, median of {runs} runs after a "
                      f"warm-up (Fig. 2 loop, -O2 -fno-tree-vectorize); one_thread_GBps: the "
                      f"first {one >> 20} MiB on one thread, median of {runs} runs"}


def _cpu_model():
    """The host CPU's model name, from lscpu (or /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2412_16370_gb300 import binding as pp
    from paper_2412_16370_gb300 import build as pkg_build
    from paper_2412_16370_gb300 import synth, synth_device

    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo",
                                device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    if rank == 0 or world == 1:
        pkg_build.build()
    if world > 1:
        dist.barrier()
    pp.init(local)
    peaks, peak_kind = _measured_peaks()
    hbm_peak = float(peaks["hbm_gbs"])

    total_bytes = args.gib * GIB
    if args.shard:
        # one array (seed 0) split across the ranks; each makes only its shard
        from paper_2412_16370_gb300 import shard
        lo, hi = shard.shard_range(total_bytes, rank, world)
        nbytes = hi - lo
        data = torch.empty(max(1, nbytes), dtype=torch.uint8, device=dev)[:nbytes]
        synth_device.bernoulli_(data, 0.5, seed=0, start=lo, nbytes=nbytes)
    else:
        # independent replicas: rank r counts its own array (seed r)
        nbytes = total_bytes
        data = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        synth_device.bernoulli_(data, 0.5, seed=0 + rank)
    counts = torch.zeros((len(WIDTHS), 64), dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()

    def step(ev=None):
        if args.shard:
            counts.zero_()
        for k, w in enumerate(WIDTHS):
            if ev is not None:
                ev[k][0].record(stream)
            pp.pospopcnt_async(w, counts[k], data, nbytes, stream)
            if ev is not None:
                ev[k][1].record(stream)
        if args.shard and world > 1:
            dist.all_reduce(counts, op=dist.ReduceOp.SUM)   # w x 8 bytes per width

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in WIDTHS]
           for _ in range(args.steps)]
    start_ev = torch.cuda.Event(enable_timing=True)
    end_ev = torch.cuda.Event(enable_timing=True)
    launches0 = pp.pospopcnt_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    start_ev.record(stream)
    for i in range(args.steps):
        step(evs[i])
    end_ev.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    if world > 1:
        dist.barrier()
    launches = pp.pospopcnt_launch_count() - launches0
    time.sleep(0.1)
    sampler.stop()
    clocks = sampler.summary(t0, t1)

    total_ms = start_ev.elapsed_time(end_ev)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_step = total_ms / args.steps
    bytes_step = nbytes * len(WIDTHS)
    job_bytes_step = (total_bytes if args.shard else world * nbytes) * len(WIDTHS)
    value = job_bytes_step * args.steps / (total_ms / 1e3) / 1e9

    per_w = {}
    launch_ms_all = []
    for k, w in enumerate(WIDTHS):
        ms = [evs[i][k][0].elapsed_time(evs[i][k][1]) for i in range(args.steps)]
        launch_ms_all += ms
        gbs = nbytes / (float(np.mean(ms)) / 1e3) / 1e9
        per_w[str(w)] = {"GBps": round(gbs, 1), "frac_of_hbm_peak": round(gbs / hbm_peak, 4),
                         "ms_per_launch": round(float(np.mean(ms)), 4)}
    avg_launch_ms = float(np.mean(launch_ms_all))
    achieved = nbytes / (avg_launch_ms / 1e3) / 1e9
    traffic, traffic_note = _profile_traffic(nbytes)

    # correctness of the timed counts: every w's counts add up to the same
    # total (the array's popcount), and each equals the oracle's count
    tot = counts.sum(dim=1).cpu().numpy()
    consistent = bool(np.all(tot == tot[0]))
    counts_ok = None
    if args.shard:
        # the all-reduced counters of the last step against the sum over the
        # ranks of the oracle's counts of each shard (additivity)
        exp = _oracle_counts(data, WIDTHS) if nbytes else {w: np.zeros(w, np.uint64)
                                                           for w in WIDTHS}
        e = torch.zeros((len(WIDTHS), 64), dtype=torch.int64, device=dev)
        for k, w in enumerate(WIDTHS):
            e[k, :w] = torch.from_numpy(exp[w].view(np.int64))
        if world > 1:
            dist.all_reduce(e, op=dist.ReduceOp.SUM)
        counts_ok = {"all": bool(torch.equal(e, counts)),
                     "how": "all-reduced counters of the last step == the sum over ranks of "
                            "the CPU oracle's count of each rank's shard"}
    # (the replicas' check against the oracle runs after every other section:
    # its seconds of all-core host work must not disturb their measurements)

    # roofline read kernel on the same array
    rsum = torch.zeros(1, dtype=torch.int64, device=dev)
    for _ in range(3):
        pp.pospopcnt_roofline_read(data, rsum, nbytes, stream)
    torch.cuda.synchronize()
    r0 = torch.cuda.Event(enable_timing=True)
    r1 = torch.cuda.Event(enable_timing=True)
    reps = 20
    r0.record(stream)
    for _ in range(reps):
        pp.pospopcnt_roofline_read(data, rsum, nbytes, stream)
    r1.record(stream)
    torch.cuda.synchronize()
    read_gbs = nbytes / (r0.elapsed_time(r1) / reps / 1e3) / 1e9
    # the same read with the bytes staged in shared memory by cp.async.bulk
    with _tune_entry(pp, "roofline", "roofline 256 2 1"):
        rsum.zero_()
        for _ in range(3):
            pp.pospopcnt_roofline_read(data, rsum, nbytes, stream)
        torch.cuda.synchronize()
        r0.record(stream)
        for _ in range(reps):
            pp.pospopcnt_roofline_read(data, rsum, nbytes, stream)
        r1.record(stream)
        torch.cuda.synchronize()
        bulk_gbs = nbytes / (r0.elapsed_time(r1) / reps / 1e3) / 1e9
        bulk_ok = pp.pospopcnt_batch_status(stream) == pp.POSPOP_OK

    tune_line = pp.pospopcnt_tune_describe().splitlines()[0]
    extra = {}
    sections = set(args.sections.split(",")) if args.sections else None
    want = (lambda k: sections is None or k in sections)
    if not args.quick and not args.shard:
        if want("e2e"):
            extra["e2e"] = _e2e(args, pp, data, nbytes, world, dist)
        if rank == 0:
            for key, fn in (("batched", lambda: _batched(pp, synth, synth_device, dev, stream,
                                                         achieved, hbm_peak, m=args.batched_m)),
                            ("plain", lambda: _plain(pp, synth_device, dev, stream)),
                            ("short", lambda: _short(pp, synth, synth_device, dev, stream)),
                            ("multi", lambda: _multi(pp, synth_device, data, nbytes, dev, stream,
                                                     hbm_peak)),
                            ("sizes", lambda: _sizes(pp, data, nbytes, stream, achieved)),
                            ("serving", lambda: _serving(pp, synth, data, nbytes, achieved, dev)),
                            ("masked", lambda: _masked(pp, synth_device, data, nbytes, dev,
                                                       stream, achieved, hbm_peak)),
                            ("gather", lambda: _gather(pp, synth, data, nbytes, dev, stream,
                                                       achieved, hbm_peak)),
                            ("cpu_baseline", lambda: _cpu_baseline(data)),
                            ("sweep", lambda: _sweep(pp, synth_device, data, nbytes, stream,
                                                     hbm_peak, 0 + rank)),
                            ("tuned", lambda: _tuned(pp, synth, synth_device, data, nbytes, dev,
                                                     stream, achieved))):
                if not want(key) or (key == "tuned" and sections is None):
                    continue   # (the autotuner comparison runs only when asked for)
                try:
                    extra[key] = fn()
                except Exception as e:  # report, keep the line
                    extra[key] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and not args.shard and not args.no_verify:
        counts_ok = _verify_counts(counts, data, args.warmup + args.steps)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    line = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4),
        "higher_is_better": True,
        "scaling": "strong" if args.shard else "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic (seeded SplitMix64 Bernoulli(0.5) bits, generated on the device)",
        "config": {"workload": WORKLOAD, "bytes_per_step_per_gpu": bytes_step,
                   "array_bytes": total_bytes, "widths": list(WIDTHS),
                   "l2": "inputs (8 GiB) far larger than L2 (126 MB): no flush between steps",
                   "parallelism": (f"shard x{world} (one array split at 64-byte boundaries, "
                                   "all-reduce of the counters per step)") if args.shard
                                  else f"replicas x{world}",
                   "tune": tune_line},
        "per_w": per_w,
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak,
                     "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
                     "traffic": traffic, "peak_kind": f"{peak_kind} hbm_gbs (copy, burst)",
                     "kernel": "pospop::stream_kernel (single-array count)",
                     "traffic_note": traffic_note},
        "read_roofline": {"GBps": round(read_gbs, 1), "frac_of_hbm_peak": round(read_gbs / hbm_peak, 4),
                          "kernel": "pospop::roofline_kernel (sum of the input)",
                          "bulk_staged_GBps": round(bulk_gbs, 1), "bulk_status_ok": bulk_ok,
                          "bulk_kernel": "pospop::roofline_bulk_kernel<8,3> (cp.async.bulk into "
                                         "shared memory, 3 x 8 KiB stages per warp)"},
        "gpu_launches": int(launches),
        "counts_consistent_across_w": consistent,
        "counts_ok": counts_ok,
        "clocks": clocks,
    }
    line.update(extra)
    if "e2e" not in line:
        line["e2e"] = None
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _e2e(args, pp, data, nbytes, world, dist):
    """Same metric through pospopcnt_host: pinned host input, counts read back to the host."""
    import torch
    host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    host.copy_(data)
    hc = np.zeros(64, dtype=np.uint64)
    steps = max(1, min(args.steps, args.e2e_steps))
    for w in WIDTHS:
        pp.pospopcnt_host(w, hc, host)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        for w in WIDTHS:
            pp.pospopcnt_host(w, hc, host)
    dt = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([dt], dtype=torch.float64, device=data.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dt = float(t.item())
    # the link's achievable read rate: the roofline read kernel on the same
    # pinned host buffer (device time)
    rsum = torch.zeros(1, dtype=torch.int64, device=data.device)
    stream = torch.cuda.current_stream()
    pp.pospopcnt_roofline_read(host, rsum, nbytes, stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pp.pospopcnt_roofline_read(host, rsum, nbytes, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    link_gbs = nbytes / (e0.elapsed_time(e1) / 1e3) / 1e9
    del host
    value = world * nbytes * len(WIDTHS) * steps / dt / 1e9
    return {"value": round(value, 2), "unit": "GB/s",
            "h2d_bytes_per_step": nbytes * len(WIDTHS),
            "d2h_bytes_per_step": 8 * sum(WIDTHS), "steps": steps,
            "path": "pospopcnt_host on pinned host memory (read in place over NVLink-C2C)",
            "link_read_roofline_GBps": round(link_gbs, 1),
            "frac_of_link_read": round(value / world / link_gbs, 4)}


def _batched(pp, synth, synth_device, dev, stream, large_gbs, hbm_peak, m=200000):
    import torch
    sizes = synth.log_uniform_sizes(m, 1, 4 << 20, seed=3)
    offs = synth.csr_offsets(sizes)
    total = int(offs[-1])
    base = torch.empty(total + 64, dtype=torch.uint8, device=dev)
    synth_device.one_hot_(base, 4, nbytes=total)
    offs_d = torch.from_numpy(offs.view(np.int64)).to(dev)
    c = torch.zeros((m, 8), dtype=torch.int64, device=dev)
    for _ in range(3):
        pp.pospopcnt_batch(8, c, base, offs_d, m, stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 10
    e0.record(stream)
    for _ in range(reps):
        pp.pospopcnt_batch(8, c, base, offs_d, m, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    ok = bool(np.array_equal(c.sum(dim=1).cpu().numpy(), (reps + 3) * sizes))
    # the same call captured once into a CUDA graph and replayed
    gs = torch.cuda.Stream()
    graph = pp.pospopcnt_batch_graph_create(8, c, base, offs_d, m, gs)
    try:
        for _ in range(3):
            pp.pospopcnt_graph_launch(graph, gs)
        gs.synchronize()
        e0.record(gs)
        for _ in range(reps):
            pp.pospopcnt_graph_launch(graph, gs)
        e1.record(gs)
        gs.synchronize()
        ms_graph = e0.elapsed_time(e1) / reps
    finally:
        pp.pospopcnt_graph_destroy(graph)
    # one launch per array
    c.zero_()
    basep = base.data_ptr()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record(stream)
    for a in range(m):
        if sizes[a]:
            pp.pospopcnt_async(8, c[a], basep + int(offs[a]), int(sizes[a]), stream)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms_per = e0.elapsed_time(e1)
    gbs = total / (ms / 1e3) / 1e9
    # the same batch with the other short-sequence method (per-lane bit
    # regroup vs warp transpose flush for items of <= 3 rows), for comparison
    import tempfile
    desc = pp.pospopcnt_tune_describe()
    cur = 1 if "\nshort 1" in desc else 0
    alt_text = desc.replace(f"short {cur}", f"short {1 - cur}")
    with tempfile.NamedTemporaryFile("w", suffix=".txt", delete=False) as f:
        f.write(desc)
        saved = f.name
    with tempfile.NamedTemporaryFile("w", suffix=".txt", delete=False) as f:
        f.write(alt_text)
        alt = f.name
    # a batch of only tiny arrays (every work item takes the short path)
    tsz = synth.log_uniform_sizes(m, 1, 1536, seed=71)
    toffs = synth.csr_offsets(tsz)
    toffs_d = torch.from_numpy(toffs.view(np.int64)).to(dev)

    def time_batch(offs_dev):
        for _ in range(3):
            pp.pospopcnt_batch(8, c, base, offs_dev, m, stream)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            pp.pospopcnt_batch(8, c, base, offs_dev, m, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_tiny = time_batch(toffs_d)
    pp.pospopcnt_tune_load(alt)
    ms_alt = time_batch(offs_d)
    ms_tiny_alt = time_batch(toffs_d)
    pp.pospopcnt_tune_load(saved)
    os.unlink(saved)
    os.unlink(alt)
    short_cmp = {"in_use": "regroup" if cur else "transpose",
                 "other": "transpose" if cur else "regroup",
                 "ragged_ms_in_use": round(ms, 3), "ragged_ms_other": round(ms_alt, 3),
                 "tiny_workload": f"{m} arrays of 1..1536 B (log-uniform), {int(toffs[-1])} bytes",
                 "tiny_ms_in_use": round(ms_tiny, 4), "tiny_ms_other": round(ms_tiny_alt, 4)}
    # the oracle on the first 2000 arrays, timed on the host cores
    import oracle
    orc = oracle.load()
    k = 2000
    sub_off = offs[:k + 1]
    sub = base[:int(sub_off[-1])].cpu().numpy()
    ora = _oracle_rate(lambda: orc.batch(8, sub, sub_off), lambda: sub.size)
    del base
    torch.cuda.empty_cache()
    return {"oracle_GBps": ora, "oracle_sample": f"first {k} arrays ({sub.size} bytes), 1 thread",
            "short_sequence_method": short_cmp,
            "workload": f"{m} one-hot uint8 arrays (Zipf(1.1) over 8 classes), sizes log-uniform "
                        "1 B..4 MiB, back to back (unaligned starts), w=8",
            "bytes": total, "GBps": round(gbs, 1), "ms": round(ms, 3),
            "graph_replay_ms": round(ms_graph, 3),
            "frac_of_large_array": round(gbs / large_gbs, 4),
            "frac_of_hbm_peak": round(gbs / hbm_peak, 4),
            "per_array_launches": {"GBps": round(total / (ms_per / 1e3) / 1e9, 1),
                                   "ms": round(ms_per, 1), "host_wall_s": round(wall, 2)},
            "speedup_vs_per_array": round(ms_per / ms, 1),
            "one_hot_sums_ok": ok}


def _plain(pp, synth_device, dev, stream):
    """The plain configuration: 524288 uint16 words (1 MiB) of Bernoulli(0.5)
    bits from seed 0, 16-byte aligned, w = 16: GPU time per call (queued back
    to back, and the synchronous Fig. 2 form) next to the oracle's."""
    import torch
    n = 524288
    words = torch.empty(2 * n, dtype=torch.uint8, device=dev)
    synth_device.random_(words, 0)
    c = torch.zeros(16, dtype=torch.int64, device=dev)
    ms = _time_ms(lambda: pp.pospopcnt_async(16, c, words, 2 * n, stream), stream, reps=200)
    torch.cuda.synchronize()
    for _ in range(20):
        pp.pospopcnt_u16(c, words, n)
    t0 = time.perf_counter()
    for _ in range(200):
        pp.pospopcnt_u16(c, words, n)
    sync_us = (time.perf_counter() - t0) / 200 * 1e6
    import oracle
    orc = oracle.load()
    host = words.cpu().numpy()
    ora = _oracle_rate(lambda: orc.typed(16, host.view(np.uint16)), lambda: host.size, budget_s=1.0)
    one = torch.zeros(16, dtype=torch.int64, device=dev)
    pp.pospopcnt_u16(one, words, n)
    ok = bool(np.array_equal(one.cpu().numpy().view(np.uint64), orc.typed(16, host.view(np.uint16))))
    return {"workload": "524288 uint16 words (1 MiB), Bernoulli(0.5) bits, seed 0, 16-byte aligned, w=16",
            "device_us_per_call": round(ms * 1e3, 2), "GBps": round(2 * n / (ms / 1e3) / 1e9, 1),
            "sync_call_us": round(sync_us, 2),
            "oracle_ms_per_call": round(2 * n / (ora * 1e9) * 1e3, 3), "oracle_GBps": ora,
            "oracle_sample": "the whole array, 1 thread (Fig. 2 loop)", "counts_ok": ok}


@contextlib.contextmanager
def _tune_entry(pp, kind, line):
    """Run the body with the tune table's `kind` entry replaced by `line`."""
    saved = pp.pospopcnt_tune_describe()
    with tempfile.TemporaryDirectory() as td:
        f = os.path.join(td, "tune.txt")
        with open(f, "w") as fh:
            fh.write("\n".join(l for l in saved.splitlines() if not l.startswith(kind)))
            fh.write("\n" + line + "\n")
        pp.pospopcnt_tune_load(f)
        try:
            yield
        finally:
            with open(f, "w") as fh:
                fh.write(saved)
            pp.pospopcnt_tune_load(f)


def _short(pp, synth, synth_device, dev, stream, n=2000):
    """Short unaligned arrays (log-uniform 1 B .. 64 KiB), one launch per array."""
    import torch
    sizes = synth.log_uniform_sizes(n, 1, 65536, seed=21)
    slot = 65536 + 32
    buf = torch.empty(slot * 64, dtype=torch.uint8, device=dev)
    synth_device.random_(buf, 22)
    c = torch.zeros(64, dtype=torch.int64, device=dev)
    basep = buf.data_ptr()
    calls = [(WIDTHS[k % 4], basep + (k % 64) * slot + (k % 16), int(sizes[k])) for k in range(n)]
    for w, p, s in calls[:50]:
        pp.pospopcnt_async(w, c, p, s, stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    for w, p, s in calls:
        pp.pospopcnt_async(w, c, p, s, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    dev_us = e0.elapsed_time(e1) * 1e3 / n

    # the same calls straight through the C ABI (arguments prepared beforehand),
    # with the tune table's programmatic dependent launch on, then off
    L = pp.lib()
    cp, sp = c.data_ptr(), stream.cuda_stream

    def raw_loop():
        bad = 0
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        e0.record(stream)
        for w, p, s in calls:
            bad |= L.pospopcnt_async(w, cp, p, s, sp)
        e1.record(stream)
        torch.cuda.synchronize()
        if bad:
            raise RuntimeError(pp.strerror(bad))
        return e0.elapsed_time(e1) * 1e3 / n, (time.perf_counter() - t1) * 1e6 / n

    raw_loop()
    raw_dev, raw_host = raw_loop()
    with _tune_entry(pp, "pdl", "pdl 0"):
        raw_loop()
        nopdl_dev, _ = raw_loop()
    # graph-replayed: the same launches captured once
    g = torch.cuda.CUDAGraph()
    s2 = torch.cuda.Stream()
    with torch.cuda.stream(s2):
        g.capture_begin()
        for w, p, s in calls:
            pp.pospopcnt_async(w, c, p, s, s2)
        g.capture_end()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    e0.record(stream)
    g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    graph_us = e0.elapsed_time(e1) * 1e3 / n
    return {"workload": f"{n} arrays, sizes log-uniform 1 B..64 KiB, start offsets 0..15, "
                        "w cycling 8/16/32/64, one launch each",
            "device_us_per_call": round(dev_us, 2), "host_us_per_call": round(wall * 1e6 / n, 2),
            "c_abi_device_us_per_call": round(raw_dev, 2),
            "c_abi_host_us_per_call": round(raw_host, 2),
            "c_abi_device_us_per_call_pdl_off": round(nopdl_dev, 2),
            "graph_us_per_call": round(graph_us, 2),
            "note": "device_us/host_us: calls through the Python binding; c_abi_*: the same calls "
                    "through the C entry point with prepared arguments"}


def _multi(pp, synth_device, data, nbytes, dev, stream, hbm_peak, group=16):
    """pospopcnt_multi through the C entry point with prepared arguments:
    (1) the plain configuration (524288 uint16 words, 1 MiB, seed 0, w = 16)
    counted `group` times per launch, each into its own counters, device
    microseconds per count (L2-resident, like the plain section); (2) four
    1 GiB arrays (the first 4 GiB of the resident array, w = 8, 16, 32, 64)
    in one launch, against the same four counts as four single launches."""
    import ctypes
    import torch
    import oracle
    L = pp.lib()
    n = 524288
    words = torch.empty(2 * n, dtype=torch.uint8, device=dev)
    synth_device.random_(words, 0)
    c = torch.zeros((group, 16), dtype=torch.int64, device=dev)
    W = (ctypes.c_int * group)(*([16] * group))
    C = (ctypes.c_uint64 * group)(*[c[i].data_ptr() for i in range(group)])
    P = (ctypes.c_uint64 * group)(*([words.data_ptr()] * group))
    N = (ctypes.c_size_t * group)(*([2 * n] * group))
    sp = stream.cuda_stream
    calls = []
    ms = _time_ms(lambda: L.pospopcnt_multi(group, W, C, P, N, sp), stream, reps=200, calls=calls)
    orc = oracle.load()
    exp = orc.typed(16, words.cpu().numpy().view(np.uint16))
    got = c.cpu().numpy().view(np.uint64)
    ok_plain = bool(all(np.array_equal(got[i], exp * np.uint64(calls[0])) for i in range(group)))
    out = {"plain_group": {
        "workload": f"{group} counts of the plain configuration (1 MiB of uint16 words, w=16) "
                    "per launch, each into its own counters",
        "device_us_per_launch": round(ms * 1e3, 2), "device_us_per_count": round(ms * 1e3 / group, 3),
        "GBps": round(group * 2 * n / (ms / 1e3) / 1e9, 1), "counts_ok": ok_plain}}
    if nbytes >= 4 * GIB:
        ws = (8, 16, 32, 64)
        c4 = torch.zeros((4, 64), dtype=torch.int64, device=dev)
        W4 = (ctypes.c_int * 4)(*ws)
        C4 = (ctypes.c_uint64 * 4)(*[c4[i].data_ptr() for i in range(4)])
        P4 = (ctypes.c_uint64 * 4)(*[data.data_ptr() + i * GIB for i in range(4)])
        N4 = (ctypes.c_size_t * 4)(*([GIB] * 4))
        ms_multi = _time_ms(lambda: L.pospopcnt_multi(4, W4, C4, P4, N4, sp), stream, reps=10)

        def singles():
            for i, w in enumerate(ws):
                L.pospopcnt_async(w, c4[i].data_ptr(), data.data_ptr() + i * GIB, GIB, sp)

        ms_single = _time_ms(singles, stream, reps=10)
        # the two ways agree count for count (the same calls, so the same totals)
        c4.zero_()
        L.pospopcnt_multi(4, W4, C4, P4, N4, sp)
        a = c4.clone()
        c4.zero_()
        singles()
        torch.cuda.synchronize()
        gm = 4 * GIB / (ms_multi / 1e3) / 1e9
        gs = 4 * GIB / (ms_single / 1e3) / 1e9
        out["four_1GiB"] = {"workload": "the first 4 GiB of the resident array as four 1 GiB "
                                        "counts (w = 8, 16, 32, 64)",
                            "multi_GBps": round(gm, 1), "single_launches_GBps": round(gs, 1),
                            "multi_frac_of_hbm_peak": round(gm / hbm_peak, 4),
                            "same_counts": bool(torch.equal(a, c4))}
    return out


def _sizes(pp, data, nbytes, stream, large_gbs, sizes=(1 << 20, 16 << 20, 128 << 20, GIB)):
    """One count of a given size: launches back to back (each on the next
    slice of the resident array, so that arrays below the L2 size are read
    from DRAM), for the single-array count, the same count as a one-entry
    pospopcnt_multi and the roofline read kernel; plus the single-array
    count timed alone (a synchronize before each launch, so that the time
    includes the launch itself)."""
    import torch
    c = torch.zeros(64, dtype=torch.int64, device=data.device)
    rsum = torch.zeros(1, dtype=torch.int64, device=data.device)
    base = data.data_ptr()
    out = {"workload": "w = 16 counts of one array of each size, 16-byte aligned slices of the "
                       "resident array, 20 launches back to back after 5 warm-up launches",
           "large_array_GBps": round(large_gbs, 1), "sizes": []}
    for size in sizes:
        if size > nbytes:
            continue
        slots = max(1, min(16, nbytes // size))
        row = {"bytes": size}
        for name, f in (("count", lambda o: pp.pospopcnt_async(16, c, base + o, size, stream)),
                        ("multi_one", lambda o: pp.pospopcnt_multi([16], [c], [base + o], [size],
                                                                   stream)),
                        ("roofline_read", lambda o: pp.pospopcnt_roofline_read(base + o, rsum, size,
                                                                               stream))):
            k = [0]

            def call():
                f((k[0] % slots) * size)
                k[0] += 1
            us = _time_ms(call, stream, reps=20, warm=5, warm_s=0.02) * 1e3
            row[name + "_us"] = round(us, 2)
            row[name + "_GBps"] = round(size / us / 1e3, 1)
        alone = []
        for j in range(10):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pp.pospopcnt_async(16, c, base + (j % slots) * size, size, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            alone.append(e0.elapsed_time(e1) * 1e3)
        row["count_alone_us"] = round(float(np.median(alone)), 2)
        row["count_frac_of_large_array"] = round(row["count_GBps"] / large_gbs, 4)
        row["fixed_us"] = round(row["count_us"] - size / large_gbs / 1e3, 2)
        out["sizes"].append(row)
    return out


def _serving(pp, synth, pool, pool_bytes, large_gbs, dev, loads=(0.3, 0.6, 0.9),
             duration_s=0.3, budget=32 << 30):
    """Poisson request streams at fractions of the large-array rate, served by
    the continuous-batching loop over the resident 8 GiB pool."""
    import math
    import torch
    lo, hi = 64, 256 << 20
    mean = (hi - lo) / math.log((hi + 1) / lo)      # mean of the log-uniform size
    tune = {l.split()[0]: l.split()[1:] for l in pp.pospopcnt_tune_describe().splitlines()
            if l.startswith(("serve_mode", "serve_srf"))}
    mode = tune.get("serve_mode", ["0"])[0]
    if mode in ("1", "2", "3"):
        b, nl, rows = tune["serve_srf"]
        per_class = tune.get("serve_srf_class", ["0"] * 4)
        bounds = ("1 MiB", "16 MiB", "128 MiB")
        extra = "; ".join(f"{r} rows below {bounds[k]}" for k, r in enumerate(per_class[:3])
                          if r != "0")
        rows = (f"{rows} rows" if rows != "0" else "the class's rows") + \
            (f" ({extra})" if extra else "")
        if mode == "3":
            schedule = (f"smallest remaining first through a device-side queue into one resident "
                        f"grid, at most {int(b) >> 20} MiB unclaimed, {rows} a work item "
                        f"under load")
        else:
            schedule = (f"dispatch by remaining bytes{' per size class' if mode == '2' else ''}: "
                        f"smallest remaining first, {int(b) >> 20} MiB of work items a launch, "
                        f"{min(8, int(nl))} launches in flight"
                        f"{' per class' if mode == '2' else ''}, {rows} a work item under load")
    else:
        schedule = ("size classes below 1 MiB / 16 MiB / 128 MiB / above on prioritised "
                    "streams, 8 batch streams a class")
    out = {"workload": "Poisson arrivals; w uniform in {8,16,32,64}; sizes log-uniform "
                       "64 B..256 MiB at uniform offsets of the resident 8 GiB array",
           "mem_budget_bytes": budget, "max_inflight": 4096, "max_batches": 8,
           "schedule": schedule, "loads": []}
    for k, load in enumerate(loads):
        rate = load * large_gbs * 1e9 / mean
        n = max(100, int(rate * duration_s))
        r = synth.poisson_requests(n, rate, seed=500 + k, lo=lo, hi=hi, pool_bytes=pool_bytes)
        arrival = np.round(r["arrival_s"] * 1e9).astype(np.int64)
        ptrs = (pool.data_ptr() + r["offset"]).astype(np.uint64)
        results = np.zeros((n, 64), dtype=np.uint64)
        srv = pp.pospop_server_create(budget, 4096, 8)
        try:
            recs = pp.pospop_server_run_trace(srv, arrival, r["w"], ptrs, r["nbytes"], results)
        finally:
            pp.pospop_server_destroy(srv)
        lat_us = (recs["t_done_ns"] - recs["t_submit_ns"]) / 1e3
        span_s = (int(recs["t_done_ns"].max()) - int(recs["t_submit_ns"].min())) / 1e9
        total = int(r["nbytes"].sum())
        gbs = total / span_s / 1e9
        # each result equals the request's own single-array count (sampled)
        idx = np.linspace(0, n - 1, min(n, 300)).astype(np.int64)
        solo = torch.zeros((len(idx), 64), dtype=torch.int64, device=dev)
        for j, i in enumerate(idx):
            pp.pospopcnt_async(int(r["w"][i]), solo[j], int(ptrs[i]), int(r["nbytes"][i]))
        torch.cuda.synchronize()
        solo = solo.cpu().numpy().view(np.uint64)
        same = all(np.array_equal(results[i, :r["w"][i]], solo[j, :r["w"][i]])
                   for j, i in enumerate(idx))
        out["loads"].append({
            "offered_load": load, "offered_GBps": round(rate * mean / 1e9, 1), "requests": n,
            "bytes": total, "GBps": round(gbs, 1), "frac_of_large_array": round(gbs / large_gbs, 4),
            "p50_us": round(float(np.percentile(lat_us, 50)), 1),
            "p99_us": round(float(np.percentile(lat_us, 99)), 1),
            "p99_us_below_1MiB": _pct(lat_us[r["nbytes"] < (1 << 20)], 99),
            "p99_us_from_128MiB": _pct(lat_us[r["nbytes"] >= (128 << 20)], 99),
            "status_ok": bool((recs["status"] == 0).all()), "results_match_solo": bool(same)})
    out["lone_request"] = _serving_lone(pp, pool, dev)
    return out


def _serving_lone(pp, pool, dev, sizes=(64 << 10, 1 << 20, 16 << 20, 128 << 20, 256 << 20),
                  reps=20):
    """One request at a time (an idle server, light load): submit-to-done
    latency per size and the request's bytes over that latency."""
    import torch
    srv = pp.pospop_server_create(32 << 30, 4096, 8)
    out = []
    try:
        res = np.zeros(64, dtype=np.uint64)
        for nb in sizes:
            lat = []
            for r in range(reps + 3):          # 3 warm-up requests
                p0 = pool.data_ptr() + 16 * 1000 * r + 5
                pp.pospop_server_submit(srv, 16, p0, nb, res)
                rec = []
                while not rec:
                    rec = pp.pospop_server_poll(srv, 1, 1000)
                if r >= 3:
                    lat.append((rec[0].t_done_ns - rec[0].t_submit_ns) / 1e3)
            # the last request's result against its single-array count
            solo = torch.zeros(16, dtype=torch.int64, device=dev)
            pp.pospopcnt_async(16, solo, p0, nb)
            torch.cuda.synchronize()
            med = float(np.median(lat))
            out.append({"bytes": nb, "p50_us": round(med, 1),
                        "p99_us": round(float(np.percentile(lat, 99)), 1),
                        "GBps_at_p50": round(nb / (med * 1e-6) / 1e9, 1),
                        "result_matches_solo": bool(np.array_equal(
                            res[:16], solo.cpu().numpy().view(np.uint64)))})
    finally:
        pp.pospop_server_destroy(srv)
    return out


def _pct(a, q):
    return round(float(np.percentile(a, q)), 1) if a.size else None


def _oracle_rate(fn, nbytes_fn, budget_s=2.0):
    """GB/s of an oracle call on the host cores, repeated for about budget_s seconds."""
    t0 = time.perf_counter()
    done = 0
    while True:
        fn()
        done += nbytes_fn()
        if time.perf_counter() - t0 > budget_s:
            break
    return round(done / (time.perf_counter() - t0) / 1e9, 4)


def _time_ms(fn, stream, reps=10, warm=3, warm_s=0.1, calls=None):
    """Mean ms per call over `reps` calls after at least `warm` calls and
    `warm_s` seconds of warm-up (a section that follows seconds of host-only
    work, such as an oracle timing, otherwise starts on an idle GPU that has
    not come back to full clocks).  If `calls` is a list, the total number of
    calls made is appended to it."""
    import torch
    t0 = time.perf_counter()
    done = 0
    while done < warm or time.perf_counter() - t0 < warm_s:
        fn()
        done += 1
        if done % 8 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    if calls is not None:
        calls.append(done + reps)
    return e0.elapsed_time(e1) / reps


def _masked(pp, synth_device, data, nbytes, dev, stream, large_gbs, hbm_peak):
    """WHERE-selected count: the 8 GiB array as 32-bit words, half of them selected."""
    import torch
    n = nbytes // 4
    sel = torch.empty((n + 7) // 8, dtype=torch.uint8, device=dev)
    synth_device.random_(sel, 4242)
    c = torch.zeros(32, dtype=torch.int64, device=dev)
    ms = _time_ms(lambda: pp.pospopcnt_masked(32, c, data, n, sel, stream), stream)
    moved = nbytes + sel.numel()
    gbs = moved / (ms / 1e3) / 1e9
    import oracle
    orc = oracle.load()
    k = 16 << 20                     # 16 Mi words = 64 MiB sample
    wh = data[:4 * k].cpu().numpy()
    sh = sel[:k // 8].cpu().numpy()
    ora = _oracle_rate(lambda: orc.masked(32, wh, k, sh), lambda: wh.size + sh.size)
    del sel
    return {"oracle_GBps": ora, "oracle_sample": "first 64 MiB of words + their bitmap, 1 thread",
            "workload": "8 GiB array as 2^31 uint32 words, selection bitmap of 256 MiB with "
                        "Bernoulli(0.5) bits, w=32",
            "ms": round(ms, 4), "GBps": round(gbs, 1), "frac_of_hbm_peak": round(gbs / hbm_peak, 4),
            "frac_of_plain_count": round(gbs / large_gbs, 4),
            "bytes_per_launch": moved}


def _gather(pp, synth, data, nbytes, dev, stream, large_gbs, hbm_peak, m=100000):
    """Many separate regions of the resident array counted into one counter array."""
    import torch
    lens = synth.log_uniform_sizes(m, 1, 1 << 20, seed=61)
    starts = np.floor(synth.uniforms(m, 62) * (nbytes - (1 << 20))).astype(np.int64)
    ptrs = torch.from_numpy(data.data_ptr() + starts).to(dev)
    ln = torch.from_numpy(lens.astype(np.int64)).to(dev)
    c = torch.zeros(16, dtype=torch.int64, device=dev)
    ms = _time_ms(lambda: pp.pospopcnt_gather(16, c, ptrs, ln, m, stream), stream)
    total = int(lens.sum())
    gbs = total / (ms / 1e3) / 1e9
    import oracle
    orc = oracle.load()
    k = 1000
    regions = [data[int(a):int(a) + int(b)].cpu().numpy() for a, b in zip(starts[:k], lens[:k])]
    ora = _oracle_rate(lambda: orc.gather(16, regions), lambda: sum(r.size for r in regions))
    return {"oracle_GBps": ora, "oracle_sample": f"first {k} regions, 1 thread",
            "workload": f"{m} regions of the 8 GiB array, lengths log-uniform 1 B..1 MiB, "
                        "uniform unaligned starts, w=16, one counter array",
            "bytes": total, "ms": round(ms, 4), "GBps": round(gbs, 1),
            "frac_of_hbm_peak": round(gbs / hbm_peak, 4),
            "frac_of_large_array": round(gbs / large_gbs, 4)}


def _tuned(pp, synth, synth_device, data, nbytes, dev, stream, large_gbs, max_bytes=GIB):
    """The autotuner's table against the shipped one: pospopcnt_autotune on
    max_bytes of scratch, then, with each table installed in turn, the
    200000-array ragged batch, counts of 128 MiB and 1 GiB (back to back on
    rotating slices) and of the whole array, and the serving trace at 0.9
    load.  The shipped table is installed again at the end."""
    import tempfile
    import torch
    shipped = pp.pospopcnt_tune_describe()
    with tempfile.NamedTemporaryFile("w", suffix=".txt", delete=False) as f:
        f.write(shipped)
        shipped_path = f.name
    tuned_path = shipped_path + ".tuned"
    t0 = time.perf_counter()
    pp.pospopcnt_autotune(max_bytes, tuned_path)
    tune_s = time.perf_counter() - t0
    tuned = open(tuned_path).read()

    def entries(text):
        return {l for l in text.splitlines() if l and not l.startswith("#")}
    m = 200000
    sizes = synth.log_uniform_sizes(m, 1, 4 << 20, seed=3)
    offs = synth.csr_offsets(sizes)
    total = int(offs[-1])
    base = torch.empty(total + 64, dtype=torch.uint8, device=dev)
    synth_device.one_hot_(base, 4, nbytes=total)
    offs_d = torch.from_numpy(offs.view(np.int64)).to(dev)
    cb = torch.zeros((m, 8), dtype=torch.int64, device=dev)
    c = torch.zeros(64, dtype=torch.int64, device=dev)
    out = {"workload": f"pospopcnt_autotune on {max_bytes >> 20} MiB of scratch; each table: "
                       "the 200000-array ragged batch (w = 8), w = 16 counts of 128 MiB and "
                       "1 GiB on rotating slices and of the whole array, the serving trace at "
                       "0.9 load",
           "tune_s": round(tune_s, 1),
           "only_shipped": sorted(entries(shipped) - entries(tuned)),
           "only_tuned": sorted(entries(tuned) - entries(shipped))}
    try:
        for name, path in (("shipped", shipped_path), ("tuned", tuned_path)):
            pp.pospopcnt_tune_load(path)
            row = {}
            ms = _time_ms(lambda: pp.pospopcnt_batch(8, cb, base, offs_d, m, stream), stream)
            row["batch_GBps"] = round(total / ms / 1e6, 1)
            for size in (128 << 20, GIB):
                slots = max(1, min(16, nbytes // size))
                k = [0]

                def call():
                    pp.pospopcnt_async(16, c, data.data_ptr() + (k[0] % slots) * size, size,
                                       stream)
                    k[0] += 1
                row[f"count_{size >> 20}MiB_us"] = round(_time_ms(call, stream, reps=20) * 1e3, 2)
            ms = _time_ms(lambda: pp.pospopcnt_async(16, c, data, nbytes, stream), stream)
            row["count_whole_GBps"] = round(nbytes / ms / 1e6, 1)
            sv = _serving(pp, synth, data, nbytes, large_gbs, dev, loads=(0.9,))
            ld = sv["loads"][0]
            row["serving_0.9"] = {k: ld[k] for k in ("GBps", "p50_us", "p99_us", "results_match_solo")}
            out[name] = row
    finally:
        pp.pospopcnt_tune_load(shipped_path)
        del base, cb
        torch.cuda.empty_cache()
    return out


def _sweep(pp, synth_device, data, nbytes, stream, hbm_peak, seed):
    """The large-array sweep: w x {1 GiB, 8 GiB} x Bernoulli(p) for p in
    {0.01, 0.5, 0.99} plus all-ones, each cell timed like the headline launch
    and its counts checked (all-ones: the closed form; Bernoulli: within 6
    sigma of n*p).  The resident array is restored to the headline data."""
    import torch
    sizes = [z for z in (GIB, 8 * GIB) if z <= nbytes]
    cells = []
    ok = True
    warm, reps = 3, 10
    # the read roofline at each size: the roofline read kernel, timed the same way
    rsum = torch.zeros(1, dtype=torch.int64, device=data.device)
    read_gbs = {size: size / (_time_ms(lambda: pp.pospopcnt_roofline_read(data, rsum, size, stream),
                                        stream, reps=reps, warm=warm) / 1e3) / 1e9
                for size in sizes}
    for p in (0.01, 0.5, 0.99, 1.0):
        if p == 1.0:
            synth_device.fill_(data, 0xFF, nbytes=sizes[-1], stream=stream)
        else:
            synth_device.bernoulli_(data, p, 7000 + int(p * 100), nbytes=sizes[-1], stream=stream)
        for size in sizes:
            for w in WIDTHS:
                c = torch.zeros(w, dtype=torch.int64, device=data.device)
                ncalls = []
                ms = _time_ms(lambda: pp.pospopcnt_async(w, c, data, size, stream), stream,
                              reps=reps, warm=warm, calls=ncalls)
                per = c.cpu().numpy().view(np.uint64).astype(np.float64) / ncalls[0]
                words = size * 8 // w
                if p == 1.0:
                    good = bool(np.all(per == words))
                else:
                    good = bool(np.all(np.abs(per - words * p) <= 6 * np.sqrt(words * p * (1 - p))))
                ok &= good
                gbs = size / (ms / 1e3) / 1e9
                cells.append({"w": w, "bytes": size, "p": "ones" if p == 1.0 else p,
                              "GBps": round(gbs, 1), "frac_of_hbm_peak": round(gbs / hbm_peak, 4),
                              "frac_of_read_roofline": round(gbs / read_gbs[size], 4),
                              "counts_ok": good})
    synth_device.bernoulli_(data, 0.5, seed, stream=stream)
    torch.cuda.synchronize()
    fr = [c["frac_of_hbm_peak"] for c in cells]
    return {"workload": "w in {8,16,32,64} x {1 GiB, 8 GiB} x Bernoulli(p), p in {0.01,0.5,0.99} "
                        "plus all-ones; 10 launches per cell after at least 3 warm-up launches "
                        "and 0.1 s",
            "min_frac_of_hbm_peak": min(fr), "max_frac_of_hbm_peak": max(fr),
            "read_roofline_GBps": {str(z): round(g, 1) for z, g in read_gbs.items()},
            "min_frac_of_read_roofline": min(c["frac_of_read_roofline"] for c in cells),
            "all_counts_ok": ok, "cells": cells}


def run_reference(args):
    """The CPU oracle (the reference arm of this tier) on the same workload."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_2412_16370_gb300 import synth
    orc = oracle.load()
    cores = os.cpu_count() or 1
    sample = args.ref_sample_mib << 20
    host = synth.bernoulli_bytes(sample, 0.5, seed=0)
    for _ in range(args.warmup):
        orc.bytes_mt(16, host[:1 << 20], cores)
    step_rates = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        t1 = time.perf_counter()
        for w in WIDTHS:
            orc.bytes_mt(w, host, cores)
        step_rates.append(sample * len(WIDTHS) / (time.perf_counter() - t1) / 1e9)
    dt = time.perf_counter() - t0
    value = sample * len(WIDTHS) * args.steps / dt / 1e9
    desc = (f"first {args.ref_sample_mib} MiB of the 8 GiB Bernoulli(0.5) array (seed 0), "
            f"counted for w in {{8,16,32,64}} per step with {cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt * 1e3 / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic (seeded SplitMix64 Bernoulli(0.5) bits)",
            "config": {"workload": WORKLOAD, "parallelism": "host cores",
                       "sample_bytes_per_step": sample * len(WIDTHS)},
            "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": cores,
                             "kind": "oracle", "sample": desc, "cpu_model": _cpu_model(),
                             "step_GBps_min_median_max": [round(min(step_rates), 4),
                                                          round(float(np.median(step_rates)), 4),
                                                          round(max(step_rates), 4)]},
            "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--gib", type=int, default=8, help="array size in GiB (8 = the workload)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--batched-m", type=int, default=200000,
                    help="arrays in the batched section (200000 = the workload)")
    ap.add_argument("--ref-sample-mib", type=int, default=1024,
                    help="sample of the array the reference arm counts per step (MiB; "
                         "the same size as cpu_baseline's sample)")
    ap.add_argument("--shard", action="store_true",
                    help="split one array across the ranks (strong scaling) instead of "
                         "independent replicas")
    ap.add_argument("--no-verify", action="store_true",
                    help="skip the oracle check of the timed counts (about 10 s of host work)")
    ap.add_argument("--quick", action="store_true",
                    help="skip every section after the headline (e2e, batched, plain, "
                         "short, multi, sizes, serving, masked, gather, cpu_baseline, sweep)")
    ap.add_argument("--sections", default="",
                    help="comma list of extra sections to run (e2e,batched,plain,short,multi,"
                         "sizes,serving,masked,gather,cpu_baseline,sweep,tuned)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
