#!/usr/bin/env python
"""Throughput of the GB300 Huskysort string argsort.

One step = one full stable argsort (encode, radix sort of the codes, tie
fix-up) of the largest single-GPU workload, 1e9 skewed strings (first letter
Zipf(1.5) over a..z, lengths normal(10, 3) clipped to 1..24) with a u64
permutation, inputs resident in HBM.  The same line carries the metric's
comparison: the learned bucketer on the same strings, and the batched form
(2,000 of the 20,000 log-uniform instances by default) against a loop of
single sorts and against one plain sort of all its strings.  Prints one JSON
line.  `--impl reference` times the CPU oracle (the plain stable merge sort)
on the host cores instead, on a bounded sample of the same workload.

Under torchrun (N > 1) every rank sorts its own copy of the workload
(replicas: a single sort has no shard-local form without an exchange step);
value = strings sorted by all ranks / max-over-ranks time.
"""

from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "strings sorted/sec (M keys/s) and % of HBM roofline, learned/batched vs plain radix"
UNIT = "M keys/s"
DEFAULT_WORKLOAD = "skewed_1e9"
L2_FLUSH_BYTES = 256 << 20
CPU_SAMPLE_MAX = 10_000_000   # strings the CPU baseline sorts at most


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=DEFAULT_WORKLOAD,
                   help="one of workloads.STANDARD (batched_* use hs_argsort_batched) or NUMERIC "
                        "(arrays sorted by hs_argsort_numeric)")
    p.add_argument("--scale", type=float, default=1.0, help="scale the workload's size")
    p.add_argument("--mode", default="plain", choices=["plain", "learned", "loop"],
                   help="loop: a batched workload sorted one instance at a time with hs_argsort")
    p.add_argument("--index", default=None, choices=["u32", "u64"],
                   help="permutation index type (default: u64 above 2^31 strings or for skewed_1e9, else u32)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the default radix tile shape instead of timing the candidates on the first sort "
                        "(for profiler runs, whose serialised launches distort the comparison)")
    p.add_argument("--stats", default=None, help="write per-kernel stats JSON here")
    p.add_argument("--no-compare", dest="compare", action="store_false",
                   help="skip the learned and batched comparison blocks of a plain single-sort run")
    p.add_argument("--batched-scale", type=float, default=0.1,
                   help="size of the batched comparison block as a fraction of batched_20000's 20,000 instances")
    p.add_argument("--parity-samples", type=int, default=100_000,
                   help="adjacent output pairs checked with the oracle's comparison at full size (0: none)")
    return p.parse_args()


# ---- distributed plumbing ---------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, local, backend="nccl"):
    import torch
    if world > 1:
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def job_throughput(n_per_rank, world, ms):
    """Whole-job M keys/s: the strings all ranks sorted over the slowest
    rank's time (replicas: every rank sorts its own copy of the workload)."""
    return n_per_rank * world / (ms / 1e3) / 1e6


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- clocks -------------------------------------------------------------------

REASONS = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


class ClockSampler:
    """nvidia-smi sampling (200 ms) of the bench GPU during the timed region."""

    def __init__(self, uuid):
        self.uuid = uuid
        self.rows = []
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        cmd = ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, seen = [], [], set()
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(REASONS[1:], r[5:9]):
                if v.lower() in ("active", "0x1", "1", "yes"):
                    seen.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(seen)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


TRAFFIC_SOURCES = ["paper_2012_00866_gb300/csrc/sort.cu", "paper_2012_00866_gb300/csrc/hs_device.cuh",
                   "paper_2012_00866_gb300/csrc/hs_internal.h"]


def _code_only(src: str) -> str:
    """C/CUDA source without comments and blank lines: the digest follows
    the code, so an edited comment does not void a capture."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.strip() for line in src.split("\n") if line.strip())


def sources_digest(paths=TRAFFIC_SOURCES):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), encoding="utf-8") as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()


def profile_traffic(key: str):
    """DRAM bytes per launch (read + write, averaged over the step's launches
    of the kernel) from the committed ncu summary profiles/traffic.json, if
    the kernel's sources are unchanged since the capture (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            data = json.load(f)
    except OSError:
        return None
    entry = data.get(key)
    if not entry:
        return None
    try:
        digest = sources_digest(entry.get("sources", TRAFFIC_SOURCES))
    except OSError:
        return None
    if entry.get("sources_sha256") != digest:
        return None
    return entry.get("dram_bytes_per_launch")


# ---- our arm --------------------------------------------------------------------

def _sample(w, limit):
    """The first `limit` strings of a workload (same distribution)."""
    import workloads
    if w.n <= limit:
        return w
    off = w.offsets[: limit + 1]
    return workloads.Workload(w.bytes[: int(off[-1])], off.copy())


def _prefix(name, scale, limit):
    """The first `limit` strings of a standard single-sort workload, generated
    on their own (the generators are keyed by string index, so these are the
    same strings as in the full workload)."""
    import workloads
    spec = workloads.STANDARD[name]
    n = max(1, int(round(spec["n"] * scale)))
    return workloads.generate(spec["kind"], min(n, limit), spec["seed"]), n


def _gpu_uuid(device):
    import torch
    try:
        uuid = str(torch.cuda.get_device_properties(device).uuid)
        return uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        return None


def _time_steps(step, steps, flush, stream):
    """CUDA-event times (ms) of `steps` calls of step(), the L2 flushed by a
    256 MiB write before each."""
    import torch
    out = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def _kernel_stats(hs, step, steps, flush, stream):
    """Per-kernel CUDA-event stats of `steps` more calls, outside any timed
    region (the launches are bracketed by events)."""
    import torch
    hs.stats_enable(True)
    _time_steps(step, steps, flush, stream)
    torch.cuda.synchronize()
    kstats = hs.stats_read()
    hs.stats_enable(False)
    return kstats


def _roofline(kstats, steps, ms, traffic_key=None):
    """Roofline of the kernel with the most time: algorithmic bytes per launch
    over its mean CUDA-event launch time, against the measured copy peak."""
    peaks, peak_src = measured_peaks()
    timed = {k: v for k, v in kstats.items() if v["launches"] and v["total_ms"] > 0}
    if not timed:
        return None
    top = max(timed, key=lambda k: timed[k]["total_ms"])
    st = timed[top]
    achieved = st["algo_bytes"] / (st["total_ms"] / 1e3) / 1e9
    return {"kernel": top + "_kernel", "bound": "hbm", "achieved": round(achieved, 1),
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
            "peak_source": ("measured (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                            else "fallback 6.8 TB/s"),
            "algo_bytes_per_launch": st["algo_bytes"] / st["launches"],
            "launch_ms": round(st["total_ms"] / st["launches"], 5),
            "share_of_step": round(st["total_ms"] / steps / ms, 3),
            "traffic": profile_traffic(f"{top}_kernel/{traffic_key}") if traffic_key else None}


def _stages(kstats, steps):
    return {k: {"launches_per_step": v["launches"] / steps, "ms_per_step": round(v["total_ms"] / steps, 4),
                "GBps": round(v["algo_bytes"] / (v["total_ms"] / 1e3) / 1e9, 1) if v["total_ms"] > 0 else None}
            for k, v in kstats.items() if v["launches"]}


def _sampled_pairs_in_order(w, perm_np, samples, seed=0):
    """Sampled parity at full size: `samples` random adjacent positions k of
    the permutation are checked with the oracle's string comparison (string
    perm[k] before string perm[k+1], ties by index).  Returns the number of
    pairs out of order."""
    import oracle
    rng = np.random.default_rng(seed)
    n = perm_np.size
    if n < 2:
        return 0
    bad = 0
    for k in rng.integers(0, n - 1, size=min(samples, n - 1)):
        a, b = int(perm_np[k]), int(perm_np[k + 1])
        c = oracle.string_compare(w.bytes, w.offsets, a, b)
        bad += c > 0 or (c == 0 and a > b)
    return bad


def _learned_block(hs, args, w, data, off, perm_plain, index_u64, flush, stream, n):
    """The learned bucketer on the same strings: throughput, its roofline and
    its parity (equal to the plain path's permutation, and sampled adjacent
    pairs in order by the oracle's comparison)."""
    import torch
    perm = torch.empty_like(perm_plain)

    def step():
        return hs.argsort_device(data, off, mode=hs.MODE_LEARNED, index_u64=index_u64, out=perm)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ms_list = _time_steps(step, args.steps, flush, stream)
    ms = sum(ms_list) / len(ms_list)
    kstats = _kernel_stats(hs, step, args.steps, flush, stream)
    equal = bool(torch.equal(perm, perm_plain))
    sample = None
    if args.parity_samples:
        sample = _sampled_pairs_in_order(w, perm.cpu().numpy().view(np.uint64 if index_u64 else np.uint32),
                                         args.parity_samples)
    return {"value": round(n / (ms / 1e3) / 1e6, 3), "unit": UNIT, "ms_per_step": round(ms, 4),
            "vs_plain": None,
            "parity": {"equal_to_plain_permutation": equal,
                       "oracle_sampled_pairs": args.parity_samples, "pairs_out_of_order": sample},
            "roofline": _roofline(kstats, args.steps, ms, f"{args.workload}/learned"),
            "gpu_launches": int(sum(v["launches"] for v in kstats.values()) / args.steps),
            "stages": _stages(kstats, args.steps)}


def _batched_block(hs, args, device, flush, stream):
    """hs_argsort_batched on the batched workload (at --batched-scale of its
    20,000 instances) against two references on the same GPU: the
    per-instance loop of hs_argsort calls, and one plain hs_argsort of all
    the strings as a single instance."""
    import torch
    import oracle
    import workloads
    w = workloads.standard("batched_20000", scale=args.batched_scale)
    n = w.n
    data = torch.from_numpy(w.bytes).to(device)
    off = torch.from_numpy(w.offsets.view(np.int64)).to(device)
    seg = torch.from_numpy(w.seg_offsets.view(np.int64)).to(device)
    perm = torch.empty(n, dtype=torch.int32, device=device)

    def batched():
        return hs.argsort_batched(data, off, seg, out=perm)

    for _ in range(args.warmup):
        batched()
    torch.cuda.synchronize()
    ms_list = _time_steps(batched, args.steps, flush, stream)
    ms = sum(ms_list) / len(ms_list)
    kstats = _kernel_stats(hs, batched, args.steps, flush, stream)
    got = perm.cpu().numpy().view(np.uint32)
    # parity: every instance of at most 20,000 strings among the first 400
    # instances, against the oracle's stable argsort of that instance
    checked, bad = 0, 0
    for k in range(min(400, len(w.seg_offsets) - 1)):
        lo, hi = int(w.seg_offsets[k]), int(w.seg_offsets[k + 1])
        if hi - lo > 20_000:
            continue
        o = w.offsets[lo:hi + 1]
        want = oracle.stable_argsort(w.bytes[int(o[0]):int(o[-1])], o - o[0])
        bad += int(not np.array_equal(got[lo:hi], want))
        checked += 1

    views = []
    for k in range(len(w.seg_offsets) - 1):
        lo, hi = int(w.seg_offsets[k]), int(w.seg_offsets[k + 1])
        if hi > lo:
            views.append((data[int(w.offsets[lo]):int(w.offsets[hi])],
                          off[lo:hi + 1] - int(w.offsets[lo]), perm[lo:hi]))

    def loop():
        for d, o, p in views:
            hs.argsort_device(d, o, out=p)

    loop_steps = max(1, min(args.steps, 5))
    loop()
    torch.cuda.synchronize()
    loop_ms = sum(_time_steps(loop, loop_steps, flush, stream)) / loop_steps

    def single():
        return hs.argsort_device(data, off, out=perm)

    for _ in range(args.warmup):
        single()
    torch.cuda.synchronize()
    single_ms = sum(_time_steps(single, args.steps, flush, stream)) / args.steps
    del data, off, seg, perm, views
    torch.cuda.synchronize()
    return {"workload": "batched_20000" + (f"@{args.batched_scale:g}" if args.batched_scale != 1.0 else ""),
            "instances": int(len(w.seg_offsets) - 1), "n": n, "bytes": int(w.bytes.size),
            "value": round(n / (ms / 1e3) / 1e6, 3), "unit": UNIT, "ms_per_step": round(ms, 4),
            "per_instance_loop": {"value": round(n / (loop_ms / 1e3) / 1e6, 3), "ms_per_step": round(loop_ms, 3),
                                  "steps": loop_steps},
            "one_plain_sort_of_all_strings": {"value": round(n / (single_ms / 1e3) / 1e6, 3),
                                              "ms_per_step": round(single_ms, 4)},
            "vs_loop": round(loop_ms / ms, 2), "vs_one_plain_sort": round(single_ms / ms, 3),
            "parity": {"instances_checked_against_oracle": checked, "instances_differing": bad},
            "roofline": _roofline(kstats, args.steps, ms,
                                  "batched_20000" + (f"@{args.batched_scale:g}" if args.batched_scale != 1.0 else "")),
            "gpu_launches": int(sum(v["launches"] for v in kstats.values()) / args.steps),
            "stages": _stages(kstats, args.steps)}


def run_ours(args, rank, world, local):
    import torch
    import workloads
    import paper_2012_00866_gb300 as hs

    dist_init(world, local)
    device = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(device)
    hs.load()
    if args.no_autotune:
        hs.autotune(0)
    mode = hs.MODE_LEARNED if args.mode == "learned" else hs.MODE_PLAIN

    w = workloads.standard(args.workload, scale=args.scale)
    n = w.n
    batched = w.seg_offsets is not None
    index = args.index or ("u64" if (args.workload.startswith("skewed") and not batched) else "u32")
    index_u64 = index == "u64" and not batched
    data = torch.from_numpy(w.bytes).to(device)
    off = torch.from_numpy(w.offsets.view(np.int64)).to(device)
    seg = torch.from_numpy(w.seg_offsets.view(np.int64)).to(device) if batched else None
    perm = torch.empty(n, dtype=torch.int64 if index_u64 else torch.int32, device=device)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)
    stream = torch.cuda.current_stream(device)

    loop = args.mode == "loop" and batched
    if loop:  # per-instance views: string offsets rebased to the instance's first byte
        views = []
        for k in range(len(w.seg_offsets) - 1):
            lo, hi = int(w.seg_offsets[k]), int(w.seg_offsets[k + 1])
            if hi > lo:
                views.append((data[int(w.offsets[lo]):int(w.offsets[hi])],
                              off[lo:hi + 1] - int(w.offsets[lo]), perm[lo:hi]))

    def step():
        if loop:
            for d, o, p in views:
                hs.argsort_device(d, o, out=p)
            return perm
        if batched:
            return hs.argsort_batched(data, off, seg, out=perm)
        return hs.argsort_device(data, off, mode=mode, index_u64=index_u64, out=perm)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(device)

    clocks = ClockSampler(_gpu_uuid(device))
    # the timed region: no per-kernel instrumentation
    clocks.start()
    barrier(world)
    torch.cuda.synchronize(device)
    step_ms = _time_steps(step, args.steps, flush, stream)
    torch.cuda.synchronize(device)
    barrier(world)
    clock_info = clocks.stop()
    # the same steps again with per-kernel CUDA events (the stage breakdown
    # and the roofline's launch durations), outside the timed region
    kstats = _kernel_stats(hs, step, args.steps, flush, stream)

    ms = sum(step_ms) / len(step_ms)
    ms = max_over_ranks(ms, world, device)
    value = job_throughput(n, world, ms)

    # end to end through the public API: pinned host inputs in, host perm out
    e2e = None
    if not batched:
        h_data = torch.from_numpy(w.bytes).pin_memory()
        h_off = torch.from_numpy(w.offsets.view(np.int64)).pin_memory()
        # one pinned host permutation, allocated once and reused (the copy
        # back into it is inside every timed call)
        host_perm = torch.empty(n, dtype=torch.int64 if index_u64 else torch.int32, pin_memory=True)
        for _ in range(args.warmup):
            hs.argsort(h_data, h_off, mode=mode, index_u64=index_u64, out=host_perm)
        torch.cuda.synchronize(device)
        barrier(world)
        e2e_ms = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize(device)
            t0 = time.perf_counter()
            hs.argsort(h_data, h_off, mode=mode, index_u64=index_u64, out=host_perm)
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        barrier(world)
        e2e_t = max_over_ranks(sum(e2e_ms) / len(e2e_ms), world, device)
        e2e = {"value": round(n * world / (e2e_t / 1e3) / 1e6, 3), "unit": UNIT,
               "h2d_bytes_per_step": int(w.bytes.nbytes + w.offsets.nbytes),
               "d2h_bytes_per_step": int(n * (8 if index_u64 else 4)), "ms_per_step": round(e2e_t, 3)}
        del host_perm, h_data, h_off

    coder_name = "auto"
    if not batched:
        _, _, used = hs.encode(data, off)
        coder_name = "auto(" + {1: "ascii7", 2: "byte8", 3: "alpha"}.get(used, str(used)) + ")"

    roofline = _roofline(kstats, args.steps, ms, args.workload)
    launches = sum(v["launches"] for v in kstats.values()) / args.steps * args.steps
    stages = _stages(kstats, args.steps)

    # the metric's comparison: learned and batched forms against plain radix
    learned = None
    if (rank == 0 and world == 1 and not batched and not loop and mode == hs.MODE_PLAIN
            and args.compare and n >= 65536):
        learned = _learned_block(hs, args, w, data, off, perm, index_u64, flush, stream, n)
        learned["vs_plain"] = round(learned["value"] / value, 3)
    parity_plain = None
    if rank == 0 and not batched and not loop and args.parity_samples:
        parity_plain = {"oracle_sampled_pairs": args.parity_samples,
                        "pairs_out_of_order": _sampled_pairs_in_order(
                            w, perm.cpu().numpy().view(np.uint64 if index_u64 else np.uint32), args.parity_samples)}
    del data, off, seg
    batched_block = None
    if rank == 0 and world == 1 and not batched and args.compare:
        torch.cuda.synchronize(device)
        batched_block = _batched_block(hs, args, device, flush, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        threads = os.cpu_count() or 1
        if batched:
            k = 1
            while k < len(w.seg_offsets) - 1 and int(w.seg_offsets[k + 1]) <= CPU_SAMPLE_MAX:
                k += 1
            cut = int(w.seg_offsets[k])
            t0 = time.perf_counter()
            oracle.stable_argsort_batched(w.bytes, w.offsets[: cut + 1], w.seg_offsets[: k + 1], threads=threads)
            dt = time.perf_counter() - t0
            what = f"the first {k} instances ({cut} strings)"
            ns = cut
        else:
            sw = _sample(w, CPU_SAMPLE_MAX)
            t0 = time.perf_counter()
            oracle.stable_argsort(sw.bytes, sw.offsets, threads=threads)
            dt = time.perf_counter() - t0
            ns = sw.n
            what = "the full workload" if sw.n == n else f"the first {sw.n} strings"
        cpu = {"value": round(ns / dt / 1e6, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{what} of {args.workload}, one run, stable merge sort on {threads} threads"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": args.workload + (f"@{args.scale:g}" if args.scale != 1.0 else ""),
                       "n": n, "bytes": int(w.bytes.size),
                       "instances": int(len(w.seg_offsets) - 1) if batched else 1,
                       "mode": ("loop" if loop else "batched") if batched else args.mode,
                       "index": "u32" if not index_u64 else "u64",
                       "coder": coder_name,
                       "tile_keys_per_thread": {"packed_words": hs.autotune_choice(0, n),
                                                "pairs": hs.autotune_choice(1, n)},
                       "l2": "flushed by a 256 MiB write before every timed step",
                       "parallelism": "replicas" if world > 1 else "single"},
            "e2e": e2e,
            "gpu_launches": int(launches),
            "roofline": roofline,
            "parity": parity_plain,
            "learned": learned,
            "batched": batched_block,
            "cpu_baseline": cpu,
            "clocks": clock_info,
            "stages": stages,
        }
        print(json.dumps(line), flush=True)
        if args.stats:
            with open(args.stats, "w") as f:
                json.dump({"kernels": kstats, "steps": args.steps, "step_ms": step_ms}, f, indent=1)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---- numeric workloads: hs_argsort_numeric --------------------------------------

# name: (type, n, seed).  f64: normal values over many decades with 1% of
# +-0, +-infinity, NaN and subnormals; datetime: ns instants over 1900..2100
# with repeats; i32: full-range integers; bigint and bigdecimal: byte strings
# (see their generators below).
NUMERIC = {"f64_1e8": ("f64", 100_000_000, 11), "datetime_1e8": ("datetime", 100_000_000, 12),
           "i32_1e8": ("i32", 100_000_000, 13), "bigint_1e7": ("bigint", 10_000_000, 14),
           "bigdecimal_1e7": ("bigdecimal", 10_000_000, 15)}
BYTES_KINDS = ("bigint", "bigdecimal")  # values given as byte strings in the strings' data model


def bigdecimal_workload(n, seed):
    """n decimal texts (the form Java's BigDecimal(String) accepts): a minus
    sign on 45%, 1..20 digits, a point inside the digits on 70%, an exponent
    E[+-]d or E[+-]dd on 30%; 10% repeats of earlier texts."""
    import workloads
    rng = np.random.default_rng(seed)
    width = 1 + 20 + 1 + 4
    neg = (rng.random(n) < 0.45).astype(np.int64)
    m = rng.integers(1, 21, size=n)
    hasdot = (rng.random(n) < 0.7) & (m >= 2)
    q = np.where(hasdot, rng.integers(1, np.maximum(m, 2)), m)
    hasexp = rng.random(n) < 0.3
    ed = rng.integers(1, 3, size=n)
    chars = np.zeros((n, width), np.uint8)
    rows = np.arange(n)
    chars[rows[neg == 1], 0] = ord("-")
    digits = rng.integers(ord("0"), ord("9") + 1, size=(n, 20), dtype=np.uint8)
    for k in range(20):
        ok = k < m
        col = neg + k + (hasdot & (k >= q))
        chars[rows[ok], col[ok]] = digits[ok, k]
    chars[rows[hasdot], (neg + q)[hasdot]] = ord(".")
    e0 = neg + m + hasdot
    chars[rows[hasexp], e0[hasexp]] = ord("E")
    chars[rows[hasexp], (e0 + 1)[hasexp]] = np.where(rng.random(int(hasexp.sum())) < 0.5, ord("+"), ord("-"))
    for k in range(2):
        ok = hasexp & (k < ed)
        chars[rows[ok], (e0 + 2 + k)[ok]] = rng.integers(ord("0"), ord("9") + 1, size=int(ok.sum()))
    rep = rng.random(n) < 0.1
    src = rng.integers(0, n, size=n)
    rep &= ~rep[src]
    chars[rep] = chars[src[rep]]
    keep = chars != 0
    lens = keep.sum(axis=1).astype(np.uint64)
    off = np.zeros(n + 1, np.uint64)
    np.cumsum(lens, out=off[1:])
    return workloads.Workload(chars[keep], off)


def bytes_workload(kind, n, seed):
    return bigint_workload(n, seed) if kind == "bigint" else bigdecimal_workload(n, seed)


def bytes_argsort(hs, kind):
    return hs.argsort_bigint if kind == "bigint" else hs.argsort_bigdecimal


def bigint_workload(n, seed):
    """n big integers as minimal two's complement bytes (Java's toByteArray):
    lengths U{1..32}, random bytes, the leading byte adjusted where it would
    be a redundant sign byte; 10% repeats of earlier values."""
    import workloads
    rng = np.random.default_rng(seed)
    lens = rng.integers(1, 33, size=n).astype(np.uint64)
    rep = rng.random(n) < 0.1
    src = rng.integers(0, n, size=n)
    rep &= ~rep[src]  # a repeat copies a value that is not itself a repeat
    lens[rep] = lens[src[rep]]
    off = np.zeros(n + 1, np.uint64)
    np.cumsum(lens, out=off[1:])
    data = rng.integers(0, 256, size=int(off[-1]), dtype=np.uint8)
    first = off[:-1].astype(np.int64)
    multi = lens >= 2
    b0, b1 = data[first[multi]], data[first[multi] + 1]
    fix0 = (b0 == 0x00) & (b1 < 0x80)
    fixf = (b0 == 0xFF) & (b1 >= 0x80)
    idx = first[multi]
    data[idx[fix0]] = 0x01
    data[idx[fixf]] = 0xFE
    # repeats take the bytes of their source value (same length)
    s = np.where(rep, src, np.arange(n))
    vid = np.repeat(np.arange(n), lens.astype(np.int64))
    rel = np.arange(int(off[-1]), dtype=np.int64) - first[vid]
    data = data[first[s[vid]] + rel]
    return workloads.Workload(data, off)


def numeric_values(name, scale):
    kind, n, seed = NUMERIC[name]
    n = max(2, int(n * scale))
    rng = np.random.default_rng(seed)
    if kind == "f64":
        v = rng.standard_normal(n) * 10.0 ** rng.integers(-300, 300, size=n)
        pick = rng.random(n) < 0.01
        v[pick] = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324])[rng.integers(0, 6, size=int(pick.sum()))]
        return v, 3
    if kind == "datetime":
        v = rng.integers(-70 * 365 * 86400 * 10**9, 130 * 365 * 86400 * 10**9, size=n, dtype=np.int64)
        rep = rng.random(n) < 0.3
        v[rep] = v[rng.integers(0, n, size=int(rep.sum()))]
        return v, 5
    return rng.integers(-(1 << 31), 1 << 31, size=n, dtype=np.int64).astype(np.int32), 2


def run_numeric(args, rank, world, local):
    import torch
    import paper_2012_00866_gb300 as hs

    dist_init(world, local)
    device = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(device)
    hs.load()
    if args.no_autotune:
        hs.autotune(0)
    kind = NUMERIC[args.workload][0]
    index_u64 = args.index == "u64"
    if kind in BYTES_KINDS:
        bw = bytes_workload(kind, max(2, int(NUMERIC[args.workload][1] * args.scale)), NUMERIC[args.workload][2])
        n = bw.offsets.size - 1
        v = None
        xb = torch.from_numpy(bw.bytes).to(device)
        xo = torch.from_numpy(bw.offsets.view(np.int64)).to(device)
    else:
        v, t = numeric_values(args.workload, args.scale)
        n = v.size
        x = torch.from_numpy(v).to(device)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)
    stream = torch.cuda.current_stream(device)

    def step():
        if kind in BYTES_KINDS:
            return bytes_argsort(hs, kind)(xb, xo, index_u64=index_u64)
        return hs.argsort_numeric(x, type=t, index_u64=index_u64)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(device)
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(device).uuid)
        if not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)

    def timed_steps():
        out = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        return out

    clocks.start()
    barrier(world)
    torch.cuda.synchronize(device)
    step_ms = timed_steps()
    torch.cuda.synchronize(device)
    barrier(world)
    clock_info = clocks.stop()
    hs.stats_enable(True)
    timed_steps()
    torch.cuda.synchronize(device)
    kstats = hs.stats_read()
    hs.stats_enable(False)
    ms = max_over_ranks(sum(step_ms) / len(step_ms), world, device)
    value = job_throughput(n, world, ms)

    # end to end through the public call: pinned host values in, host permutation out
    h_perm = torch.empty(n, dtype=torch.int64 if index_u64 else torch.int32).pin_memory()
    if kind in BYTES_KINDS:
        hb = torch.from_numpy(bw.bytes).pin_memory()
        ho = torch.from_numpy(bw.offsets.view(np.int64)).pin_memory()
        h2d = int(bw.bytes.nbytes + bw.offsets.nbytes)

        def host_call():
            return bytes_argsort(hs, kind)(hb.to(device, non_blocking=True), ho.to(device, non_blocking=True),
                                           index_u64=index_u64)
    else:
        h_vals = torch.from_numpy(v).pin_memory()
        h2d = int(v.nbytes)

        def host_call():
            return hs.argsort_numeric(h_vals.to(device, non_blocking=True), type=t, index_u64=index_u64)
    for _ in range(2):
        h_perm.copy_(host_call())
    torch.cuda.synchronize(device)
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        h_perm.copy_(host_call())
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_t = max_over_ranks(sum(e2e_ms) / len(e2e_ms), world, device)
    e2e = {"value": round(n * world / (e2e_t / 1e3) / 1e6, 3), "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": int(n * (8 if index_u64 else 4)),
           "ms_per_step": round(e2e_t, 3)}

    peaks, peak_src = measured_peaks()
    timed = {k: s for k, s in kstats.items() if s["launches"] and s["total_ms"] > 0}
    top = max(timed, key=lambda k: timed[k]["total_ms"])
    st = timed[top]
    achieved = st["algo_bytes"] / (st["total_ms"] / 1e3) / 1e9
    roofline = {"kernel": top + "_kernel", "bound": "hbm", "achieved": round(achieved, 1),
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback 6.8 TB/s",
                "algo_bytes_per_launch": st["algo_bytes"] / st["launches"],
                "launch_ms": round(st["total_ms"] / st["launches"], 5),
                "share_of_step": round(st["total_ms"] / args.steps / ms, 3), "traffic": None}
    stages = {k: {"launches_per_step": s["launches"] / args.steps, "ms_per_step": round(s["total_ms"] / args.steps, 4),
                  "GBps": round(s["algo_bytes"] / (s["total_ms"] / 1e3) / 1e9, 1) if s["total_ms"] > 0 else None}
              for k, s in kstats.items() if s["launches"]}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        if kind in BYTES_KINDS:
            m = min(n, 1_000_000 if kind == "bigint" else 300_000)
            t0 = time.perf_counter()
            (oracle.bigint_argsort if kind == "bigint" else oracle.bigdecimal_argsort)(bw.bytes, bw.offsets[: m + 1])
            dt = time.perf_counter() - t0
            how = "Python int sort (one thread)" if kind == "bigint" else "Python Decimal sort (one thread)"
        else:
            m = min(n, CPU_SAMPLE_MAX)
            t0 = time.perf_counter()
            oracle.numeric_argsort(v[:m], t)
            dt = time.perf_counter() - t0
            how = "numpy stable sort (one thread)"
        cpu = {"value": round(m / dt / 1e6, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the first {m} values of {args.workload}, one run, {how}"}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": args.workload + (f"@{args.scale:g}" if args.scale != 1.0 else ""), "n": n,
                       "index": "u64" if index_u64 else "u32", "coder": f"numeric({NUMERIC[args.workload][0]})",
                       "l2": "flushed by a 256 MiB write before every timed step",
                       "parallelism": "replicas" if world > 1 else "single"},
            "e2e": e2e, "gpu_launches": int(sum(s["launches"] for s in kstats.values())),
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clock_info, "stages": stages}), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---- reference arm: the oracle on the host cores --------------------------------

def run_reference(args, rank, world, local):
    if rank != 0:
        return
    import oracle
    import workloads
    threads = os.cpu_count() or 1
    if args.workload in NUMERIC:
        kind = NUMERIC[args.workload][0]
        if kind in BYTES_KINDS:
            bw = bytes_workload(kind, max(2, int(NUMERIC[args.workload][1] * args.scale)), NUMERIC[args.workload][2])
            m = min(bw.offsets.size - 1, 1_000_000 if kind == "bigint" else 300_000)
            fn = oracle.bigint_argsort if kind == "bigint" else oracle.bigdecimal_argsort
            sort = lambda: fn(bw.bytes, bw.offsets[: m + 1])
            v = np.zeros(bw.offsets.size - 1)
        else:
            v, t = numeric_values(args.workload, args.scale)
            m = min(v.size, CPU_SAMPLE_MAX)
            sort = lambda: oracle.numeric_argsort(v[:m], t)
        times = []
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            sort()
            if k >= args.warmup:
                times.append(time.perf_counter() - t0)
        ms = sum(times) / len(times) * 1e3
        value = m / (ms / 1e3) / 1e6
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": args.workload + (f"@{args.scale:g}" if args.scale != 1.0 else ""), "n": int(v.size),
                       "mode": "oracle", "index": "u32", "parallelism": "host (numpy, one thread)"},
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"the first {m} values of {args.workload} each step"},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
            flush=True)
        return
    if workloads.STANDARD[args.workload]["kind"] != 4:
        # single sorts: only the sampled prefix is generated (the same strings
        # as the workload's first ones)
        w, full_n = _prefix(args.workload, args.scale, CPU_SAMPLE_MAX)
    else:
        w = workloads.standard(args.workload, scale=args.scale)
        full_n = w.n
    if w.seg_offsets is not None:   # batched: the leading instances up to the sample bound
        k = 1
        while k < len(w.seg_offsets) - 1 and int(w.seg_offsets[k + 1]) <= CPU_SAMPLE_MAX:
            k += 1
        cut = int(w.seg_offsets[k])
        sort = lambda: oracle.stable_argsort_batched(w.bytes, w.offsets[: cut + 1], w.seg_offsets[: k + 1],
                                                     threads=threads)
        n = cut
    else:
        sw = _sample(w, CPU_SAMPLE_MAX)
        index_u64 = (args.index or ("u64" if args.workload.startswith("skewed") else "u32")) == "u64"
        sort = lambda: oracle.stable_argsort(sw.bytes, sw.offsets, index_u64=index_u64, threads=threads)
        n = sw.n
    for _ in range(args.warmup):
        sort()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        sort()
        times.append(time.perf_counter() - t0)
    ms = sum(times) / len(times) * 1e3
    value = n / (ms / 1e3) / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": args.workload + (f"@{args.scale:g}" if args.scale != 1.0 else ""),
                   "n": full_n, "sample_bytes": int(w.bytes.size), "mode": "oracle",
                   "index": ("u64" if (w.seg_offsets is None and (args.index or (
                       "u64" if args.workload.startswith("skewed") else "u32")) == "u64") else "u32"),
                   "parallelism": "host threads"},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": (f"the full {args.workload} workload each step" if n == full_n else
                                    f"the first {n} strings of {args.workload} each step")},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world, local)
    elif args.workload in NUMERIC:
        run_numeric(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
