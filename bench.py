#!/usr/bin/env python
"""Benchmark of the nsort plain sort on GB300.

One step = one full sort (tile sort + every merge pass) of 2^28 uniform
uint32 keys (seed = rank), inputs resident in HBM, output to a separate
buffer.  Inputs (1 GiB) are larger than L2, so no flush between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nsort|reference]

N > 1 runs under torchrun: every rank sorts its own array (replicas; the
plain sort has no exchange step), timing is the max over ranks and `value`
counts the keys of all ranks.  Rank 0 prints one JSON line.

`--impl reference` times the CPU oracle (a plain bottom-up merge sort) on the
host cores, on a bounded sample of the same workload each step.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GKeys/s & % HBM roofline, 2^28 u32 on 1 GB300"
UNIT = "GKeys/s"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "source": "fallback"}
REFERENCE_SAMPLE_LOG2 = 22       # keys per oracle step in --impl reference
CPU_BASELINE_LOG2 = 22           # keys per oracle repetition in cpu_baseline
CPU_BASELINE_SECONDS = 12.0      # bounded CPU work for cpu_baseline


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["nsort", "reference"], default="nsort")
    ap.add_argument("--log2n", type=int, default=28)
    ap.add_argument("--dtype", choices=["u32", "i32", "f32"], default="u32")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


# ---- distributed plumbing ----------------------------------------------------

def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- clocks ------------------------------------------------------------------

CLOCK_FIELDS = ["uuid", "clocks.sm", "clocks.max.sm", "power.draw", "utilization.gpu",
                "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
                "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed
    region (read-only queries)."""

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + ",".join(CLOCK_FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) != len(CLOCK_FIELDS):
                continue
            if self.uuid and parts[0] != self.uuid:
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(s):
            try:
                return float(s)
            except ValueError:
                return float("nan")
        load = [r for r in rows if num(r[4]) >= 50] or rows
        sm = [num(r[1]) for r in load]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in load:
            for i, nm in enumerate(names):
                if r[5 + i].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.nanmedian(sm)), "sm_max_mhz": num(load[0][2]),
                "samples": len(rows), "samples_under_load": len(load),
                "power_w_max": float(np.nanmax([num(r[3]) for r in load])),
                "reasons": sorted(reasons)}


# ---- roofline inputs -----------------------------------------------------------

def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return dict(FALLBACK_PEAKS)


def source_hash(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(kernel: str):
    """Per-key DRAM bytes of `kernel` from the committed ncu summary, or None
    when the kernel's sources changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel)
    if not d:
        return None
    if source_hash(d["sources"]) != d["source_sha"]:
        return None
    return d


# ---- CPU oracle timing ---------------------------------------------------------

def time_oracle(bits: np.ndarray, dtype: str, seconds: float):
    import oracle
    oracle.build()
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.sort_keys(bits, dtype)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return reps, el


def cpu_baseline(dtype: str):
    from paper_2409_03970_gb300 import inputs
    n = 1 << CPU_BASELINE_LOG2
    x = inputs.keys(n, dtype, "uniform", seed=0)
    reps, el = time_oracle(x, dtype, CPU_BASELINE_SECONDS)
    return {"value": reps * n / el / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first 2^{CPU_BASELINE_LOG2} keys of the workload (uniform {dtype}, "
                      f"seed 0), sorted {reps} times in {el:.1f} s by the single-threaded "
                      f"oracle; host has {len(os.sched_getaffinity(0))} cores"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2409_03970_gb300 import inputs
    n = 1 << REFERENCE_SAMPLE_LOG2
    x = inputs.keys(n, args.dtype, "uniform", seed=0)
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle.sort_keys(x, args.dtype)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sort_keys(x, args.dtype)
    el = time.perf_counter() - t0
    ms = el * 1e3 / args.steps
    value = n / (ms / 1e3) / 1e9
    sample = (f"each step sorts the first 2^{REFERENCE_SAMPLE_LOG2} keys of the workload "
              f"(uniform {args.dtype}, seed 0) with the single-threaded CPU oracle; host has "
              f"{len(os.sched_getaffinity(0))} cores")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": f"plain sort, 2^{args.log2n} {args.dtype} keys, uniform, seed 0 "
                               f"(oracle on a 2^{REFERENCE_SAMPLE_LOG2}-key sample per step)",
                   "n": 1 << args.log2n, "sample_n": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---- the GPU benchmark -----------------------------------------------------------

def main():
    args = parse()
    rank, local_rank, world = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    from paper_2409_03970_gb300 import build as nbuild
    from paper_2409_03970_gb300 import inputs, nsort

    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    nbuild.build()
    nsort.lib()

    n = 1 << args.log2n
    code = {"u32": nsort.U32, "i32": nsort.I32, "f32": nsort.F32}[args.dtype]
    bits = inputs.keys(n, args.dtype, "uniform", seed=rank)
    host_in = torch.from_numpy(bits.view(np.int32)).pin_memory()
    del bits
    x = host_in.cuda()
    out = torch.empty_like(x)
    tmp = nsort.scratch(nsort.KIND_KEYS, n)
    passes, sort_tile, merge_tile = nsort.nsort_plan(nsort.KIND_KEYS, n)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    def step():
        rc = nsort.nsort_keys(x, out, n, code, tmp, tmp.numel(), sh)
        if rc != nsort.OK:
            raise nsort.NsortError(rc, "nsort_keys")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local_rank).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    nsort.nsort_trace_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    trace = nsort.nsort_trace_read()
    nsort.nsort_trace_enable(False)
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    value = world * n / (ms / 1e3) / 1e9

    peaks = load_peaks()
    alg_bytes_sort = passes * 8 * n                      # every pass reads and writes 4 B/key
    sort_frac = alg_bytes_sort / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]
    mk = trace.get("merge_keys")
    roofline = None
    if mk:
        per_launch_ms = mk["total_ms"] / mk["launches"]
        achieved = 8 * n / (per_launch_ms / 1e3) / 1e9
        tr = load_traffic("merge_keys")
        roofline = {"bound": "hbm", "kernel": "merge_keys", "achieved": achieved,
                    "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                    "peak_source": peaks["source"],
                    "traffic": (tr["bytes_per_key"] * n) if tr else None,
                    "algorithmic_bytes": 8 * n, "launch_ms": per_launch_ms,
                    "share_of_step": mk["total_ms"] / (ms * args.steps)}
    launches = sum(v["launches"] for v in trace.values()) // args.steps

    e2e = None
    if not args.no_e2e:
        host_out = torch.empty_like(host_in).pin_memory()
        ke = max(3, min(args.steps, 20))
        for _ in range(2):
            x.copy_(host_in, non_blocking=True)
            step()
            host_out.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        barrier(world)
        e0.record(stream)
        for _ in range(ke):
            x.copy_(host_in, non_blocking=True)
            step()
            host_out.copy_(out, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ems = max_over_ranks(e0.elapsed_time(e1) / ke, world)
        e2e = {"value": world * n / (ems / 1e3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * n, "ms_per_step": ems,
               "steps": ke}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.dtype)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": f"plain sort, 2^{args.log2n} {args.dtype} keys, uniform, "
                                   f"seed = rank; replicas (one array per GPU)",
                       "n": n, "passes": passes, "sort_tile": sort_tile, "merge_tile": merge_tile,
                       "l2": "inputs (1 GiB) larger than L2; no flush",
                       "sort_hbm_roofline_frac": sort_frac,
                       "sort_algorithmic_bytes": alg_bytes_sort,
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches * args.steps,
            "kernels": {k: {"launches": v["launches"], "ms_per_launch": v["total_ms"] / v["launches"]}
                        for k, v in trace.items()},
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
