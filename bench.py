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
import collections
import gc
import glob
import hashlib
import json
import os
import re
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
    ap.add_argument("--dtype", choices=["u32", "i32", "f32", "u64", "i64", "f64"], default="u32")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched (segmented) and served measurements")
    ap.add_argument("--workload", choices=["plain", "segmented", "served", "ablation", "sharded"],
                    default="plain",
                    help="plain: the headline line (with batched/served extras); segmented / "
                         "served: that measurement alone, as its own line")
    ap.add_argument("--served-duration", type=float, default=60.0,
                    help="seconds of Poisson arrivals in the served measurement (60 = the stated workload)")
    ap.add_argument("--segments", type=int, default=100_000)
    ap.add_argument("--merge-ways", type=int, choices=[2, 4], default=2,
                    help="merge levels per pass over the array for 32-bit keys: 2 = one level "
                         "(the library's default), 4 = two levels (four-way passes)")
    ap.add_argument("--no-numa-bind", action="store_true",
                    help="do not restrict the process to the GPU's NUMA node")
    return ap.parse_args()


# ---- distributed plumbing ----------------------------------------------------

def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest x over all ranks (the slowest rank's time).  device is
    where the one-element reduction tensor lives: "cuda" under NCCL, "cpu"
    under gloo."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(ms_local: float, n_per_rank: int, world: int,
                       device: str = "cuda") -> tuple[float, float]:
    """Whole-job rate of `world` replicas that each sorted n_per_rank keys in
    ms_local milliseconds: (max-over-ranks ms, GKeys/s of all ranks over that
    time)."""
    ms = max_over_ranks(ms_local, world, device)
    return ms, world * n_per_rank / (ms / 1e3) / 1e9


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
    """Hash of the code in `files` with comments and blank lines left out:
    an edit to a comment leaves the kernels, and so their traffic, as they
    were; any other edit changes the hash."""
    h = hashlib.sha256()
    for f in files:
        text = open(os.path.join(ROOT, f), encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("\n".join(l.rstrip() for l in text.splitlines() if l.strip()).encode())
    return h.hexdigest()[:16]


def load_traffic(kernel: str):
    """DRAM bytes read and written by one launch of `kernel`, from the
    committed ncu capture (profiles/traffic.json: captured_n, read_bytes,
    write_bytes), or None when the kernel's sources changed since the
    counters were taken."""
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

WIDE = ("u64", "i64", "f64")


def sample_keys(n: int, dtype: str, seed: int = 0) -> np.ndarray:
    """Uniform keys of the plain workload: uint32 patterns, or uint64 ones
    for the 64-bit dtypes."""
    from paper_2409_03970_gb300 import inputs
    if dtype in WIDE:
        return inputs.keys64(n, dtype, "uniform", seed=seed)
    return inputs.keys(n, dtype, "uniform", seed=seed)


def oracle_sort(bits: np.ndarray, dtype: str):
    import oracle
    return oracle.sort_keys64(bits, dtype) if dtype in WIDE else oracle.sort_keys(bits, dtype)


def time_oracle(bits: np.ndarray, dtype: str, seconds: float):
    import oracle
    oracle.build()
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle_sort(bits, dtype)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return reps, el


def parallel_oracle_rate(x: np.ndarray, dtype: str, threads: int, seconds: float):
    """Keys/s of the oracle's multi-threaded form on `threads` host threads
    (32-bit dtypes only)."""
    import oracle
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.sort_keys_par(x, dtype, threads)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return reps * x.size / el


def cpu_baseline(dtype: str):
    from paper_2409_03970_gb300 import inputs
    n = 1 << CPU_BASELINE_LOG2
    x = sample_keys(n, dtype)
    reps, el = time_oracle(x, dtype, CPU_BASELINE_SECONDS)
    cores = len(os.sched_getaffinity(0))
    line = {"value": reps * n / el / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first 2^{CPU_BASELINE_LOG2} keys of the workload (uniform {dtype}, "
                      f"seed 0), sorted {reps} times in {el:.1f} s by the single-threaded "
                      f"oracle; host has {cores} cores"}
    if dtype not in WIDE:
        # context: the same sort on every host core (chunk sorts, then pairwise
        # merges); never allowed to break the line
        try:
            rate = parallel_oracle_rate(x, dtype, cores, CPU_BASELINE_SECONDS / 2)
            line["parallel"] = {"value": rate / 1e9, "unit": UNIT, "cores": cores,
                                "kind": "oracle, multi-threaded: chunk sorts, then pairwise "
                                        "merges (context, not the baseline)"}
        except Exception as e:   # noqa: BLE001
            line["parallel"] = {"error": str(e)[:200]}
    return line


def run_reference(args, rank, world):
    if rank != 0:
        return
    n = 1 << REFERENCE_SAMPLE_LOG2
    x = sample_keys(n, args.dtype)
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle_sort(x, args.dtype)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_sort(x, args.dtype)
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


def bind_to_gpu_numa_node(torch, dev: int):
    """Restricts this process to the CPUs of the GPU's NUMA node (when sysfs
    names one and it overlaps the allowed CPUs), so that pinned host buffers
    allocated afterwards sit next to the GPU.  Returns the node or None."""
    try:
        pr = torch.cuda.get_device_properties(dev)
        bdf = f"{pr.pci_domain_id:04x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
        node = int(open(f"/sys/bus/pci/devices/{bdf}/numa_node").read().strip())
        if node < 0:
            return None
        cpus = set()
        for part in open(f"/sys/devices/system/node/node{node}/cpulist").read().strip().split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        allowed = cpus & os.sched_getaffinity(0)
        if not allowed:
            return None
        os.sched_setaffinity(0, allowed)
        return node
    except (OSError, ValueError, AttributeError):
        return None


def copy_bandwidths(torch, host, dev_a, dev_b, reps: int = 3):
    """GB/s of a host-to-device copy of `host` (pinned) into dev_a alone, a
    device-to-host copy of dev_b alone, and of both at once on two streams:
    the best of `reps` repeats each (what the link sustains, not one sample
    that another process on the host happened to slow down)."""
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    back = torch.empty_like(host).pin_memory()
    nbytes = host.numel() * host.element_size()
    res = {}
    for name in ("h2d", "d2h", "both"):
        best = 0.0
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(s1)
            s2.wait_event(a)
            if name in ("h2d", "both"):
                with torch.cuda.stream(s1):
                    dev_a.copy_(host, non_blocking=True)
            if name in ("d2h", "both"):
                with torch.cuda.stream(s2):
                    back.copy_(dev_b, non_blocking=True)
            s1.wait_stream(s2)
            b.record(s1)
            torch.cuda.synchronize()
            gbs = (2 if name == "both" else 1) * nbytes / (a.elapsed_time(b) / 1e3) / 1e9
            best = max(best, gbs)
        res[name + "_gbs"] = best
    return res


def bench_e2e(nsort, torch, host_in, x, out, tmp, n, code, steps, world, esize=4):
    """The same sort through the public API with HOST buffers: every step
    copies its input from pinned host memory, sorts, and copies the result
    back to pinned host memory.  Pipelined over three streams with three
    device arrays per direction, so the upload of step i+1 and the download
    of step i-1 overlap the sort of step i (the way a stream of host arrays
    is sorted) and neither copy waits on the other's buffer; the unpipelined
    time of one step is reported beside it."""
    ke = max(3, min(steps, 50))     # fill and drain of the pipeline amortised over the steps
    NB = 3                          # device buffers per direction
    h2d, comp, d2h = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    din = [x] + [torch.empty_like(x) for _ in range(NB - 1)]
    dout = [out] + [torch.empty_like(out) for _ in range(NB - 1)]
    hout = [torch.empty_like(host_in).pin_memory() for _ in range(NB)]
    ev = lambda: torch.cuda.Event(enable_timing=False)
    up, sorted_, down = [ev() for _ in range(NB)], [ev() for _ in range(NB)], [ev() for _ in range(NB)]
    tev = lambda: torch.cuda.Event(enable_timing=True)
    # per-step timing events, read after the loop: upload, sort, download
    marks = [[tev() for _ in range(6)] for _ in range(NB + ke)]
    torch.cuda.synchronize()

    def step(i):
        b = i % NB
        m = marks[i]
        if i >= NB:
            h2d.wait_event(sorted_[b])        # din[b] no longer read by step i-NB
        with torch.cuda.stream(h2d):
            m[0].record(h2d)
            din[b].copy_(host_in, non_blocking=True)
            m[1].record(h2d)
            up[b].record(h2d)
        comp.wait_event(up[b])
        if i >= NB:
            comp.wait_event(down[b])          # dout[b] downloaded by step i-NB
        m[2].record(comp)
        rc = nsort.nsort_keys(din[b], dout[b], n, code, tmp, tmp.numel(), comp.cuda_stream)
        if rc != nsort.OK:
            raise nsort.NsortError(rc, "nsort_keys")
        m[3].record(comp)
        sorted_[b].record(comp)
        d2h.wait_event(sorted_[b])
        with torch.cuda.stream(d2h):
            m[4].record(d2h)
            hout[b].copy_(dout[b], non_blocking=True)
            m[5].record(d2h)
            down[b].record(d2h)

    for i in range(NB):
        step(i)
    torch.cuda.synchronize()
    barrier(world)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(h2d)
    for i in range(NB, NB + ke):
        step(i)
    t1.record(d2h)
    torch.cuda.synchronize()
    barrier(world)
    ems, e2e_value = replica_throughput(t0.elapsed_time(t1) / ke, n, world)
    stages = {name: float(np.mean([marks[i][2 * j].elapsed_time(marks[i][2 * j + 1])
                                   for i in range(NB, NB + ke)]))
              for j, name in enumerate(("upload_ms", "sort_ms", "download_ms"))}
    # one step alone, start to finish (no overlap between steps); the best
    # of three, as for the copy bandwidths
    serial_ms = float("inf")
    for _ in range(3):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(comp)
        with torch.cuda.stream(comp):
            din[0].copy_(host_in, non_blocking=True)
            nsort.nsort_keys(din[0], dout[0], n, code, tmp, tmp.numel(), comp.cuda_stream)
            hout[0].copy_(dout[0], non_blocking=True)
        s1.record(comp)
        torch.cuda.synchronize()
        serial_ms = min(serial_ms, s0.elapsed_time(s1))
    bw = copy_bandwidths(torch, host_in, din[1], dout[1])
    return {"value": e2e_value, "unit": UNIT, "copy_bandwidths": bw,
            "stages_in_pipeline": stages,
            "h2d_bytes_per_step": esize * n, "d2h_bytes_per_step": esize * n, "ms_per_step": ems,
            "steps": ke, "pipelined": f"3 streams, {NB} device arrays per direction",
            "one_step_unpipelined_ms": serial_ms}


def time_sort(nsort, torch, fn, reps: int = 5, warm: int = 2):
    """Device time of fn() (one sort), median of `reps` after `warm` runs."""
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def bench_configs(nsort, torch):
    """The other plain-sort configurations: 2^28 int32 / float32 keys over
    the five distributions (uniform, sorted, reverse, 16 distinct, Zipf), 2^27 stable float32 key / uint32 value pairs
    (Normal(0,1) with 0.1% IEEE specials, payload = index), the same keys
    with 64-bit payloads, and 2^27 64-bit keys."""
    from paper_2409_03970_gb300 import inputs
    n = 1 << 28
    out = {}
    tmp = nsort.scratch(nsort.KIND_KEYS, n)
    ko = torch.empty(n, dtype=torch.int32, device="cuda")
    for dt, dist in [(d, x) for d in ("i32", "f32") for x in inputs.DISTRIBUTIONS]:
        x = torch.from_numpy(inputs.keys(n, dt, dist, seed=0).view(np.int32)).cuda()
        code = {"i32": nsort.I32, "f32": nsort.F32}[dt]
        ms = time_sort(nsort, torch,
                       lambda: nsort.nsort_keys(x, ko, n, code, tmp, tmp.numel()))
        out[f"keys_{dt}_{dist}_2e28"] = {"ms": ms, "gkeys_s": n / ms / 1e6}
        del x
    del tmp, ko
    torch.cuda.empty_cache()
    # the small plain case: 2^20 uniform uint32 keys, seed 0 (launch-latency bound)
    s = 1 << 20
    x = torch.from_numpy(inputs.keys(s, "u32", "uniform", seed=0).view(np.int32)).cuda()
    y = torch.empty_like(x)
    tmp = nsort.scratch(nsort.KIND_KEYS, s)
    ms = time_sort(nsort, torch, lambda: nsort.nsort_keys(x, y, s, nsort.U32, tmp, tmp.numel()),
                   reps=51, warm=5)
    out["keys_u32_uniform_2e20"] = {"ms": ms, "gkeys_s": s / ms / 1e6,
                                    "l2": "inputs fit in L2 (4 MiB): not an HBM measurement"}
    del x, y, tmp
    m = 1 << 27
    k, v = inputs.normal_pairs(m, seed=0)
    kt = torch.from_numpy(k.view(np.int32)).cuda()
    vt = torch.from_numpy(v.view(np.int32)).cuda()
    del k, v
    kout, vout = torch.empty_like(kt), torch.empty_like(vt)
    tmp = nsort.scratch(nsort.KIND_PAIRS, m)
    passes, _, _ = nsort.nsort_plan(nsort.KIND_PAIRS, m)
    ms = time_sort(nsort, torch, lambda: nsort.nsort_pairs(kt, vt, kout, vout, m, nsort.F32, tmp,
                                                           tmp.numel()))
    out["pairs_f32_normal_specials_2e27"] = {
        "ms": ms, "gpairs_s": m / ms / 1e6, "passes": passes,
        "hbm_roofline_frac": passes * 16 * m / (ms / 1e3) / 1e9 / load_peaks()["hbm_gbs"]}
    del vt, vout, tmp
    torch.cuda.empty_cache()
    # the same keys with 64-bit payloads (nsort_pairs64): 24 B per pair per pass
    vt = torch.arange(m, dtype=torch.int64, device="cuda")
    vout = torch.empty_like(vt)
    tmp = nsort.scratch(nsort.KIND_PAIRS64, m)
    ms = time_sort(nsort, torch, lambda: nsort.nsort_pairs64(kt, vt, kout, vout, m, nsort.F32, tmp,
                                                             tmp.numel()))
    out["pairs64_f32_normal_specials_2e27"] = {
        "ms": ms, "gpairs_s": m / ms / 1e6, "passes": passes,
        "hbm_roofline_frac": passes * 24 * m / (ms / 1e3) / 1e9 / load_peaks()["hbm_gbs"]}
    del kt, vt, kout, vout, tmp
    torch.cuda.empty_cache()
    out.update(bench_keys64(nsort, torch))
    return out


def bench_keys64(nsort, torch):
    """64-bit keys (the wider-key variant): 2^27 uint64 / int64 / float64 keys
    (1 GiB), 16 B per key per pass; the merge pass's own roofline from its
    traced launches."""
    from paper_2409_03970_gb300 import inputs
    m = 1 << 27
    peak = load_peaks()["hbm_gbs"]
    tmp = nsort.scratch(nsort.KIND_KEYS, m, dtype=nsort.U64)
    ko = torch.empty(m, dtype=torch.int64, device="cuda")
    passes, _, _ = nsort.nsort_plan(nsort.KIND_KEYS, m, nsort.U64)
    codes = {"u64": nsort.U64, "i64": nsort.I64, "f64": nsort.F64}
    out = {}
    for dt, dist in (("u64", "uniform"), ("i64", "uniform"), ("f64", "uniform"),
                     ("f64", "specials")):
        x = torch.from_numpy(inputs.keys64(m, dt, dist, seed=0).view(np.int64)).cuda()
        code = codes[dt]
        fn = lambda: nsort.nsort_keys(x, ko, m, code, tmp, tmp.numel())
        ms = time_sort(nsort, torch, fn)
        nsort.nsort_trace_enable(True)            # launch durations from a traced repeat
        time_sort(nsort, torch, fn, reps=3, warm=0)
        tr = nsort.nsort_trace_read()
        nsort.nsort_trace_enable(False)
        r = {"ms": ms, "gkeys_s": m / ms / 1e6, "passes": passes,
             "hbm_roofline_frac": passes * 16 * m / (ms / 1e3) / 1e9 / peak}
        mk = tr.get("merge_keys64")
        if mk and mk["launches"]:
            lms = mk["total_ms"] / mk["launches"]
            r["merge_keys64_ms"] = lms
            r["merge_keys64_frac"] = 16 * m / (lms / 1e3) / 1e9 / peak
        ts = tr.get("tile_sort_keys64")
        if ts and ts["launches"]:
            r["tile_sort_keys64_ms"] = ts["total_ms"] / ts["launches"]
        out[f"keys_{dt}_{dist}_2e27"] = r
        del x
    del tmp, ko
    torch.cuda.empty_cache()
    return out


# ---- batched (segmented) and served measurements -----------------------------

def bench_merge_ways(nsort, torch):
    """Plain sorts of uniform u32 keys with one merge level per pass over
    the array (two-way passes, the default) and with two (four-way passes):
    ms per sort at 2^20 to 2^28."""
    from paper_2409_03970_gb300 import inputs
    res = {}
    for log2n in (20, 22, 24, 26, 28):
        n = 1 << log2n
        x = torch.from_numpy(inputs.keys(n, "u32", "uniform", seed=0).view(np.int32)).cuda()
        y = torch.empty_like(x)
        row = {}
        for ways, setting in ((2, nsort.FOUR_WAY_NEVER), (4, 0)):
            prev = nsort.nsort_testing_set_four_way_min(setting)
            try:
                tmp = nsort.scratch(nsort.KIND_KEYS, n)
                row[f"{ways}-way_ms"] = time_sort(
                    nsort, torch, lambda: nsort.nsort_keys(x, y, n, nsort.U32, tmp, tmp.numel()),
                    reps=11, warm=3)
                del tmp
            finally:
                nsort.nsort_testing_set_four_way_min(prev)
        res[f"2^{log2n}"] = row
        del x, y
        torch.cuda.empty_cache()
    return {"unit": "ms per sort", "table": res}


def bench_ablation(nsort, torch):
    """Column-network, keys-per-thread and merger ablation (Tables 1-3).

    in_register: GKeys/s of producing sorted runs of X keys (column sort
    with IPT keys per thread, then log2(X / IPT) warp merge levels) on 2^23
    u32 keys that stay in L2 between repetitions (64 MiB in + out), as the
    paper times its in-register sort on cache-resident data.  block_sort:
    GKeys/s of the whole block sort (tiles of 512 * IPT keys) on 2^26 keys
    (256 MiB, larger than L2), the production tile sort being best / 16.
    mergers: GKeys/s of merging sorted runs of L into 2L with the hybrid,
    all-shuffle and serial merge-path mergers (Table 3), 2^23 keys in L2."""
    from paper_2409_03970_gb300 import inputs
    fams = {"best": nsort.NET_BEST, "oddeven": nsort.NET_ODDEVEN, "bitonic": nsort.NET_BITONIC}
    ipts = (4, 8, 16, 32)
    out = {"comparators": {f: {w: len(nsort.nsort_network(c, w)) for w in ipts}
                           for f, c in fams.items()}}

    def table(n, runs_of, reps):
        x = torch.from_numpy(inputs.keys(n, "u32", "uniform", seed=21).view(np.int32)).cuda()
        y = torch.empty_like(x)
        res = {}
        for f, c in fams.items():
            res[f] = {}
            for ipt in ipts:
                res[f][ipt] = {}
                for run in runs_of(ipt):
                    def fn(run=run, ipt=ipt, c=c):
                        rc = nsort.nsort_runs(x, y, n, c, ipt, run)
                        if rc != nsort.OK:
                            raise nsort.NsortError(rc, "nsort_runs")
                    ms = time_sort(nsort, torch, fn, reps=reps, warm=3)
                    res[f][ipt][run] = n / (ms / 1e3) / 1e9
        del x, y
        return res

    n_reg = 1 << 23
    out["in_register"] = {"n": n_reg, "unit": "GKeys/s", "l2": "resident (64 MiB in + out)",
                          "table": table(n_reg, lambda ipt: [ipt << l for l in range(6)], 21)}
    # Table 3: merge two sorted runs of L into 2L, by merger and keys per thread
    x = torch.from_numpy(inputs.keys(n_reg, "u32", "uniform", seed=22).view(np.int32)).cuda()
    y = torch.empty_like(x)
    mergers = {"hybrid": nsort.MERGE_HYBRID, "shuffle": nsort.MERGE_SHUFFLE,
               "serial": nsort.MERGE_SERIAL}
    mt = {}
    for L in (8, 16, 32, 64, 128, 256):
        rc = nsort.nsort_runs(x, x, n_reg, nsort.NET_BEST, 4, L) if L <= 128 else \
            nsort.nsort_runs(x, x, n_reg, nsort.NET_BEST, 8, L)
        if rc != nsort.OK:
            raise nsort.NsortError(rc, "nsort_runs")
        mt[f"2x{L}"] = {}
        for m, code in mergers.items():
            mt[f"2x{L}"][m] = {}
            for ipt in ipts:
                if L not in nsort.merge_run_lengths(code, ipt):
                    continue

                def fn(L=L, code=code, ipt=ipt):
                    rc = nsort.nsort_merge_runs(x, y, n_reg, L, code, ipt)
                    if rc != nsort.OK:
                        raise nsort.NsortError(rc, "nsort_merge_runs")
                ms = time_sort(nsort, torch, fn, reps=21, warm=3)
                mt[f"2x{L}"][m][ipt] = n_reg / (ms / 1e3) / 1e9
    del x, y
    out["mergers"] = {"n": n_reg, "unit": "GKeys/s", "l2": "resident (64 MiB in + out)",
                      "table": mt}
    out["merge_ways"] = bench_merge_ways(nsort, torch)
    n_blk = 1 << 26
    blk = table(n_blk, lambda ipt: [512 * ipt], 11)
    out["block_sort"] = {"n": n_blk, "unit": "GKeys/s", "l2": "inputs (256 MiB) larger than L2",
                         "table": {f: {ipt: v[512 * ipt] for ipt, v in t.items()}
                                   for f, t in blk.items()}}
    return out


def bench_batched(nsort, torch, nseg: int, reps: int = 5):
    """100,000 uint32 arrays (lengths log-uniform in [1, 65536], uniform keys)
    sorted by one graph-captured nsort_segmented launch with the autotuned
    configuration, against one plain nsort_keys call per array."""
    from paper_2409_03970_gb300 import autotune, inputs
    off = inputs.segment_offsets(nseg, seed=0)
    total = int(off[-1])
    keys = inputs.keys(total, "u32", "uniform", seed=0)
    kt = torch.from_numpy(keys.view(np.int32)).cuda()
    del keys
    ot = torch.from_numpy(off).cuda()
    ko = torch.empty_like(kt)
    t0 = time.perf_counter()
    tune = autotune.tune_segmented(kt, ot, reps=2)
    tune_s = time.perf_counter() - t0
    tmp = nsort.scratch(nsort.KIND_SEGMENTED, total, nseg)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(2):
            assert nsort.nsort_segmented(kt, ko, None, None, ot, nseg, total, nsort.U32, tmp,
                                         tmp.numel(), s) == nsort.OK
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        nsort.nsort_segmented(kt, ko, None, None, ot, nseg, total, nsort.U32, tmp, tmp.numel(), s)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g.replay()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1) / reps
    assert nsort.nsort_device_status(tmp) == nsort.OK
    batched_out = ko.clone()
    # one plain launch (nsort_keys) per array, on one stream
    lens = np.diff(off)
    ptmp = nsort.scratch(nsort.KIND_KEYS, int(lens.max()))
    pb = ptmp.numel()
    st = torch.cuda.current_stream()
    sh = st.cuda_stream
    kin, kout = kt.data_ptr(), ko.data_ptr()
    lib = nsort.lib()
    offs = off.tolist()
    ms_p = []
    for _ in range(2):
        torch.cuda.synchronize()
        e0.record(st)
        for i in range(nseg):
            o, L = offs[i], offs[i + 1] - offs[i]
            lib.nsort_keys(kin + 4 * o, kout + 4 * o, L, 0, ptmp.data_ptr(), pb, sh)
        e1.record(st)
        torch.cuda.synchronize()
        ms_p.append(e0.elapsed_time(e1))
    same = bool(torch.equal(batched_out, ko))
    return {"metric": "GKeys/s", "workload": f"{nseg} uint32 arrays, lengths log-uniform in "
            f"[1, 65536], {total} keys, uniform, seed 0",
            "batched_gkeys_s": total / ms_b / 1e6, "batched_ms": ms_b,
            "plain_per_array_gkeys_s": total / min(ms_p) / 1e6, "plain_per_array_ms": min(ms_p),
            "speedup": min(ms_p) / ms_b, "identical_results": same,
            "launch": "one graph-captured nsort_segmented: 3 set-up kernels, 1 persistent kernel (level-0 tiles and short segments), then 3 kernels per merge level (tile list, partition, persistent bulk-copy merge)",
            "autotuned_config": tune["config"], "autotune_seconds": tune_s,
            "candidates": len(tune["table"])}


def bench_sharded(nsort, torch, nshards: int = 8, log2n: int = 28):
    """The sharded sort's steps on one GPU: 2^28 uniform u32 keys cut into
    `nshards` equal shards.  Device times (CUDA events) of what each GPU of
    an nshards-GPU run does: sort its shard, find the segmentation points
    (here one co-rank kernel over all shards), and merge its part's nshards
    runs; plus the whole one-GPU emulation (every shard sorted, slices
    gathered by device copies, every part merged), checked for order."""
    from paper_2409_03970_gb300 import inputs, shard
    n = 1 << log2n
    x = torch.from_numpy(inputs.keys(n, "u32", "uniform", seed=0).view(np.int32)).cuda()
    s = [(r * n) // nshards for r in range(nshards + 1)]
    m = s[1] - s[0]
    sk = torch.empty_like(x)
    tmp = nsort.scratch(nsort.KIND_KEYS, max(s[r + 1] - s[r] for r in range(nshards)))
    shard_ms = time_sort(nsort, torch, lambda: nsort.nsort_keys(x[:m], sk[:m], m, nsort.U32, tmp,
                                                                 tmp.numel()))
    for r in range(nshards):
        a, b = s[r], s[r + 1]
        rc = nsort.nsort_keys(x[a:b], sk[a:b], b - a, nsort.U32, tmp, tmp.numel())
        assert rc == nsort.OK
    del tmp
    d = shard.part_bounds(n, nshards)
    off_t = torch.tensor(s, dtype=torch.int64, device="cuda")
    tgt_t = torch.tensor(d, dtype=torch.int64, device="cuda")
    cr = torch.empty((nshards + 1) * nshards, dtype=torch.int64, device="cuda")
    corank_ms = time_sort(nsort, torch, lambda: nsort.nsort_shard_coranks(
        sk, off_t, nshards, tgt_t, nshards + 1, nsort.U32, cr), reps=21, warm=3)
    c = cr.view(nshards + 1, nshards).cpu().numpy()
    # the largest part: its slices gathered back to back, then merged
    q = int(np.argmax(np.diff(d)))
    lens = c[q + 1] - c[q]
    run_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    p = int(run_off[-1])
    rk = torch.empty(p, dtype=torch.int32, device="cuda")
    for r in range(nshards):
        a, b = s[r] + int(c[q][r]), s[r] + int(c[q + 1][r])
        rk[run_off[r]:run_off[r + 1]].copy_(sk[a:b])
    ko = torch.empty_like(rk)
    tmp = nsort.scratch(nsort.KIND_MERGE, p, nshards)
    merge_ms = time_sort(nsort, torch, lambda: nsort.nsort_merge_shards(
        rk, None, ko, None, run_off, nsort.U32, tmp, tmp.numel()))
    passes = max(1, (nshards - 1).bit_length())      # a tree of pairwise passes
    del rk, ko, tmp, sk
    torch.cuda.empty_cache()
    res = {}
    whole_ms = time_sort(nsort, torch, lambda: res.update(
        out=shard.sort_sharded_one_gpu(x, nshards, nsort.U32)[0]), reps=3, warm=1)
    y = res.pop("out")
    ordered = bool((y[1:].view(torch.int32).to(torch.int64) & 0xFFFFFFFF).ge(
        y[:-1].view(torch.int32).to(torch.int64) & 0xFFFFFFFF).all())
    del x, y
    torch.cuda.empty_cache()
    per_gpu = shard_ms + corank_ms + merge_ms
    return {"workload": f"2^{log2n} uniform u32 keys as {nshards} shards of 2^{log2n}/{nshards}",
            "shard_sort_ms": shard_ms, "corank_ms": corank_ms,
            "part_merge_ms": merge_ms, "part_keys": p, "part_runs": nshards,
            "part_merge_gkeys_s": p / merge_ms / 1e6,
            "part_merge_passes": passes,
            "part_merge_hbm_frac": passes * 8 * p / (merge_ms / 1e3) / 1e9 / load_peaks()["hbm_gbs"],
            "per_gpu_compute_ms": per_gpu,
            "one_gpu_emulation_ms": whole_ms, "one_gpu_emulation_ordered": ordered,
            "note": "per_gpu_compute_ms = shard sort + co-ranks + part merge; an "
                    f"{nshards}-GPU run adds the all-to-all exchange and the "
                    "bisection's all-reduces"}


def bench_served(nsort, torch, duration: float, rate: float = 2000.0, budget: int = 64 << 30,
                 streams: int = 8, batch_max_keys: int = 1 << 16, seed: int = 0):
    """Open-loop Poisson arrivals (rate/s for `duration` s), sizes log-uniform
    in [2^10, 2^26], dtype uniform over {u32, i32, f32, f32 key + u32 value},
    against a 64 GB scratch budget.  Latency = completion - scheduled arrival.
    The same schedule runs through the continuous-batching server and through
    plain FIFO sorting (one request at a time, no batching)."""
    from paper_2409_03970_gb300 import inputs
    count = int(rate * duration)
    u = inputs.unit_double(inputs.counter_u64(seed, inputs.S_SERVE, 0, count))
    gaps = -np.log1p(-u) / rate
    arrival = np.cumsum(gaps)
    us = inputs.unit_double(inputs.counter_u64(seed, inputs.S_SERVE + 1, 0, count))
    sizes = np.floor(np.exp2(10 + 16 * us)).astype(np.int64)
    modes = (inputs.counter_u32(seed, inputs.S_SERVE + 2, 0, count) % 4).astype(np.int64)
    starts = (inputs.counter_u64(seed, inputs.S_SERVE + 3, 0, count) %
              np.uint64((1 << 28) - (1 << 26))).astype(np.int64) & ~3
    pool_k = torch.from_numpy(inputs.keys(1 << 28, "u32", "uniform", seed=seed).view(np.int32)).cuda()
    pool_v = torch.arange(1 << 28, dtype=torch.int32, device="cuda")
    ring = 1 << 30
    out_k = torch.empty(ring, dtype=torch.int32, device="cuda")
    out_v = torch.empty(ring, dtype=torch.int32, device="cuda")
    total_keys = int(sizes.sum())
    state = {"count": count, "total_keys": total_keys}

    def run(streams_, batch_):
        count = state["count"]
        total_keys = state["total_keys"]
        due_at = arrival[:count]
        srv = nsort.SortServer(0, budget, streams_, batch_)
        # warm-up: one request of each mode and a small batch
        for m in range(4):
            for n in (1 << 12, 1 << 20):
                kind = nsort.KIND_PAIRS if m == 3 else nsort.KIND_KEYS
                dt = [nsort.U32, nsort.I32, nsort.F32, nsort.F32][m]
                t = nsort.nsort_submit(srv.ctx, kind, dt, n, pool_k, out_k,
                                       pool_v if m == 3 else None, out_v if m == 3 else None)
                srv.wait(t)
        kb, vb = pool_k.data_ptr(), pool_v.data_ptr()
        ob, ovb = out_k.data_ptr(), out_v.data_ptr()
        # the client's own garbage-collector pauses would delay submissions
        # and count as latency: no collection while the stream runs
        gc_on = gc.isenabled()
        gc.collect()
        gc.disable()
        try:
            return timed_stream(srv, kb, vb, ob, ovb, count, total_keys, due_at, streams_, batch_)
        finally:
            if gc_on:
                gc.enable()

    def timed_stream(srv, kb, vb, ob, ovb, count, total_keys, due_at, streams_, batch_):
        tickets = []
        inflight = collections.deque()   # (start, end, ticket) of output regions in use
        rpos = 0
        t0 = time.monotonic()
        for i in range(count):
            n = int(sizes[i])
            if rpos + n > ring:
                rpos = 0
            # an output region is reused only after the request writing it is done
            # (a sort uses its output as working space); latency still counts from
            # the scheduled arrival
            while inflight and inflight[0][0] < rpos + n and inflight[0][1] > rpos:
                srv.wait(inflight.popleft()[2], 600000)
            m = int(modes[i])
            kind = nsort.KIND_PAIRS if m == 3 else nsort.KIND_KEYS
            dt = [nsort.U32, nsort.I32, nsort.F32, nsort.F32][m]
            st = int(starts[i])
            due = t0 + due_at[i]
            while True:
                d = due - time.monotonic()
                if d <= 0:
                    break
                if d > 0.002:
                    time.sleep(d - 0.001)
            tickets.append(nsort.nsort_submit(srv.ctx, kind, dt, n, kb + 4 * st, ob + 4 * rpos,
                                              vb + 4 * st if m == 3 else None,
                                              ovb + 4 * rpos if m == 3 else None))
            inflight.append((rpos, rpos + n, tickets[-1]))
            rpos = (rpos + n + 3) & ~3
        done_t = np.empty(count)
        batched = 0
        for i, t in enumerate(tickets):
            rc = srv.wait(t, 600000)
            if rc != nsort.OK:
                raise nsort.NsortError(rc, "served request")
            _, tm = srv.poll(t)
            done_t[i] = tm["t_done"]
            batched += tm["batched"]
        srv.close()
        lat = (done_t - (t0 + due_at)) * 1e3
        span = done_t.max() - t0
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "max_ms": float(lat.max()),
                "mean_ms": float(lat.mean()), "gkeys_s": total_keys / span / 1e9,
                "makespan_s": float(span), "batched_requests": int(batched),
                "streams": streams_, "batch_max_keys": batch_}

    served = run(streams, batch_max_keys)
    fifo = run(1, 0)
    # saturation: the first 2,000 requests all due at once (closed loop), so
    # keys/s measures capacity rather than the offered load
    arrival_open = arrival.copy()
    sat_n = min(count, 2000)
    arrival[:] = 0.0
    state.update(count=sat_n, total_keys=int(sizes[:sat_n].sum()))
    sat_served = run(streams, batch_max_keys)
    sat_fifo = run(1, 0)
    arrival[:] = arrival_open
    state.update(count=count, total_keys=total_keys)
    return {"workload": f"Poisson arrivals at {rate:g}/s for {duration:g} s ({count} requests, "
                        f"{total_keys} keys), sizes log-uniform in [2^10, 2^26], dtype uniform over "
                        f"u32/i32/f32/f32+u32 pairs, {budget >> 30} GB scratch budget",
            "served": served, "plain_fifo": fifo,
            "p99_speedup": fifo["p99_ms"] / served["p99_ms"],
            "throughput_speedup": served["gkeys_s"] / fifo["gkeys_s"],
            "saturated": {"requests": sat_n, "served_gkeys_s": sat_served["gkeys_s"],
                          "plain_fifo_gkeys_s": sat_fifo["gkeys_s"],
                          "served_p99_ms": sat_served["p99_ms"],
                          "plain_fifo_p99_ms": sat_fifo["p99_ms"],
                          "throughput_speedup": sat_served["gkeys_s"] / sat_fifo["gkeys_s"]},
            "latency": "completion minus scheduled arrival (open loop)"}


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
    numa_node = None if args.no_numa_bind else bind_to_gpu_numa_node(torch, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    nbuild.build()
    nsort.lib()

    if args.workload != "plain":
        if rank == 0:
            if args.workload == "segmented":
                r = bench_batched(nsort, torch, args.segments)
                line = {"metric": "GKeys/s, batched segmented sort vs one plain launch per array",
                        "value": r["batched_gkeys_s"], "unit": "GKeys/s", "n_gpus": 1,
                        "higher_is_better": True, "data": "synthetic", "dtype": "u32",
                        "config": r, "vs_baseline": None}
            elif args.workload == "ablation":
                r = bench_ablation(nsort, torch)
                line = {"metric": "block-sort GKeys/s by column network and keys per thread",
                        "value": r["block_sort"]["table"]["best"][16], "unit": "GKeys/s",
                        "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
                        "dtype": "u32", "config": r, "vs_baseline": None}
            elif args.workload == "sharded":
                r = bench_sharded(nsort, torch)
                line = {"metric": "sharded sort steps on one GPU: per-GPU compute ms of an 8-way split",
                        "value": r["per_gpu_compute_ms"], "unit": "ms", "n_gpus": 1,
                        "higher_is_better": False, "data": "synthetic", "dtype": "u32",
                        "config": r, "vs_baseline": None}
            else:
                r = bench_served(nsort, torch, args.served_duration)
                line = {"metric": "served sort stream: keys/s and p50/p99 latency vs plain FIFO",
                        "value": r["served"]["gkeys_s"], "unit": "GKeys/s", "n_gpus": 1,
                        "higher_is_better": True, "data": "synthetic", "dtype": "mixed",
                        "config": r, "vs_baseline": None}
            print(json.dumps(line), flush=True)
        return

    if args.merge_ways == 4:
        nsort.nsort_testing_set_four_way_min(0)
    n = 1 << args.log2n
    code = {"u32": nsort.U32, "i32": nsort.I32, "f32": nsort.F32,
            "u64": nsort.U64, "i64": nsort.I64, "f64": nsort.F64}[args.dtype]
    wide = args.dtype in WIDE
    esize = 8 if wide else 4                              # bytes per key
    bits = sample_keys(n, args.dtype, seed=rank)
    host_in = torch.from_numpy(bits.view(np.int64 if wide else np.int32)).pin_memory()
    del bits
    x = host_in.cuda()
    out = torch.empty_like(x)
    tmp = nsort.scratch(nsort.KIND_KEYS, n, dtype=code)
    passes, sort_tile, merge_tile = nsort.nsort_plan(nsort.KIND_KEYS, n, code)
    mk_name = "merge_keys64" if wide else ("merge4_keys" if args.merge_ways == 4 else "merge_keys")
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
    ms, value = replica_throughput(e0.elapsed_time(e1) / args.steps, n, world)
    # per-kernel durations: the same steps once more with the library's
    # tracing on (CUDA events around every launch on its stream).  Tracing
    # puts events between the kernels, which costs time and undoes the
    # overlapped launches, so the step time above is taken without it.
    nsort.nsort_trace_enable(True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    traced_ms = e0.elapsed_time(e1) / args.steps
    trace = nsort.nsort_trace_read()
    nsort.nsort_trace_enable(False)

    peaks = load_peaks()
    alg_bytes_sort = passes * 2 * esize * n              # every pass reads and writes each key
    sort_frac = alg_bytes_sort / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]
    mk = trace.get(mk_name)
    roofline = None
    if mk:
        per_launch_ms = mk["total_ms"] / mk["launches"]
        achieved = 2 * esize * n / (per_launch_ms / 1e3) / 1e9
        tr = load_traffic(mk_name)
        # the counters of one launch at this very workload size, else nothing
        # (no scaling from another size)
        tr = tr if tr and tr["captured_n"] == n else None
        roofline = {"bound": "hbm", "kernel": mk_name, "achieved": achieved,
                    "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                    "peak_source": peaks["source"],
                    "traffic": (tr["read_bytes"] + tr["write_bytes"]) if tr else None,
                    "traffic_read": tr["read_bytes"] if tr else None,
                    "traffic_write": tr["write_bytes"] if tr else None,
                    "algorithmic_bytes": 2 * esize * n, "launch_ms": per_launch_ms,
                    "share_of_step": mk["total_ms"] / (traced_ms * args.steps),
                    "timing": "launch durations from a traced repeat of the timed steps "
                              f"({traced_ms:.3f} ms per traced step)"}
    launches = sum(v["launches"] for v in trace.values()) // args.steps

    e2e = None
    if not args.no_e2e:
        e2e = bench_e2e(nsort, torch, host_in, x, out, tmp, n, code, args.steps, world, esize)
        e2e["host_numa_node"] = numa_node

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.dtype)

    batched = served = configs = sharded = None
    if rank == 0 and world == 1 and not args.no_extras:
        del x, out, tmp, host_in
        torch.cuda.empty_cache()
        configs = bench_configs(nsort, torch)
        torch.cuda.empty_cache()
        batched = bench_batched(nsort, torch, args.segments)
        torch.cuda.empty_cache()
        served = bench_served(nsort, torch, args.served_duration)
        torch.cuda.empty_cache()
        sharded = bench_sharded(nsort, torch)
        torch.cuda.empty_cache()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": f"plain sort, 2^{args.log2n} {args.dtype} keys, uniform, "
                                   f"seed = rank; replicas (one array per GPU)",
                       "n": n, "passes": passes, "sort_tile": sort_tile, "merge_tile": merge_tile,
                       "l2": (f"inputs ({esize * n / 2**30:.2f} GiB) larger than L2; no flush"
                              if esize * n > (256 << 20) else
                              "inputs not larger than L2: a small-case run, not a bench value"),
                       "sort_hbm_roofline_frac": sort_frac,
                       "sort_algorithmic_bytes": alg_bytes_sort,
                       "merge_levels_per_pass": 2 if args.merge_ways == 4 and not wide else 1,
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches * args.steps,
            "kernels": {k: {"launches": v["launches"], "ms_per_launch": v["total_ms"] / v["launches"]}
                        for k, v in trace.items()},
            "clocks": clk,
            "other_configs": configs,
            "batched": batched,
            "served": served,
            "sharded_one_gpu": sharded,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
