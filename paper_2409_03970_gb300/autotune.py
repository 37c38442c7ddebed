"""Autotuner for the segmented sort.

Times nsort_segmented on the caller's own batch under each candidate
configuration (block size, network width of the one-thread bin, keys per
lane of the one-warp bin, persistent CTAs per SM), keeps the fastest, and
caches it per (GPU, key dtype, kind) in a JSON file
($NSORT_TUNE_CACHE, default ~/.cache/nsort/tune.json).  ``apply_cached``
loads a cached choice into the library; ``tune_segmented`` measures and
stores one.  Every candidate produces the same sorted bits (the
configuration only changes how the work is split), so tuning never changes
results.
"""
from __future__ import annotations

import itertools
import json
import os
import time

from . import nsort

DEFAULT_CANDIDATES = [
    dict(block_threads=b, tiny_width=w, small_ipt=i, blocks_per_sm=c)
    for b, w, i, c in itertools.product((256, 512), (8, 16), (8, 16), (0, 1))
]


def cache_path() -> str:
    return os.environ.get("NSORT_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "nsort", "tune.json"))


def _key(device_name: str, dtype: int, pairs: bool) -> str:
    return f"{device_name}|dtype={dtype}|{'pairs' if pairs else 'keys'}"


def _load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(d: dict) -> None:
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def apply_cached(dtype: int = nsort.U32, pairs: bool = False) -> dict | None:
    """Applies the cached configuration for this GPU, if any; returns it."""
    import torch
    entry = _load_cache().get(_key(torch.cuda.get_device_name(), dtype, pairs))
    if not entry:
        return None
    cfg = entry["config"]
    if nsort.nsort_segmented_set_config(**cfg) != nsort.OK:
        return None
    return cfg


def tune_segmented(keys, offsets, vals=None, candidates=None, reps: int = 3,
                   store: bool = True) -> dict:
    """Times each candidate on this batch (device tensors) and applies the
    fastest.  Returns {"config": ..., "ms": ..., "table": [...]}."""
    import torch
    candidates = candidates or DEFAULT_CANDIDATES
    dt = nsort.dtype_code(keys)
    n, nseg = keys.numel(), offsets.numel() - 1
    kind = nsort.KIND_SEGMENTED if vals is None else nsort.KIND_SEGMENTED_PAIRS
    tmp = nsort.scratch(kind, n, nseg, device=keys.device)
    ko = torch.empty_like(keys)
    vo = None if vals is None else torch.empty_like(vals)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    table = []
    for cfg in candidates:
        if nsort.nsort_segmented_set_config(**cfg) != nsort.OK:
            continue
        rc = nsort.nsort_segmented(keys, ko, vals, vo, offsets, nseg, n, dt, tmp, tmp.numel(),
                                   stream)
        if rc != nsort.OK:
            continue
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0.record(stream)
            nsort.nsort_segmented(keys, ko, vals, vo, offsets, nseg, n, dt, tmp, tmp.numel(),
                                  stream)
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        if nsort.nsort_device_status(tmp, stream) != nsort.OK:
            continue
        table.append({"config": cfg, "ms": best})
    if not table:
        raise RuntimeError("autotune: no candidate configuration ran")
    win = min(table, key=lambda r: r["ms"])
    nsort.nsort_segmented_set_config(**win["config"])
    if store:
        d = _load_cache()
        d[_key(torch.cuda.get_device_name(), dt, vals is not None)] = {
            "config": win["config"], "ms": win["ms"], "n": n, "nseg": nseg,
            "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
        _store_cache(d)
    return {"config": win["config"], "ms": win["ms"], "table": table}
