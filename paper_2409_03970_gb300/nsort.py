"""Thin ctypes binding of libnsort (include/nsort.h): the same entry points,
with argument marshalling only.  Every step of a sort runs in the CUDA
kernels of libnsort; torch only provides device memory and streams.

The raw names (``nsort_keys``, ``nsort_pairs``, ...) take torch tensors or
integer device addresses.  ``sort`` / ``sort_pairs`` are conveniences that
allocate the output and the scratch with torch and raise on error.

There is no CPU fallback: if libnsort.so has not been built this module
raises on first use.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libnsort.so")

U32, I32, F32 = 0, 1, 2
U64, I64, F64 = 3, 4, 5           # 64-bit keys (nsort_keys only)
KIND_KEYS, KIND_PAIRS, KIND_SEGMENTED, KIND_SEGMENTED_PAIRS = 0, 1, 2, 3
KIND_MERGE, KIND_MERGE_PAIRS, KIND_PAIRS64 = 4, 5, 6
OK, EINVAL, ENOMEM, ECUDA, EBUSY, ETIMEOUT, ENOTFOUND = range(7)
NET_BITONIC, NET_ODDEVEN, NET_BEST = 0, 1, 2     # include/nsort_ablation.h
MERGE_HYBRID, MERGE_SHUFFLE, MERGE_SERIAL = 0, 1, 2

_lock = threading.Lock()
_lib = None


class Request(ctypes.Structure):
    """nsort_request."""
    _fields_ = [("kind", ctypes.c_int), ("dtype", ctypes.c_int), ("n", ctypes.c_uint64),
                ("d_keys_in", ctypes.c_void_p), ("d_keys_out", ctypes.c_void_p),
                ("d_vals_in", ctypes.c_void_p), ("d_vals_out", ctypes.c_void_p)]


class Timing(ctypes.Structure):
    """nsort_timing: host monotonic-clock seconds."""
    _fields_ = [("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("status", ctypes.c_int), ("batched", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SegConfig(ctypes.Structure):
    """nsort_seg_config: tunables of the segmented sort."""
    _fields_ = [("block_threads", ctypes.c_int), ("tiny_width", ctypes.c_int),
                ("small_ipt", ctypes.c_int), ("blocks_per_sm", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class NsortError(RuntimeError):
    def __init__(self, status: int, what: str):
        lib = _load()
        msg = lib.nsort_status_string(status).decode()
        detail = lib.nsort_last_error().decode()
        super().__init__(f"{what}: {msg} ({status}){': ' + detail if detail else ''}")
        self.status = status


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libnsort.so is not built ({LIB_PATH}); run "
                "`python -c 'import __graft_entry__ as g; g.build()'` first")
        lib = ctypes.CDLL(LIB_PATH)
        vp, u64, i32, sz = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t
        ip = ctypes.POINTER(ctypes.c_int)
        lib.nsort_temp_bytes.argtypes = [i32, u64, u64, i32]
        lib.nsort_temp_bytes.restype = sz
        lib.nsort_plan.argtypes = [i32, u64, ip, ip, ip]
        lib.nsort_plan.restype = i32
        lib.nsort_plan_dtype.argtypes = [i32, u64, i32, ip, ip, ip]
        lib.nsort_plan_dtype.restype = i32
        i64p_ = ctypes.POINTER(ctypes.c_int64)
        lib.nsort_shard_coranks.argtypes = [vp, vp, i32, vp, i32, i32, vp, vp]
        lib.nsort_shard_coranks.restype = i32
        lib.nsort_count_le.argtypes = [vp, u64, i32, vp, u64, vp, vp]
        lib.nsort_count_le.restype = i32
        lib.nsort_merge_shards.argtypes = [vp, vp, vp, vp, i64p_, i32, i32, vp, sz, vp]
        lib.nsort_merge_shards.restype = i32
        lib.nsort_merge_grid.argtypes = [i32, i32]
        lib.nsort_merge_grid.restype = i32
        lib.nsort_keys.argtypes = [vp, vp, u64, i32, vp, sz, vp]
        lib.nsort_keys.restype = i32
        lib.nsort_pairs.argtypes = [vp, vp, vp, vp, u64, i32, vp, sz, vp]
        lib.nsort_pairs.restype = i32
        lib.nsort_pairs64.argtypes = [vp, vp, vp, vp, u64, i32, vp, sz, vp]
        lib.nsort_pairs64.restype = i32
        lib.nsort_segmented.argtypes = [vp, vp, vp, vp, vp, u64, u64, i32, vp, sz, vp]
        lib.nsort_segmented.restype = i32
        lib.nsort_device_status.argtypes = [vp, vp]
        lib.nsort_device_status.restype = i32
        lib.nsort_segmented_set_config.argtypes = [ctypes.POINTER(SegConfig)]
        lib.nsort_segmented_set_config.restype = i32
        lib.nsort_segmented_get_config.argtypes = [ctypes.POINTER(SegConfig)]
        lib.nsort_segmented_get_config.restype = i32
        lib.nsort_ctx_create.argtypes = [i32, sz, i32, u64, ctypes.POINTER(vp)]
        lib.nsort_ctx_create.restype = i32
        lib.nsort_ctx_destroy.argtypes = [vp]
        lib.nsort_ctx_destroy.restype = None
        lib.nsort_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(u64)]
        lib.nsort_submit.restype = i32
        lib.nsort_poll.argtypes = [vp, u64, ip, ctypes.POINTER(Timing)]
        lib.nsort_poll.restype = i32
        lib.nsort_wait.argtypes = [vp, u64, ctypes.c_uint32]
        lib.nsort_wait.restype = i32
        u64p = ctypes.POINTER(u64)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.nsort_policy_pick_batch.argtypes = [u64p, ip, ip, u64p, i32, u64, i32, u64, u64, i32,
                                                u64p, ip]
        lib.nsort_policy_pick_batch.restype = i32
        lib.nsort_policy_arena_replay.argtypes = [u64, i64p, i32, i64p]
        lib.nsort_policy_arena_replay.restype = i32
        lib.nsort_selftest_wait.argtypes = [vp, sz, ctypes.c_uint32, vp]
        lib.nsort_selftest_wait.restype = i32
        lib.nsort_testing_set_four_way_min.argtypes = [u64]
        lib.nsort_testing_set_four_way_min.restype = u64
        lib.nsort_keys_noalloc.argtypes = [vp, vp, u64, i32, vp]
        lib.nsort_keys_noalloc.restype = i32
        lib.nsort_keys_noalloc_status.argtypes = [vp]
        lib.nsort_keys_noalloc_status.restype = i32
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.nsort_network.argtypes = [i32, i32, i32p, i32p, i32]
        lib.nsort_network.restype = i32
        lib.nsort_network_apply.argtypes = [vp, vp, u64, i32, i32, vp]
        lib.nsort_network_apply.restype = i32
        lib.nsort_runs.argtypes = [vp, vp, u64, i32, i32, u64, vp]
        lib.nsort_runs.restype = i32
        lib.nsort_merge_runs.argtypes = [vp, vp, u64, u64, i32, i32, vp]
        lib.nsort_merge_runs.restype = i32
        lib.nsort_trace_enable.argtypes = [i32]
        lib.nsort_trace_enable.restype = i32
        lib.nsort_trace_read.argtypes = [vp, i32, ip]
        lib.nsort_trace_read.restype = i32
        lib.nsort_status_string.argtypes = [i32]
        lib.nsort_status_string.restype = ctypes.c_char_p
        lib.nsort_last_error.argtypes = []
        lib.nsort_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


def lib():
    """The loaded ctypes library (loads it on first call)."""
    return _load()


# ---- marshalling ------------------------------------------------------------

def _ptr(x) -> int:
    """Device address of a buffer argument: None -> 0, an int is taken as a
    device address as is, a tensor must be a contiguous CUDA tensor (every
    buffer of the C ABI is a contiguous device array)."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if not getattr(x, "is_cuda", False):
        raise ValueError("nsort buffers must be CUDA tensors (or raw device addresses)")
    if not x.is_contiguous():
        raise ValueError("nsort buffers must be contiguous")
    return x.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def dtype_code(t) -> int:
    """nsort_dtype of a torch tensor (uint32 / int32 / float32, or the 64-bit
    uint64 / int64 / float64)."""
    import torch
    codes = {torch.int32: I32, torch.float32: F32, torch.int64: I64, torch.float64: F64}
    if hasattr(torch, "uint32"):
        codes[torch.uint32] = U32
    if hasattr(torch, "uint64"):
        codes[torch.uint64] = U64
    if t.dtype not in codes:
        raise TypeError(f"keys must be (u)int32, float32, (u)int64 or float64, not {t.dtype}")
    return codes[t.dtype]


def _check_1d(t, name):
    if not t.is_cuda or not t.is_contiguous() or t.dim() != 1:
        raise ValueError(f"{name} must be a contiguous 1-D CUDA tensor")


# ---- raw entry points (same names as the C ABI) ----------------------------

def nsort_temp_bytes(kind: int, n: int, nseg: int = 0, dtype: int = U32) -> int:
    return int(_load().nsort_temp_bytes(kind, n, nseg, dtype))


def nsort_merge_grid(kind: int, dtype: int = U32) -> int:
    """CTAs of the persistent merge pass on the current device (0 on error)."""
    return int(_load().nsort_merge_grid(kind, dtype))


def nsort_plan(kind: int, n: int, dtype: int = U32):
    """(passes, sort_tile, merge_tile) of a plain sort of n keys of dtype."""
    p, s, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rc = _load().nsort_plan_dtype(kind, n, dtype, ctypes.byref(p), ctypes.byref(s),
                                  ctypes.byref(m))
    if rc != OK:
        raise NsortError(rc, "nsort_plan_dtype")
    return p.value, s.value, m.value


def nsort_keys(keys_in, keys_out, n: int, dtype: int, tmp, tmp_bytes: int, stream=None) -> int:
    return _load().nsort_keys(_ptr(keys_in), _ptr(keys_out), n, dtype, _ptr(tmp), tmp_bytes,
                              _stream(stream))


def nsort_pairs(keys_in, vals_in, keys_out, vals_out, n: int, dtype: int, tmp, tmp_bytes: int,
                stream=None) -> int:
    return _load().nsort_pairs(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out), n,
                               dtype, _ptr(tmp), tmp_bytes, _stream(stream))


def nsort_pairs64(keys_in, vals_in, keys_out, vals_out, n: int, dtype: int, tmp, tmp_bytes: int,
                  stream=None) -> int:
    """nsort_pairs with 64-bit payloads (vals: 8-byte words)."""
    return _load().nsort_pairs64(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out), n,
                                 dtype, _ptr(tmp), tmp_bytes, _stream(stream))


def nsort_segmented(keys_in, keys_out, vals_in, vals_out, offsets, nseg: int, n: int,
                    dtype: int, tmp, tmp_bytes: int, stream=None) -> int:
    return _load().nsort_segmented(_ptr(keys_in), _ptr(keys_out), _ptr(vals_in), _ptr(vals_out),
                                   _ptr(offsets), nseg, n, dtype, _ptr(tmp), tmp_bytes,
                                   _stream(stream))


def nsort_shard_coranks(keys, shard_off, nshards: int, targets, ntargets: int, dtype: int,
                        coranks, stream=None) -> int:
    """Segmentation points of nshards sorted shards in one device buffer
    (shard_off, targets, coranks: device int64 arrays)."""
    return _load().nsort_shard_coranks(_ptr(keys), _ptr(shard_off), nshards, _ptr(targets),
                                       ntargets, dtype, _ptr(coranks), _stream(stream))


def nsort_count_le(sorted_keys, n: int, dtype: int, bounds, m: int, le, stream=None) -> int:
    """le[i] = keys of the sorted array whose order key is <= bounds[i]
    (bounds: device uint32 / uint64 order keys; le: device int64)."""
    return _load().nsort_count_le(_ptr(sorted_keys), n, dtype, _ptr(bounds), m, _ptr(le),
                                  _stream(stream))


def nsort_merge_shards(keys_in, vals_in, keys_out, vals_out, run_off, dtype: int, tmp,
                       tmp_bytes: int, stream=None) -> int:
    """Merges sorted runs stored back to back; run_off: the nruns+1 host
    offsets (any integer sequence)."""
    offs = [int(x) for x in run_off]
    arr = (ctypes.c_int64 * len(offs))(*offs)
    return _load().nsort_merge_shards(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out),
                                      _ptr(vals_out), arr, len(offs) - 1, dtype, _ptr(tmp),
                                      tmp_bytes, _stream(stream))


def nsort_device_status(tmp, stream=None) -> int:
    """Device status word of the last call that used scratch `tmp` (syncs)."""
    return _load().nsort_device_status(_ptr(tmp), _stream(stream))


def nsort_segmented_set_config(block_threads=512, tiny_width=16, small_ipt=16,
                               blocks_per_sm=0) -> int:
    cfg = SegConfig(block_threads, tiny_width, small_ipt, blocks_per_sm)
    return _load().nsort_segmented_set_config(ctypes.byref(cfg))


def nsort_segmented_get_config() -> dict:
    cfg = SegConfig()
    rc = _load().nsort_segmented_get_config(ctypes.byref(cfg))
    if rc != OK:
        raise NsortError(rc, "nsort_segmented_get_config")
    return cfg.as_dict()


# ---- serving ---------------------------------------------------------------

def nsort_ctx_create(device: int = 0, mem_budget_bytes: int = 1 << 30, streams: int = 4,
                     batch_max_keys: int = 1 << 16) -> int:
    """A sort-serving context (opaque handle)."""
    h = ctypes.c_void_p()
    rc = _load().nsort_ctx_create(device, mem_budget_bytes, streams, batch_max_keys,
                                  ctypes.byref(h))
    if rc != OK:
        raise NsortError(rc, "nsort_ctx_create")
    return h.value


def nsort_ctx_destroy(ctx: int) -> None:
    _load().nsort_ctx_destroy(ctx)


def nsort_submit(ctx: int, kind: int, dtype: int, n: int, keys_in, keys_out, vals_in=None,
                 vals_out=None) -> int:
    """Submits a request; returns its ticket."""
    req = Request(kind, dtype, n, _ptr(keys_in), _ptr(keys_out), _ptr(vals_in), _ptr(vals_out))
    t = ctypes.c_uint64()
    rc = _load().nsort_submit(ctx, ctypes.byref(req), ctypes.byref(t))
    if rc != OK:
        raise NsortError(rc, "nsort_submit")
    return t.value


def nsort_poll(ctx: int, ticket: int):
    """(done, timing dict or None)."""
    done = ctypes.c_int()
    tm = Timing()
    rc = _load().nsort_poll(ctx, ticket, ctypes.byref(done), ctypes.byref(tm))
    if rc != OK:
        raise NsortError(rc, "nsort_poll")
    return bool(done.value), (tm.as_dict() if done.value else None)


def nsort_wait(ctx: int, ticket: int, timeout_ms: int = 60000) -> int:
    return _load().nsort_wait(ctx, ticket, timeout_ms)


class SortServer:
    """Context manager around an nsort serving context."""

    def __init__(self, device=0, mem_budget_bytes=1 << 30, streams=4, batch_max_keys=1 << 16):
        self.ctx = nsort_ctx_create(device, mem_budget_bytes, streams, batch_max_keys)

    def submit(self, keys_in, keys_out, vals_in=None, vals_out=None, n=None, dtype=None):
        kind = KIND_KEYS if vals_in is None else KIND_PAIRS
        n = keys_in.numel() if n is None else n
        dtype = dtype_code(keys_in) if dtype is None else dtype
        return nsort_submit(self.ctx, kind, dtype, n, keys_in, keys_out, vals_in, vals_out)

    def poll(self, ticket):
        return nsort_poll(self.ctx, ticket)

    def wait(self, ticket, timeout_ms=60000):
        return nsort_wait(self.ctx, ticket, timeout_ms)

    def close(self):
        if self.ctx:
            nsort_ctx_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def nsort_selftest_wait(tmp, limit_us: int = 20000, stream=None) -> int:
    """Runs the library's bounded waits on events that never happen (test hook)."""
    return _load().nsort_selftest_wait(_ptr(tmp), tmp.numel() if hasattr(tmp, "numel") else 512,
                                       limit_us, _stream(stream))


def nsort_testing_set_four_way_min(min_keys: int) -> int:
    """Smallest 32-bit key sort that merges two levels per pass (test hook);
    returns the previous setting."""
    return int(_load().nsort_testing_set_four_way_min(min_keys))


FOUR_WAY_NEVER = (1 << 64) - 1


SERVE_LARGE_MIN_KEYS = 1 << 22   # the server runs requests this large one at a time


def policy_pick_batch(queue, batch_max_keys, max_batch=4096, max_batch_keys=1 << 24,
                      large_min_keys=(1 << 64) - 1, large_running=False):
    """The server's admission choice for a queue of (ticket, kind, dtype, n)."""
    m = len(queue)
    T = (ctypes.c_uint64 * max(m, 1))(*[q[0] for q in queue])
    K = (ctypes.c_int * max(m, 1))(*[q[1] for q in queue])
    D = (ctypes.c_int * max(m, 1))(*[q[2] for q in queue])
    N = (ctypes.c_uint64 * max(m, 1))(*[q[3] for q in queue])
    out = (ctypes.c_uint64 * max(m, 1))()
    cnt = ctypes.c_int()
    rc = _load().nsort_policy_pick_batch(T, K, D, N, m, batch_max_keys, max_batch, max_batch_keys,
                                         large_min_keys, int(large_running), out,
                                         ctypes.byref(cnt))
    if rc != OK:
        raise NsortError(rc, "nsort_policy_pick_batch")
    return [out[i] for i in range(cnt.value)]


def policy_arena_replay(capacity, ops):
    """Offsets the server's arena gives for a list of alloc (>0) / release (<0) ops."""
    m = len(ops)
    O = (ctypes.c_int64 * max(m, 1))(*ops)
    R = (ctypes.c_int64 * max(m, 1))()
    rc = _load().nsort_policy_arena_replay(capacity, O, m, R)
    if rc != OK:
        raise NsortError(rc, "nsort_policy_arena_replay")
    return [R[i] for i in range(m)]


NOALLOC_MAX_KEYS = 1 << 20


def nsort_keys_noalloc(keys_in, keys_out, n: int, dtype: int, stream=None) -> int:
    """nsort_keys without a scratch argument, for callers that cannot
    allocate device memory (scratch is a fixed array inside the library;
    n <= NOALLOC_MAX_KEYS; calls that overlap on the GPU race on it)."""
    return _load().nsort_keys_noalloc(_ptr(keys_in), _ptr(keys_out), n, dtype, _stream(stream))


def nsort_keys_noalloc_status(stream=None) -> int:
    """Device status of the last nsort_keys_noalloc on the current device
    (synchronises `stream`)."""
    return _load().nsort_keys_noalloc_status(_stream(stream))


class TraceEntry(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_char * 32), ("launches", ctypes.c_uint64),
                ("total_ms", ctypes.c_double)]


# ---- ablation of the column-sort network and keys per thread ------------

def nsort_network(family: int, width: int):
    """The comparator list (lo, hi) pairs the device column sort of this
    family and width is generated from; None for an unknown one."""
    n = _load().nsort_network(family, width, None, None, 0)
    if n < 0:
        return None
    lo = (ctypes.c_int32 * max(n, 1))()
    hi = (ctypes.c_int32 * max(n, 1))()
    _load().nsort_network(family, width, lo, hi, n)
    return [(lo[c], hi[c]) for c in range(n)]


def nsort_network_apply(keys_in, keys_out, groups: int, family: int, width: int,
                        stream=None) -> int:
    return _load().nsort_network_apply(_ptr(keys_in), _ptr(keys_out), groups, family, width,
                                       _stream(stream))


def nsort_runs(keys_in, keys_out, n: int, family: int, ipt: int, run: int, stream=None) -> int:
    return _load().nsort_runs(_ptr(keys_in), _ptr(keys_out), n, family, ipt, run,
                              _stream(stream))


def nsort_merge_runs(keys_in, keys_out, n: int, run: int, method: int, ipt: int,
                     stream=None) -> int:
    return _load().nsort_merge_runs(_ptr(keys_in), _ptr(keys_out), n, run, method, ipt,
                                    _stream(stream))


def merge_run_lengths(method: int, ipt: int):
    """The run lengths nsort_merge_runs accepts for this merger and width."""
    lo, hi = {MERGE_HYBRID: (ipt, 16 * ipt), MERGE_SHUFFLE: (1, 16 * ipt),
              MERGE_SERIAL: (max(1, ipt // 2), 256 * ipt)}[method]
    out, r = [], 1
    while r <= hi:
        if r >= lo:
            out.append(r)
        r *= 2
    return out


def nsort_trace_enable(on: bool) -> int:
    return _load().nsort_trace_enable(1 if on else 0)


def nsort_trace_read() -> dict:
    """{kernel name: {"launches": L, "total_ms": T}} since tracing was enabled."""
    buf = (TraceEntry * 32)()
    cnt = ctypes.c_int()
    rc = _load().nsort_trace_read(ctypes.addressof(buf), 32, ctypes.byref(cnt))
    if rc != OK:
        raise NsortError(rc, "nsort_trace_read")
    return {buf[i].kernel.decode(): {"launches": int(buf[i].launches),
                                     "total_ms": float(buf[i].total_ms)}
            for i in range(min(cnt.value, 32))}


# ---- conveniences -----------------------------------------------------------

def scratch(kind: int, n: int, nseg: int = 0, device=None, dtype: int = U32):
    """A uint8 device tensor of nsort_temp_bytes(kind, n, nseg, dtype) bytes
    (at least one byte, so that it has an address)."""
    import torch
    nbytes = max(1, nsort_temp_bytes(kind, n, nseg, dtype))
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def sort(keys, out=None, tmp=None, stream=None):
    """Sorts a 1-D CUDA tensor of uint32 / int32 / float32 (or 64-bit) keys
    ascending (floats in IEEE totalOrder).  Returns `out` (new tensor if
    None)."""
    import torch
    _check_1d(keys, "keys")
    dt = dtype_code(keys)
    n = keys.numel()
    if out is None:
        out = torch.empty_like(keys)
    _check_1d(out, "out")
    if tmp is None:
        tmp = scratch(KIND_KEYS, n, device=keys.device, dtype=dt)
    rc = nsort_keys(keys, out, n, dt, tmp, tmp.numel(), stream)
    if rc != OK:
        raise NsortError(rc, "nsort_keys")
    return out


def sort_segmented(keys, offsets, vals=None, keys_out=None, vals_out=None, tmp=None,
                   stream=None, check=True):
    """Sorts each segment [offsets[s], offsets[s+1]) of a 1-D CUDA key tensor
    on its own (stable with values).  offsets: int64 CUDA tensor of nseg+1
    entries.  check=True synchronises and raises on a device-side error
    (malformed offsets)."""
    import torch
    _check_1d(keys, "keys")
    if offsets.dtype != torch.int64 or not offsets.is_cuda or offsets.dim() != 1:
        raise ValueError("offsets must be a 1-D int64 CUDA tensor")
    dt = dtype_code(keys)
    n, nseg = keys.numel(), offsets.numel() - 1
    keys_out = torch.empty_like(keys) if keys_out is None else keys_out
    if vals is not None:
        vals_out = torch.empty_like(vals) if vals_out is None else vals_out
    kind = KIND_SEGMENTED if vals is None else KIND_SEGMENTED_PAIRS
    if tmp is None:
        tmp = scratch(kind, n, nseg, device=keys.device)
    rc = nsort_segmented(keys, keys_out, vals, vals_out, offsets, nseg, n, dt, tmp, tmp.numel(),
                         stream)
    if rc != OK:
        raise NsortError(rc, "nsort_segmented")
    if check:
        st = nsort_device_status(tmp, stream)
        if st != OK:
            raise NsortError(st, "nsort_segmented (device status)")
    return keys_out if vals is None else (keys_out, vals_out)


def sort_pairs(keys, vals, keys_out=None, vals_out=None, tmp=None, stream=None):
    """Stable sort of (key, uint32/int32 payload) pairs by key.  Returns
    (keys_out, vals_out)."""
    import torch
    _check_1d(keys, "keys")
    _check_1d(vals, "vals")
    if vals.numel() != keys.numel() or vals.element_size() != 4:
        raise ValueError("vals must be a 32-bit tensor of the same length as keys")
    dt = dtype_code(keys)
    n = keys.numel()
    keys_out = torch.empty_like(keys) if keys_out is None else keys_out
    vals_out = torch.empty_like(vals) if vals_out is None else vals_out
    if tmp is None:
        tmp = scratch(KIND_PAIRS, n, device=keys.device)
    rc = nsort_pairs(keys, vals, keys_out, vals_out, n, dt, tmp, tmp.numel(), stream)
    if rc != OK:
        raise NsortError(rc, "nsort_pairs")
    return keys_out, vals_out
