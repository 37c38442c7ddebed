"""Sharded sort of one array over P workers: the paper's parallel merge of
sorted parts after a load-balanced partition (Sec. 2.1, last paragraph;
Sec. 3.2, "segmentation points"), with one worker per GPU.

1. Every rank sorts its shard (nsort_keys / nsort_pairs).
2. The output is split evenly: rank q receives the output positions
   [d_q, d_{q+1}), d_q = 4 * floor(q * N / (4 P)) (multiples of 4, so every
   part starts 16-byte aligned).  The segmentation points, how many keys of
   each shard precede each d_q, are found by bisection on the order-key
   space: each round every rank counts its keys at most the candidate key of
   every splitter (nsort_count_le) and one all-reduce sums the counts; after
   the last round an all-gather of each rank's counts below and at the
   splitter's key shares the equal keys out in rank order.
3. One all-to-all moves every slice to its rank.
4. Every rank merges the P slices it received (nsort_merge_shards).

The result is the stable sort of the concatenated shards (rank order, then
position within the shard); for pairs the payloads follow their keys.

This module is host logic: every step on the data runs in libnsort's
kernels or in the collective library (NCCL for CUDA tensors).  The local
steps are methods of an `ops` object, so that the collective logic also runs
on CPU ranks (gloo) with stand-in local steps.

`sort_sharded_one_gpu` runs the same algorithm on one GPU with every shard in
one buffer: nsort_shard_coranks computes all segmentation points in one
kernel, and the exchange becomes device-to-device copies.
"""
from __future__ import annotations

import numpy as np

from . import nsort

KEY_BITS = {nsort.U32: 32, nsort.I32: 32, nsort.F32: 32,
            nsort.U64: 64, nsort.I64: 64, nsort.F64: 64}


def part_bounds(total: int, parts: int) -> list[int]:
    """Output position where each part starts (and the total at the end):
    d_q = 4 * floor(q * total / (4 * parts))."""
    return [4 * ((q * total) // (4 * parts)) for q in range(parts)] + [total]


def share_equal_keys(d: np.ndarray, lt: np.ndarray, le: np.ndarray) -> np.ndarray:
    """Segmentation points from per-shard counts at each splitter's key v*:
    lt[r, j] keys of shard r below v*_j, le[r, j] at most v*_j.  Shard r gives
    its keys below v* and then, in shard order, the equal keys still needed
    to reach d_j outputs.  Returns c[r, j]."""
    eq = le - lt
    rem = d[None, :] - lt.sum(axis=0, keepdims=True)
    before = np.cumsum(eq, axis=0) - eq
    return lt + np.clip(rem - before, 0, eq)


def _sort_into(keys, vals, ko, vo, dtype: int):
    """nsort_keys / nsort_pairs of keys (and vals) into ko (and vo), with the
    key order of dtype."""
    n = int(keys.numel())
    if vals is None:
        tmp = nsort.scratch(nsort.KIND_KEYS, n, device=keys.device, dtype=dtype)
        rc = nsort.nsort_keys(keys, ko, n, dtype, tmp, tmp.numel())
    else:
        tmp = nsort.scratch(nsort.KIND_PAIRS, n, device=keys.device)
        rc = nsort.nsort_pairs(keys, vals, ko, vo, n, dtype, tmp, tmp.numel())
    if rc != nsort.OK:
        raise nsort.NsortError(rc, "nsort_keys" if vals is None else "nsort_pairs")


class GpuOps:
    """The local steps on one GPU, through libnsort (CUDA tensors)."""

    def __init__(self, device=None):
        import torch
        self.torch = torch
        self.device = torch.device(device) if device is not None else torch.device("cuda")

    def comm_tensor(self, a: np.ndarray):
        return self.torch.from_numpy(np.ascontiguousarray(a)).to(self.device)

    def sort(self, keys, vals, dtype):
        ko = self.torch.empty_like(keys)
        vo = None if vals is None else self.torch.empty_like(vals)
        _sort_into(keys, vals, ko, vo, dtype)
        return ko, vo

    def count_le(self, sorted_keys, bounds: np.ndarray, dtype) -> np.ndarray:
        torch = self.torch
        wide = KEY_BITS[dtype] == 64
        b = np.ascontiguousarray(bounds, dtype=np.uint64 if wide else np.uint32)
        bt = torch.from_numpy(b.view(np.int64 if wide else np.int32)).to(self.device)
        le = torch.empty(b.size, dtype=torch.int64, device=self.device)
        rc = nsort.nsort_count_le(sorted_keys, sorted_keys.numel(), dtype, bt, b.size, le)
        if rc != nsort.OK:
            raise nsort.NsortError(rc, "nsort_count_le")
        return le.cpu().numpy()

    def empty_like(self, x, n):
        return self.torch.empty(n, dtype=x.dtype, device=x.device)

    def merge(self, keys, vals, run_off, dtype):
        torch = self.torch
        n = int(run_off[-1])
        ko = torch.empty(n, dtype=keys.dtype, device=keys.device)
        vo = None if vals is None else torch.empty(n, dtype=vals.dtype, device=vals.device)
        kind = nsort.KIND_MERGE if vals is None else nsort.KIND_MERGE_PAIRS
        tmp = nsort.scratch(kind, n, len(run_off) - 1, device=keys.device, dtype=dtype)
        rc = nsort.nsort_merge_shards(keys, vals, ko, vo, run_off, dtype, tmp, tmp.numel())
        if rc != nsort.OK:
            raise nsort.NsortError(rc, "nsort_merge_shards")
        return ko, vo


def _all_reduce_sum(a: np.ndarray, ops, group) -> np.ndarray:
    import torch.distributed as dist
    t = ops.comm_tensor(a.astype(np.int64))
    dist.all_reduce(t, group=group)
    return t.cpu().numpy()


def _all_gather(a: np.ndarray, ops, group, world: int) -> np.ndarray:
    import torch.distributed as dist
    t = ops.comm_tensor(a.astype(np.int64))
    out = [ops.comm_tensor(np.zeros_like(a, dtype=np.int64)) for _ in range(world)]
    dist.all_gather(out, t, group=group)
    return np.stack([o.cpu().numpy() for o in out])


def segmentation_points(sorted_keys, dtype: int, ops, group=None):
    """This rank's segmentation points: c[q] = how many of its keys precede
    output position d_q, for q = 0..P (c[0] = 0, c[P] = its key count), and
    the part bounds d.  One all-gather of the shard sizes, one all-reduce per
    bisection round (32, or 64 for 64-bit keys), one all-gather at the end."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    n_local = int(sorted_keys.shape[0])
    sizes = _all_gather(np.array([n_local]), ops, group, world)[:, 0]
    total = int(sizes.sum())
    d = np.array(part_bounds(total, world), dtype=np.int64)
    inner = d[1:world]                                   # the P-1 interior splitters
    bits = KEY_BITS[dtype]
    lo = np.zeros(inner.size, dtype=np.uint64)
    hi = np.full(inner.size, (1 << bits) - 1, dtype=np.uint64)
    for _ in range(bits):                                # each round halves every interval
        act = lo < hi
        mid = np.where(act, lo + (hi - lo) // np.uint64(2), lo)
        tot = _all_reduce_sum(ops.count_le(sorted_keys, mid, dtype), ops, group)
        low = tot > inner
        hi = np.where(act & low, mid, hi)
        lo = np.where(act & ~low, mid + np.uint64(1), lo)
    below = np.where(lo > 0, lo - np.uint64(1), np.uint64(0))
    lt = np.where(lo > 0, ops.count_le(sorted_keys, below, dtype), 0)
    le = ops.count_le(sorted_keys, lo, dtype)
    both = _all_gather(np.concatenate([lt, le]), ops, group, world)
    c_all = share_equal_keys(inner, both[:, :inner.size], both[:, inner.size:])
    c = np.concatenate([[0], c_all[rank], [n_local]]).astype(np.int64)
    return c, d


def _exchange(x, send_counts: np.ndarray, ops, group):
    """One all-to-all of the slices of x (rank order); returns the received
    buffer and the received counts."""
    import torch.distributed as dist
    sc = ops.comm_tensor(send_counts.astype(np.int64))
    rc = ops.comm_tensor(np.zeros_like(send_counts, dtype=np.int64))
    dist.all_to_all_single(rc, sc, group=group)
    recv_counts = rc.cpu().numpy()
    recv = ops.empty_like(x, int(recv_counts.sum()))
    dist.all_to_all_single(recv, x, [int(v) for v in recv_counts],
                           [int(v) for v in send_counts], group=group)
    return recv, recv_counts


def sharded_sort(keys, dtype: int, vals=None, group=None, ops=None):
    """Sorts the array whose shard on this rank is `keys` (with payloads
    `vals`), over every rank of `group`.  Returns (keys_out, vals_out, d):
    this rank's part of the sorted array, output positions [d[rank],
    d[rank+1])."""
    import torch.distributed as dist
    ops = ops or GpuOps(keys.device)
    skeys, svals = ops.sort(keys, vals, dtype)
    c, d = segmentation_points(skeys, dtype, ops, group)
    send = np.diff(c)
    rk, counts = _exchange(skeys, send, ops, group)
    rv = None
    if vals is not None:
        rv, _ = _exchange(svals, send, ops, group)
    run_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    ko, vo = ops.merge(rk, rv, run_off, dtype)
    return ko, vo, d


def sort_sharded_one_gpu(keys, nshards: int, dtype: int, vals=None):
    """The sharded sort with all nshards shards in one buffer on one GPU:
    shard r = keys[s_r, s_{r+1}) with s_r = floor(r n / nshards).  Each shard
    is sorted on its own, nsort_shard_coranks finds every segmentation point
    in one kernel, slices are gathered by device copies, and each part is
    merged by nsort_merge_shards.  Returns (keys_out, vals_out) for the whole
    array."""
    import torch
    n = int(keys.numel())
    dev = keys.device
    s = [(r * n) // nshards for r in range(nshards + 1)]
    sk = torch.empty_like(keys)
    sv = None if vals is None else torch.empty_like(vals)
    for r in range(nshards):
        a, b = s[r], s[r + 1]
        if b == a:
            continue
        _sort_into(keys[a:b], None if vals is None else vals[a:b], sk[a:b],
                   None if vals is None else sv[a:b], dtype)
    d = part_bounds(n, nshards)
    off_t = torch.tensor(s, dtype=torch.int64, device=dev)
    tgt_t = torch.tensor(d, dtype=torch.int64, device=dev)
    cr = torch.empty((nshards + 1) * nshards, dtype=torch.int64, device=dev)
    rc = nsort.nsort_shard_coranks(sk, off_t, nshards, tgt_t, nshards + 1, dtype, cr)
    if rc != nsort.OK:
        raise nsort.NsortError(rc, "nsort_shard_coranks")
    c = cr.view(nshards + 1, nshards).cpu().numpy()
    ko = torch.empty_like(keys)
    vo = None if vals is None else torch.empty_like(vals)
    for q in range(nshards):
        lens = c[q + 1] - c[q]
        run_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        m = int(run_off[-1])
        if m == 0:
            continue
        rk = torch.empty(m, dtype=keys.dtype, device=dev)
        rv = None if vals is None else torch.empty(m, dtype=vals.dtype, device=dev)
        for r in range(nshards):
            a, b = s[r] + int(c[q][r]), s[r] + int(c[q + 1][r])
            if b > a:
                rk[run_off[r]:run_off[r + 1]].copy_(sk[a:b])
                if vals is not None:
                    rv[run_off[r]:run_off[r + 1]].copy_(sv[a:b])
        kind = nsort.KIND_MERGE if vals is None else nsort.KIND_MERGE_PAIRS
        tmp = nsort.scratch(kind, m, nshards, device=dev, dtype=dtype)
        rc = nsort.nsort_merge_shards(rk, rv, ko[d[q]:d[q + 1]],
                                      None if vals is None else vo[d[q]:d[q + 1]],
                                      run_off, dtype, tmp, tmp.numel())
        if rc != nsort.OK:
            raise nsort.NsortError(rc, "nsort_merge_shards")
    return ko, vo
