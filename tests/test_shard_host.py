"""The sharded sort's host logic on CPU ranks over gloo (no GPU): the
splitter search (bisection rounds with one all-reduce each, then the equal
keys shared out in rank order), the all-to-all exchange of slices and the
part bounds, with world sizes 2, 3 and 4.  The local steps (sorting a
shard, counting keys at most a bound, merging received runs) are stand-ins
built on the oracle; the gathered parts must equal the oracle's sort of the
whole input, bit for bit, payloads included."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2409_03970_gb300 import inputs

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NAMES = {0: "u32", 1: "i32", 2: "f32", 3: "u64", 4: "i64", 5: "f64"}


class OracleOps:
    """Local steps of the sharded sort on CPU tensors, by the oracle."""

    def comm_tensor(self, a):
        return torch.from_numpy(np.ascontiguousarray(a))

    def empty_like(self, x, n):
        return torch.empty(n, dtype=x.dtype)

    @staticmethod
    def _np(t, dt):
        return t.numpy().view(np.uint64 if dt >= 3 else np.uint32)

    @staticmethod
    def _t(a):
        a = np.ascontiguousarray(a)
        return torch.from_numpy(a.view(np.int64 if a.dtype.itemsize == 8 else np.int32).copy())

    def sort(self, keys, vals, dt):
        k = self._np(keys, dt)
        if vals is None:
            s = oracle.sort_keys64(k, NAMES[dt]) if dt >= 3 else oracle.sort_keys(k, NAMES[dt])
            return self._t(s), None
        sk, sv = oracle.sort_pairs(k, vals.numpy().view(np.uint32), NAMES[dt])
        return self._t(sk), self._t(sv)

    def count_le(self, sorted_keys, bounds, dt):
        k = self._np(sorted_keys, dt)
        key = oracle.key64(k, NAMES[dt]) if dt >= 3 else oracle.key(k, NAMES[dt]).astype(np.uint64)
        return np.searchsorted(key, np.asarray(bounds, dtype=np.uint64), side="right").astype(np.int64)

    def merge(self, keys, vals, run_off, dt):
        # the stable merge of sorted runs is the stable sort of their concatenation
        return self.sort(keys, vals, dt)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def global_input(n, dt, pairs, seed):
    if dt >= 3:
        k = inputs.keys64(n, NAMES[dt], "dup16", seed=seed)
    elif dt == 2:
        k, _ = inputs.normal_pairs(n, seed=seed, special_per_mille=30)
    else:
        k = inputs.keys(n, NAMES[dt], "dup16" if seed % 2 else "zipf", seed=seed)
    v = inputs.counter_u32(seed, 9, 0, n) if pairs else None
    return k, v


def rank_main(rank, world, port, n, dt, pairs, seed, sizes, out):
    import torch.distributed as dist
    from paper_2409_03970_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        k, v = global_input(n, dt, pairs, seed)
        off = np.concatenate([[0], np.cumsum(sizes)])
        a, b = int(off[rank]), int(off[rank + 1])
        kt = OracleOps._t(k[a:b])
        vt = OracleOps._t(v[a:b]) if pairs else None
        ko, vo, d = shard.sharded_sort(kt, dt, vals=vt, ops=OracleOps())
        out.put((rank, OracleOps._np(ko, dt).copy(),
                 None if vo is None else vo.numpy().view(np.uint32).copy(), list(d)))
    finally:
        dist.destroy_process_group()


def run(world, n, dt, pairs=False, seed=1, sizes=None):
    if sizes is None:
        sizes = [n // world + (1 if r < n % world else 0) for r in range(world)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, world, port, n, dt, pairs, seed, sizes, q))
             for r in range(world)]
    for p in procs:
        p.start()
    got = sorted([q.get(timeout=300) for _ in range(world)], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return got


@pytest.mark.parametrize("world,dt", [(2, 0), (3, 1), (4, 2), (2, 3), (3, 5)])
def test_sharded_sort_equals_the_oracle(world, dt):
    n = 50_003
    got = run(world, n, dt, seed=world + dt)
    k, _ = global_input(n, dt, False, world + dt)
    want = oracle.sort_keys64(k, NAMES[dt]) if dt >= 3 else oracle.sort_keys(k, NAMES[dt])
    from paper_2409_03970_gb300 import shard
    d = shard.part_bounds(n, world)
    for rank, ko, _, dr in got:
        assert dr == d
        np.testing.assert_array_equal(ko, want[d[rank]:d[rank + 1]])


def test_sharded_pairs_are_stable_and_uneven_shards_balance():
    """Heavy ties across ranks (16 distinct keys) and shards of very
    different sizes, one of them empty: the parts are balanced and the
    payloads come out in input order within equal keys."""
    n = 40_000
    world = 4
    got = run(world, n, 1, pairs=True, seed=3, sizes=[25_000, 0, 5_000, 10_000])
    k, v = global_input(n, 1, True, 3)
    wk, wv = oracle.sort_pairs(k, v, "i32")
    for rank, ko, vo, d in got:
        assert d[rank + 1] - d[rank] in (n // world - 4, n // world, n // world + 4)
        np.testing.assert_array_equal(ko, wk[d[rank]:d[rank + 1]])
        np.testing.assert_array_equal(vo, wv[d[rank]:d[rank + 1]])


def test_share_equal_keys_against_brute_force():
    """The rule that shares the keys equal to the splitter's key out in rank
    order, against counting the first d elements of the stable merge."""
    from paper_2409_03970_gb300 import shard
    rng_keys = [np.sort(inputs.counter_u32(s, 2, 0, 50) % 4) for s in range(3)]
    allk = np.concatenate(rng_keys)
    shard_of = np.repeat(np.arange(3), [len(r) for r in rng_keys])
    order = np.argsort(allk, kind="stable")
    for d in range(allk.size + 1):
        v = allk[order[d]] if d < allk.size else allk.max() + 1
        lt = np.array([[np.sum(r < v)] for r in rng_keys])
        le = np.array([[np.sum(r <= v)] for r in rng_keys])
        c = shard.share_equal_keys(np.array([d]), lt, le)[:, 0]
        np.testing.assert_array_equal(c, np.bincount(shard_of[order[:d]], minlength=3))


def test_part_bounds():
    from paper_2409_03970_gb300 import shard
    assert shard.part_bounds(10, 3) == [0, 0, 4, 10]
    b = shard.part_bounds(1 << 28, 8)
    assert b[0] == 0 and b[-1] == 1 << 28 and all(x % 4 == 0 for x in b)
    assert all(y - x == 1 << 25 for x, y in zip(b, b[1:]))
