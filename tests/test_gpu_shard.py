"""GPU parity of the sharded sort's steps (through the C ABI) against the
oracle, bit for bit: the segmentation points of P sorted shards
(nsort_shard_coranks), the per-GPU counts of the splitter search
(nsort_count_le), the merge of sorted runs of any lengths
(nsort_merge_shards, keys and stable pairs, 32- and 64-bit keys), and the
whole sort with P shards on one GPU, up to the 2^28-key workload.

The expected segmentation points come from their definition: the stable
sort of the concatenated shards (by the oracle, payload = position) orders
every element; c[d][r] counts the elements of shard r among the first d."""
import numpy as np
import pytest

import oracle
from paper_2409_03970_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"u32": 0, "i32": 1, "f32": 2, "u64": 3, "i64": 4, "f64": 5}


@pytest.fixture(scope="module")
def ns():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03970_gb300 import build, nsort
    build.build()
    nsort.lib()
    return nsort


def wide(dt):
    return DT[dt] >= 3


def dev(a):
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(np.int64 if a.dtype.itemsize == 8 else np.int32)).cuda()


def host(t, dt):
    return t.cpu().numpy().view(np.uint64 if wide(dt) else np.uint32)


def make_keys(n, dt, dist, seed):
    if wide(dt):
        return inputs.keys64(n, dt, "specials" if dist == "specials" else dist, seed=seed)
    if dist == "specials":
        k, _ = inputs.normal_pairs(n, seed=seed, special_per_mille=50)
        return k if dt == "f32" else inputs.keys(n, dt, "dup16", seed=seed)
    return inputs.keys(n, dt, dist, seed=seed)


def osort(x, dt):
    return oracle.sort_keys64(x, dt) if wide(dt) else oracle.sort_keys(x, dt)


def okey(x, dt):
    return oracle.key64(x, dt) if wide(dt) else oracle.key(x, dt).astype(np.uint64)


def stable_order(x, dt):
    """Positions of x in the order of the stable sort of x (by the oracle:
    keys with payload = position; 64-bit keys by a stable argsort of their
    oracle order keys)."""
    if wide(dt):
        return np.argsort(oracle.key64(x, dt), kind="stable")
    _, pos = oracle.sort_pairs(x, np.arange(x.size, dtype=np.uint32), dt)
    return pos.astype(np.int64)


def shard_lengths(n, p, seed, empty=()):
    cut = np.sort(inputs.counter_u64(seed, 3, 0, p - 1) % np.uint64(n + 1)).astype(np.int64)
    lens = np.diff(np.concatenate([[0], cut, [n]]))
    for e in empty:                      # move these shards' keys to their right neighbour
        if e < p - 1:
            lens[e + 1] += lens[e]
            lens[e] = 0
    return lens


def sorted_shards(x, lens, dt):
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    return np.concatenate([osort(x[off[r]:off[r + 1]], dt) for r in range(len(lens))]), off


CORANK_CASES = [(1, "u32", "uniform"), (2, "i32", "dup16"), (3, "f32", "specials"),
                (8, "u32", "sorted"), (8, "f32", "zipf"), (17, "i32", "reverse"),
                (32, "u32", "dup16"), (5, "u64", "uniform"), (6, "i64", "dup16"),
                (4, "f64", "specials")]


@pytest.mark.parametrize("p,dt,dist", CORANK_CASES)
def test_shard_coranks_against_definition(ns, p, dt, dist):
    n = 60_001
    x = make_keys(n, dt, dist, seed=p)
    lens = shard_lengths(n, p, seed=p, empty=(1,) if p > 3 else ())
    keys, off = sorted_shards(x, lens, dt)
    order = stable_order(keys, dt)
    shard_of = np.searchsorted(off, order, side="right") - 1
    targets = np.unique(np.concatenate([
        [0, 1, 2, n - 1, n, n + 5, -3],
        inputs.counter_u64(p, 4, 0, 200) % np.uint64(n + 1)]).astype(np.int64))
    cr = torch.empty(targets.size * p, dtype=torch.int64, device="cuda")
    rc = ns.nsort_shard_coranks(dev(keys), dev(off), p, dev(targets), targets.size, DT[dt], cr)
    assert rc == ns.OK, ns.lib().nsort_last_error()
    got = cr.view(targets.size, p).cpu().numpy()
    for j, d in enumerate(targets):
        d = min(max(int(d), 0), n)
        want = np.bincount(shard_of[:d], minlength=p)
        np.testing.assert_array_equal(got[j], want, err_msg=f"target {d}")


@pytest.mark.parametrize("dt", ["u32", "i32", "f32", "u64", "f64"])
def test_count_le_against_searchsorted(ns, dt):
    x = osort(make_keys(100_003, dt, "dup16", seed=7), dt)
    k = okey(x, dt)
    top = np.uint64((1 << (64 if wide(dt) else 32)) - 1)
    pick = inputs.counter_u64(7, 5, 0, 300) % np.uint64(x.size)
    edges = np.array([0, 1, int(top) - 1, int(top)], dtype=np.uint64)
    bounds = np.concatenate([edges, k[pick.astype(np.int64)],
                             k[pick.astype(np.int64)] - np.uint64(1),
                             inputs.counter_u64(7, 6, 0, 100) & top])
    bounds = bounds.astype(np.uint64 if wide(dt) else np.uint32)
    le = torch.empty(bounds.size, dtype=torch.int64, device="cuda")
    rc = ns.nsort_count_le(dev(x), x.size, DT[dt], dev(bounds), bounds.size, le)
    assert rc == ns.OK
    want = np.searchsorted(k, bounds.astype(np.uint64), side="right")
    np.testing.assert_array_equal(le.cpu().numpy(), want)


def merge_gpu(ns, runs_keys, off, dt, vals=None):
    n = int(off[-1])
    kin = dev(runs_keys)
    kout = torch.empty_like(kin)
    vin = vout = None
    if vals is not None:
        vin = dev(vals)
        vout = torch.empty_like(vin)
    kind = ns.KIND_MERGE if vals is None else ns.KIND_MERGE_PAIRS
    tmp = ns.scratch(kind, n, len(off) - 1, dtype=DT[dt])
    rc = ns.nsort_merge_shards(kin, vin, kout, vout, off, DT[dt], tmp, tmp.numel())
    assert rc == ns.OK, ns.lib().nsort_last_error()
    return host(kout, dt), None if vals is None else vout.cpu().numpy().view(np.uint32)


MERGE_CASES = [(1, "u32", "uniform", 5000), (2, "u32", "uniform", 100_003),
               (3, "i32", "dup16", 77_777), (7, "f32", "specials", 250_001),
               (8, "u32", "sorted", 1 << 20), (16, "i32", "zipf", 300_007),
               (33, "f32", "reverse", 123_457), (64, "u32", "dup16", 500_009),
               (2, "u64", "uniform", 70_001), (5, "i64", "dup16", 90_001),
               (9, "f64", "specials", 120_003)]


@pytest.mark.parametrize("p,dt,dist,n", MERGE_CASES)
def test_merge_shards_keys_against_oracle(ns, p, dt, dist, n):
    """Runs of ragged and empty lengths, sorted by the oracle; their merge
    must equal the oracle's sort of their concatenation."""
    x = make_keys(n, dt, dist, seed=n)
    lens = shard_lengths(n, p, seed=n, empty=(0, p // 2) if p > 2 else ())
    keys, off = sorted_shards(x, lens, dt)
    got, _ = merge_gpu(ns, keys, off, dt)
    np.testing.assert_array_equal(got, osort(keys, dt))


@pytest.mark.parametrize("p,dt,dist", [(2, "f32", "specials"), (5, "i32", "dup16"),
                                       (12, "u32", "zipf"), (64, "f32", "dup16")])
def test_merge_shards_pairs_stable(ns, p, dt, dist):
    """Stable: equal keys keep run order, then position (payload = position
    in the concatenation)."""
    n = 200_003
    x = make_keys(n, dt, dist, seed=p)
    lens = shard_lengths(n, p, seed=p + 1, empty=(1,) if p > 2 else ())
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    v = np.arange(n, dtype=np.uint32)
    ks, vs = [], []
    for r in range(p):
        a, b = off[r], off[r + 1]
        k1, v1 = oracle.sort_pairs(x[a:b], v[a:b], dt)
        ks.append(k1)
        vs.append(v1)
    keys, vals = np.concatenate(ks), np.concatenate(vs)
    gk, gv = merge_gpu(ns, keys, off, dt, vals=vals)
    wk, wv = oracle.sort_pairs(keys, vals, dt)
    np.testing.assert_array_equal(gk, wk)
    np.testing.assert_array_equal(gv, wv)


def test_merge_shards_errors(ns):
    x = dev(np.arange(1024, dtype=np.uint32))
    y = torch.empty_like(x)
    tmp = ns.scratch(ns.KIND_MERGE, 1024, 2)
    assert ns.nsort_merge_shards(x, None, x, None, [0, 512, 1024], 0, tmp, tmp.numel()) == ns.EINVAL
    assert ns.nsort_merge_shards(x, None, y, None, [0, 600, 500, 1024], 0, tmp,
                                 tmp.numel()) == ns.EINVAL
    assert ns.nsort_merge_shards(x, None, y, None, [1, 512, 1024], 0, tmp, tmp.numel()) == ns.EINVAL
    assert ns.nsort_merge_shards(x[1:], None, y[1:], None, [0, 500, 1023], 0, tmp,
                                 tmp.numel()) == ns.EINVAL
    assert ns.nsort_merge_shards(x, None, y, None, [0, 512, 1024], 0, tmp, 16) == ns.ENOMEM
    assert ns.nsort_merge_shards(x, None, y, None, list(range(0, 1024, 8)) + [1024], 0, tmp,
                                 tmp.numel()) == ns.EINVAL          # 128 runs > 64
    cr = torch.empty(64, dtype=torch.int64, device="cuda")
    off = dev(np.zeros(34, np.int64))
    assert ns.nsort_shard_coranks(x, off, 33, off, 1, 0, cr) == ns.EINVAL


@pytest.mark.parametrize("p", [2, 3, 8])
@pytest.mark.parametrize("dt,dist", [("u32", "uniform"), ("f32", "zipf"), ("i32", "dup16")])
def test_sort_sharded_one_gpu(ns, p, dt, dist):
    from paper_2409_03970_gb300 import shard
    n = (1 << 22) + 5
    x = make_keys(n, dt, dist, seed=p)
    ko, _ = shard.sort_sharded_one_gpu(dev(x), p, DT[dt])
    np.testing.assert_array_equal(host(ko, dt), osort(x, dt))


@pytest.mark.parametrize("p", [2, 8])
def test_sort_sharded_one_gpu_pairs(ns, p):
    from paper_2409_03970_gb300 import shard
    n = 1_000_003
    k, v = inputs.normal_pairs(n, seed=p, special_per_mille=20)
    ko, vo = shard.sort_sharded_one_gpu(dev(k), p, DT["f32"], vals=dev(v))
    wk, wv = oracle.sort_pairs(k, v, "f32")
    np.testing.assert_array_equal(host(ko, "f32"), wk)
    np.testing.assert_array_equal(vo.cpu().numpy().view(np.uint32), wv)


def test_sort_sharded_one_gpu_u64(ns):
    from paper_2409_03970_gb300 import shard
    x = inputs.keys64(3_000_017, "f64", "specials", seed=4)
    ko, _ = shard.sort_sharded_one_gpu(dev(x), 4, DT["f64"])
    np.testing.assert_array_equal(host(ko, "f64"), oracle.sort_keys64(x, "f64"))


def test_sort_sharded_full_size_against_oracle(ns):
    """The 2^28 uniform uint32 workload as 8 shards on one GPU, compared
    element by element with the oracle."""
    import os
    from paper_2409_03970_gb300 import shard
    n = 1 << 28
    x = inputs.keys(n, "u32", "uniform", seed=0)
    ko, _ = shard.sort_sharded_one_gpu(dev(x), 8, DT["u32"])
    got = host(ko, "u32")
    del ko
    torch.cuda.empty_cache()
    threads = max(1, len(os.sched_getaffinity(0)))
    assert np.array_equal(got, oracle.sort_keys_par(x, "u32", threads))
