"""GPU parity for 64-bit keys (uint64 / int64 / float64 in IEEE totalOrder)
through nsort_keys, against the CPU oracle, bit for bit.  Sizes span the
4096-key tiles and the 1920-key merge tiles with ragged tails; every dtype
and distribution; in-place and 8-byte-aligned (not 16-byte-aligned)
buffers, which take the staged-load merge pass; and a full-size 2^27-key
(1 GiB) workload."""
import numpy as np
import pytest

import oracle
from paper_2409_03970_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"u64": 3, "i64": 4, "f64": 5}


@pytest.fixture(scope="module")
def ns():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03970_gb300 import build, nsort
    build.build()
    nsort.lib()
    return nsort


def dev(bits):
    return torch.from_numpy(np.ascontiguousarray(bits, dtype=np.uint64).view(np.int64)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint64)


def gpu_sort64(ns, bits, dt, inplace=False, offset=0):
    n = bits.size
    x = dev(np.concatenate([np.zeros(offset, np.uint64), bits]))[offset:]
    out = x if inplace else torch.empty(n + offset, dtype=torch.int64, device="cuda")[offset:]
    tmp = ns.scratch(ns.KIND_KEYS, n, dtype=DT[dt])
    rc = ns.nsort_keys(x, out, n, DT[dt], tmp, tmp.numel())
    assert rc == ns.OK, ns.lib().nsort_last_error()
    if tmp.numel() >= 256:
        assert ns.nsort_device_status(tmp) == ns.OK
    return host(out)


SIZES = [0, 1, 2, 3, 1919, 1920, 1921, 4095, 4096, 4097, 8191, 8192, 8193,
         3 * 4096 + 5, 65537, 100_003, 1 << 20, (1 << 20) + 12345]


@pytest.mark.parametrize("n", SIZES)
def test_keys64_u64_uniform_sizes(ns, n):
    x = inputs.keys64(n, "u64", "uniform", seed=n)
    assert np.array_equal(gpu_sort64(ns, x, "u64"), oracle.sort_keys64(x, "u64"))


@pytest.mark.parametrize("dt", ["u64", "i64", "f64"])
@pytest.mark.parametrize("dist", list(inputs.DISTRIBUTIONS64))
@pytest.mark.parametrize("n", [5000, 300_001])
def test_keys64_all_dtypes_distributions(ns, dt, dist, n):
    x = inputs.keys64(n, dt, dist, seed=7)
    assert np.array_equal(gpu_sort64(ns, x, dt), oracle.sort_keys64(x, dt))


def test_keys64_f64_totalorder_table(ns, golden):
    """Every binary64 special of the totalOrder table, shuffled and repeated."""
    rows = golden("f64_total_order.txt")
    table = np.array([int(r[0], 16) for r in rows], dtype=np.uint64)
    pick = inputs.counter_u64(8, 0, 0, 50_000) % np.uint64(table.size)
    x = table[pick.astype(np.int64)]
    got = gpu_sort64(ns, x, "f64")
    assert np.array_equal(got, oracle.sort_keys64(x, "f64"))
    # the output walks the table in order
    first = [int(np.argmax(got == v)) for v in table if np.any(got == v)]
    assert first == sorted(first)


@pytest.mark.parametrize("point", [1, 2])
@pytest.mark.parametrize("extra", [0, 1])
def test_keys64_splitter_modes(ns, point, extra):
    """Sizes at the boundaries between merge passes that find their own
    splitters (at most one, or two, merge tiles per CTA of the persistent
    merge grid on this device) and passes that launch the partition kernel."""
    grid = ns.nsort_merge_grid(ns.KIND_KEYS, DT["i64"])
    assert grid > 0
    tile = ns.nsort_plan(ns.KIND_KEYS, 1 << 24, DT["i64"])[2]
    n = point * grid * tile + extra
    x = inputs.keys64(n, "i64", "dup16", seed=n)
    assert np.array_equal(gpu_sort64(ns, x, "i64"), oracle.sort_keys64(x, "i64"))


@pytest.mark.parametrize("n", [4096, 70_000, 1 << 19])
def test_keys64_in_place(ns, n):
    x = inputs.keys64(n, "i64", "uniform", seed=9)
    assert np.array_equal(gpu_sort64(ns, x, "i64", inplace=True), oracle.sort_keys64(x, "i64"))


@pytest.mark.parametrize("n", [4097, 77_777, 1 << 20])
def test_keys64_8_byte_aligned_buffers(ns, n):
    """Buffers 8 bytes past a 16-byte boundary: the merge passes take the
    staged-load fallback (bulk copies need 16-byte alignment)."""
    x = inputs.keys64(n, "f64", "specials", seed=10)
    assert np.array_equal(gpu_sort64(ns, x, "f64", offset=1), oracle.sort_keys64(x, "f64"))


def test_keys64_scratch_too_small_is_rejected(ns):
    n = 1 << 16
    x = dev(inputs.keys64(n, "u64", "uniform", seed=1))
    tmp = ns.scratch(ns.KIND_KEYS, n, dtype=DT["u64"])
    rc = ns.nsort_keys(x, x, n, DT["u64"], tmp, tmp.numel() - 1)
    assert rc == ns.ENOMEM


@pytest.mark.parametrize("dt,dist", [("u64", "uniform"), ("i64", "uniform"), ("f64", "uniform"),
                                     ("f64", "specials")])
def test_full_size_keys64_against_oracle(ns, dt, dist):
    """The benchmark's 64-bit key workloads: 2^27 keys (1 GiB) of each
    dtype, on the benchmark's own inputs and launch configuration, compared
    element by element."""
    n = 1 << 27
    x = inputs.keys64(n, dt, dist, seed=0)
    got = gpu_sort64(ns, x, dt)
    assert np.array_equal(got, oracle.sort_keys64(x, dt))
