"""GPU parity of the four-way merge passes (two merge levels per pass over
the array) against the oracle, bit for bit.  The test hook turns them on
for every sort with two or more merge levels, so that small arrays cover
groups of one to four runs, ragged last runs and groups, a one-level pass
before the four-way ones, every dtype and input distribution (heavy ties
included), in place and misaligned outputs (which take the staged-load
passes instead)."""
import numpy as np
import pytest

import oracle
from paper_2409_03970_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"u32": 0, "i32": 1, "f32": 2}
TILE = 16384   # keys per tile sort: the runs of the first merge level


@pytest.fixture(scope="module")
def ns():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03970_gb300 import build, nsort
    build.build()
    nsort.lib()
    assert nsort.nsort_plan(nsort.KIND_KEYS, 1 << 20)[1] == TILE
    prev = nsort.nsort_testing_set_four_way_min(0)
    try:
        yield nsort
    finally:
        nsort.nsort_testing_set_four_way_min(prev)


def gpu_sort(ns, bits, dt, inplace=False, offset=0, trace=False):
    n = bits.size
    x = torch.from_numpy(np.concatenate([np.zeros(offset, np.uint32), bits]).view(np.int32)).cuda()
    x = x[offset:]
    out = x if inplace else torch.empty(n + offset, dtype=torch.int32, device="cuda")[offset:]
    tmp = ns.scratch(ns.KIND_KEYS, n)
    if trace:
        ns.nsort_trace_enable(True)
    rc = ns.nsort_keys(x, out, n, DT[dt], tmp, tmp.numel())
    assert rc == ns.OK, ns.lib().nsort_last_error()
    if tmp.numel() > 1:
        assert ns.nsort_device_status(tmp) == ns.OK
    res = out.cpu().numpy().view(np.uint32)
    if trace:
        tr = ns.nsort_trace_read()
        ns.nsort_trace_enable(False)
        return res, tr
    return res


# merge levels 2 (one four-way pass), 3 (a two-way pass, then a four-way
# one), 4, 5, 6 and 10; groups of 1-4 runs; ragged runs and groups.  At
# 2^23 + 5 the last pass's group holds 131,073 samples: its partition
# chunks (4096 merged samples each) start on a tile boundary (rank
# 126,976 = 62 x 2048)
SIZES = [2 * TILE + 1, 3 * TILE, 3 * TILE + 7, 4 * TILE, 4 * TILE + 5, 5 * TILE + 1,
         8 * TILE - 3, 9 * TILE + 63, 16 * TILE + 1, 100_003, 1 << 20, (1 << 20) + 12345,
         5 * (1 << 20) - 3, (1 << 23) + 5]


@pytest.mark.parametrize("n", SIZES)
def test_four_way_sizes(ns, n):
    x = inputs.keys(n, "u32", "uniform", seed=n)
    got, tr = gpu_sort(ns, x, "u32", trace=True)
    np.testing.assert_array_equal(got, oracle.sort_keys(x, "u32"))
    levels = int(np.ceil(np.log2(-(-n // TILE))))
    assert tr["merge4_keys"]["launches"] == levels // 2
    assert tr.get("merge_keys", {"launches": 0})["launches"] == levels % 2


@pytest.mark.parametrize("dt", ["u32", "i32", "f32"])
@pytest.mark.parametrize("dist", list(inputs.DISTRIBUTIONS))
@pytest.mark.parametrize("n", [4 * TILE + 3, 250_001, (1 << 21) + 3])
def test_four_way_dtypes_distributions(ns, dt, dist, n):
    x = inputs.keys(n, dt, dist, seed=2)
    np.testing.assert_array_equal(gpu_sort(ns, x, dt), oracle.sort_keys(x, dt))


@pytest.mark.parametrize("distinct", [1, 2, 3, 64, 65])
def test_four_way_few_distinct_keys(ns, distinct):
    # long stretches of equal keys put many tile boundaries on one key value:
    # their co-ranks then follow the stable order alone
    n = 6 * TILE + 11
    x = (inputs.counter_u32(distinct, 3, 0, n) % np.uint32(distinct)).astype(np.uint32)
    np.testing.assert_array_equal(gpu_sort(ns, x, "u32"), oracle.sort_keys(x, "u32"))


def test_four_way_skewed_runs(ns):
    # each run holds keys of one band only (bands interleaved across runs),
    # so tiles take most of their keys from one or two runs
    n = 8 * TILE + 9
    i = np.arange(n, dtype=np.uint64)
    band = (i // TILE) % 4
    low = inputs.counter_u32(9, 4, 0, n) & np.uint32(0x3FFFFFFF)
    x = ((np.uint64(3) - band) << np.uint64(30)).astype(np.uint32) | low
    np.testing.assert_array_equal(gpu_sort(ns, x, "u32"), oracle.sort_keys(x, "u32"))


def test_four_way_ieee_specials(ns):
    n = (1 << 20) + 77
    k, _ = inputs.normal_pairs(n, seed=4, special_per_mille=10)
    np.testing.assert_array_equal(gpu_sort(ns, k, "f32"), oracle.sort_keys(k, "f32"))


@pytest.mark.parametrize("n", [4 * TILE + 1, 700_001])
def test_four_way_in_place(ns, n):
    x = inputs.keys(n, "i32", "dup16", seed=5)
    np.testing.assert_array_equal(gpu_sort(ns, x, "i32", inplace=True),
                                  oracle.sort_keys(x, "i32"))


@pytest.mark.parametrize("offset", [1, 3])
def test_four_way_misaligned_output_falls_back(ns, offset):
    n = 6 * TILE + 5
    x = inputs.keys(n, "u32", "uniform", seed=6)
    np.testing.assert_array_equal(gpu_sort(ns, x, "u32", offset=offset),
                                  oracle.sort_keys(x, "u32"))


def test_four_way_and_two_way_agree(ns):
    # the same sort with one-level passes only gives the same bits
    n = (1 << 22) + 9
    x, _ = inputs.normal_pairs(n, seed=7, special_per_mille=10)
    four = gpu_sort(ns, x, "f32")
    prev = ns.nsort_testing_set_four_way_min(ns.FOUR_WAY_NEVER)
    try:
        two = gpu_sort(ns, x, "f32")
    finally:
        ns.nsort_testing_set_four_way_min(prev)
    np.testing.assert_array_equal(four, two)
    np.testing.assert_array_equal(four, oracle.sort_keys(x, "f32"))
