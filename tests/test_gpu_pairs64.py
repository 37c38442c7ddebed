"""GPU parity of nsort_pairs64 (32-bit keys with 64-bit payloads) against
the oracle, bit for bit.  The oracle's stable pair sort with payload =
input position gives the stable order; the expected payloads are the 64-bit
inputs taken in that order.  Sizes span one to many tiles with ragged
tails; every key dtype, heavy ties, IEEE specials, in place; misaligned
payloads or outputs are rejected."""
import numpy as np
import pytest

import oracle
from paper_2409_03970_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"u32": 0, "i32": 1, "f32": 2}


@pytest.fixture(scope="module")
def ns():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03970_gb300 import build, nsort
    build.build()
    nsort.lib()
    return nsort


def expected(k, v64, dt):
    wk, pos = oracle.sort_pairs(k, np.arange(k.size, dtype=np.uint32), dt)
    return wk, v64[pos.astype(np.int64)]


def gpu_pairs64(ns, k, v64, dt, inplace=False):
    n = k.size
    kt = torch.from_numpy(np.ascontiguousarray(k).view(np.int32)).cuda()
    vt = torch.from_numpy(np.ascontiguousarray(v64).view(np.int64)).cuda()
    ko, vo = (kt, vt) if inplace else (torch.empty_like(kt), torch.empty_like(vt))
    tmp = ns.scratch(ns.KIND_PAIRS64, n)
    rc = ns.nsort_pairs64(kt, vt, ko, vo, n, DT[dt], tmp, tmp.numel())
    assert rc == ns.OK, ns.lib().nsort_last_error()
    return ko.cpu().numpy().view(np.uint32), vo.cpu().numpy().view(np.uint64)


SIZES = [0, 1, 2, 17, 4095, 8191, 8192, 8193, 3 * 8192 + 5, 100_003, (1 << 20) + 7]


@pytest.mark.parametrize("n", SIZES)
def test_pairs64_sizes(ns, n):
    k = inputs.keys(n, "u32", "dup16" if n % 2 else "uniform", seed=n)
    v = inputs.counter_u64(n, 11, 0, n)
    gk, gv = gpu_pairs64(ns, k, v, "u32")
    wk, wv = expected(k, v, "u32")
    np.testing.assert_array_equal(gk, wk)
    np.testing.assert_array_equal(gv, wv)


@pytest.mark.parametrize("dt", ["u32", "i32", "f32"])
@pytest.mark.parametrize("dist", ["dup16", "zipf", "sorted", "reverse"])
def test_pairs64_stability_heavy_duplicates(ns, dt, dist):
    n = 300_007
    k = inputs.keys(n, dt, dist, seed=6)
    v = inputs.counter_u64(6, 12, 0, n)
    gk, gv = gpu_pairs64(ns, k, v, dt)
    wk, wv = expected(k, v, dt)
    np.testing.assert_array_equal(gk, wk)
    np.testing.assert_array_equal(gv, wv)


def test_pairs64_ieee_specials_large(ns):
    n = (1 << 24) + 3
    k, _ = inputs.normal_pairs(n, seed=7, special_per_mille=10)
    v = inputs.counter_u64(7, 13, 0, n)
    gk, gv = gpu_pairs64(ns, k, v, "f32")
    wk, wv = expected(k, v, "f32")
    np.testing.assert_array_equal(gk, wk)
    np.testing.assert_array_equal(gv, wv)


@pytest.mark.parametrize("n", [5000, 70_001])
def test_pairs64_in_place(ns, n):
    k = inputs.keys(n, "i32", "dup16", seed=8)
    v = inputs.counter_u64(8, 14, 0, n)
    gk, gv = gpu_pairs64(ns, k, v, "i32", inplace=True)
    wk, wv = expected(k, v, "i32")
    np.testing.assert_array_equal(gk, wk)
    np.testing.assert_array_equal(gv, wv)


def test_pairs64_rejects_misaligned_buffers(ns):
    n = 1 << 16
    k = torch.zeros(n + 4, dtype=torch.int32, device="cuda")
    v = torch.zeros(n + 2, dtype=torch.int64, device="cuda")
    tmp = ns.scratch(ns.KIND_PAIRS64, n)
    vb = v.view(torch.int32)
    # payloads 4 bytes off an 8-byte boundary
    assert ns.nsort_pairs64(k[:n], vb[1:].data_ptr(), k[:n], vb[1:].data_ptr(), n, 0, tmp,
                            tmp.numel()) == ns.EINVAL
    # outputs 8 bytes off a 16-byte boundary
    assert ns.nsort_pairs64(k[:n], v[:n], k[2:n + 2], v[1:n + 1], n, 0, tmp,
                            tmp.numel()) == ns.EINVAL
    assert ns.nsort_pairs64(k[:n], v[:n], k[:n], v[:n], n, 0, tmp, tmp.numel() - 1) == ns.ENOMEM


def test_full_size_pairs64_against_oracle(ns):
    """The benchmark's 64-bit payload workload: 2^27 float32 Normal(0,1)
    keys with 0.1% IEEE specials and payloads 0, 1, 2, ... as 64-bit words,
    compared element by element (keys and payloads)."""
    n = 1 << 27
    k, _ = inputs.normal_pairs(n, seed=0)
    v = np.arange(n, dtype=np.uint64)
    gk, gv = gpu_pairs64(ns, k, v, "f32")
    wk, wv = expected(k, v, "f32")
    np.testing.assert_array_equal(gk, wk)
    np.testing.assert_array_equal(gv, wv)
