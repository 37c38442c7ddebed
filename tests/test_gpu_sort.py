"""GPU parity: libnsort (through the C ABI) against the CPU oracle, bit for
bit, on seeded inputs.  Sizes span one to many tiles with ragged tails;
every dtype and input distribution; in-place and misaligned buffers; the
full-size benchmark workloads (2^28 keys, 2^27 pairs)."""
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


def dev(bits):
    return torch.from_numpy(np.ascontiguousarray(bits).view(np.int32)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint32)


def gpu_sort(ns, bits, dt, inplace=False, offset=0):
    n = bits.size
    x = dev(np.concatenate([np.zeros(offset, np.uint32), bits]))[offset:]
    out = x if inplace else torch.empty(n + offset, dtype=torch.int32, device="cuda")[offset:]
    tmp = ns.scratch(ns.KIND_KEYS, n)
    rc = ns.nsort_keys(x, out, n, DT[dt], tmp, tmp.numel())
    assert rc == ns.OK, ns.lib().nsort_last_error()
    return host(out)


def gpu_pairs(ns, k, v, dt, inplace=False):
    n = k.size
    kt, vt = dev(k), dev(v)
    ko, vo = (kt, vt) if inplace else (torch.empty_like(kt), torch.empty_like(vt))
    tmp = ns.scratch(ns.KIND_PAIRS, n)
    rc = ns.nsort_pairs(kt, vt, ko, vo, n, DT[dt], tmp, tmp.numel())
    assert rc == ns.OK, ns.lib().nsort_last_error()
    return host(ko), host(vo)


SIZES = [0, 1, 2, 3, 15, 16, 17, 511, 512, 513, 4095, 4096, 4097, 8191, 8192, 8193,
         16383, 16384, 16385, 3 * 8192 + 5, 3 * 16384 + 7, 65536 + 1, 100_003, 1 << 20,
         (1 << 20) + 12345]


@pytest.mark.parametrize("n", SIZES)
def test_keys_u32_uniform_sizes(ns, n):
    x = inputs.keys(n, "u32", "uniform", seed=n)
    np.testing.assert_array_equal(gpu_sort(ns, x, "u32"), oracle.sort_keys(x, "u32"))


@pytest.mark.parametrize("dt", ["u32", "i32", "f32"])
@pytest.mark.parametrize("dist", list(inputs.DISTRIBUTIONS))
@pytest.mark.parametrize("n", [8193, 250_001, (1 << 21) + 3])
def test_keys_all_dtypes_distributions(ns, dt, dist, n):
    x = inputs.keys(n, dt, dist, seed=1)
    np.testing.assert_array_equal(gpu_sort(ns, x, dt), oracle.sort_keys(x, dt))


# Where the merge passes find their splitters: a pass with at most one or
# two merge tiles per CTA of the persistent merge grid (SMs x resident CTAs,
# from nsort_merge_grid on this device) finds its own splitters inside the
# merge kernel; larger passes launch the partition kernel.  The last pass
# has about n / merge_tile tiles, so these sizes straddle both boundaries on
# whatever device runs the tests.
MODE_POINTS = ["1x", "1x+1", "1.5x", "2x", "2x+1", "2.1x"]


def mode_size(ns, kind, dtype, point):
    grid = ns.nsort_merge_grid(kind, dtype)
    assert grid > 0, ns.lib().nsort_last_error()
    tile = ns.nsort_plan(kind, 1 << 24, dtype)[2]
    one, two = grid * tile, 2 * grid * tile
    return {"1x": one, "1x+1": one + 1, "1.5x": (one + two) // 2 + 17, "2x": two,
            "2x+1": two + 1, "2.1x": two + two // 20 + 11}[point]


@pytest.mark.parametrize("dist", ["uniform", "sorted", "dup16"])
@pytest.mark.parametrize("point", MODE_POINTS)
def test_keys_splitter_modes(ns, point, dist):
    n = mode_size(ns, ns.KIND_KEYS, ns.U32, point)
    x = inputs.keys(n, "f32", dist, seed=n)
    np.testing.assert_array_equal(gpu_sort(ns, x, "f32"), oracle.sort_keys(x, "f32"))


@pytest.mark.parametrize("point", ["1x", "1x+1", "2x", "2x+1"])
def test_pairs_splitter_modes(ns, point):
    n = mode_size(ns, ns.KIND_PAIRS, ns.U32, point)
    k = inputs.keys(n, "i32", "dup16", seed=n)
    v = inputs.counter_u32(5, 6, 0, n)
    ko, vo = gpu_pairs(ns, k, v, "i32")
    wk, wv = oracle.sort_pairs(k, v, "i32")
    np.testing.assert_array_equal(ko, wk)
    np.testing.assert_array_equal(vo, wv)


@pytest.mark.parametrize("dt", ["u32", "i32", "f32"])
@pytest.mark.parametrize("n", [1, 300, 512, 513, 2048, 2049, 5000, 8192])
def test_keys_small_single_cta_sorts(ns, dt, n):
    """Sorts of at most 8192 keys run in one CTA of 512, 2048 or 8192 keys;
    every dtype at each size edge, misaligned and in place too."""
    x = inputs.keys(n, dt, "dup16" if n % 2 else "uniform", seed=n)
    want = oracle.sort_keys(x, dt)
    np.testing.assert_array_equal(gpu_sort(ns, x, dt), want)
    np.testing.assert_array_equal(gpu_sort(ns, x, dt, offset=1), want)
    np.testing.assert_array_equal(gpu_sort(ns, x, dt, inplace=True), want)


def test_keys_f32_specials_and_nan_payloads(ns):
    k, _ = inputs.normal_pairs(300_000, seed=2, special_per_mille=100)
    extra = np.array([0xFFFFFFFF, 0xFFC00001, 0xFF800001, 0x7F800001, 0x7FBFFFFF,
                      0x7FFFFFFF, 0x00000001, 0x80000001, 0x007FFFFF, 0x807FFFFF], np.uint32)
    k = np.concatenate([k, np.repeat(extra, 100)])
    np.testing.assert_array_equal(gpu_sort(ns, k, "f32"), oracle.sort_keys(k, "f32"))


@pytest.mark.parametrize("n", [5, 8192, 40_000, 1 << 20])
def test_keys_in_place(ns, n):
    x = inputs.keys(n, "i32", "zipf", seed=3)
    np.testing.assert_array_equal(gpu_sort(ns, x, "i32", inplace=True), oracle.sort_keys(x, "i32"))


@pytest.mark.parametrize("offset", [1, 2, 3])
def test_keys_misaligned_buffers(ns, offset):
    x = inputs.keys(70_001, "u32", "uniform", seed=offset)
    np.testing.assert_array_equal(gpu_sort(ns, x, "u32", offset=offset), oracle.sort_keys(x, "u32"))


@pytest.mark.parametrize("n", [0, 1, 2, 17, 4095, 4096, 4097, 12289, 100_000, 1 << 20, (1 << 20) + 7])
def test_pairs_normal_with_specials(ns, n):
    k, v = inputs.normal_pairs(n, seed=n, special_per_mille=5)
    ko, vo = gpu_pairs(ns, k, v, "f32")
    wk, wv = oracle.sort_pairs(k, v, "f32")
    np.testing.assert_array_equal(ko, wk)
    np.testing.assert_array_equal(vo, wv)


@pytest.mark.parametrize("dt", ["u32", "i32", "f32"])
@pytest.mark.parametrize("dist", ["dup16", "zipf", "sorted", "reverse"])
def test_pairs_stability_heavy_duplicates(ns, dt, dist):
    n = 300_007
    k = inputs.keys(n, dt, dist, seed=4)
    v = inputs.counter_u32(4, 6, 0, n)            # arbitrary payloads, not the index
    ko, vo = gpu_pairs(ns, k, v, dt)
    wk, wv = oracle.sort_pairs(k, v, dt)
    np.testing.assert_array_equal(ko, wk)
    np.testing.assert_array_equal(vo, wv)


def test_pairs_in_place(ns):
    k = inputs.keys(50_000, "u32", "dup16", seed=5)
    v = np.arange(k.size, dtype=np.uint32)
    ko, vo = gpu_pairs(ns, k, v, "u32", inplace=True)
    wk, wv = oracle.sort_pairs(k, v, "u32")
    np.testing.assert_array_equal(ko, wk)
    np.testing.assert_array_equal(vo, wv)


def test_scratch_too_small_is_rejected(ns):
    n = 1 << 16
    x = dev(inputs.keys(n, "u32", "uniform", seed=0))
    tmp = ns.scratch(ns.KIND_KEYS, n)
    assert ns.nsort_keys(x, x, n, 0, tmp, tmp.numel() - 1) == ns.ENOMEM


# ---- full-size benchmark workloads -----------------------------------------

def test_full_size_u32_uniform_against_oracle(ns):
    """The benchmark workload, 2^28 uniform uint32 keys, seed 0, in the
    launch configuration the benchmark times, compared element by element."""
    n = 1 << 28
    x = inputs.keys(n, "u32", "uniform", seed=0)
    got = gpu_sort(ns, x, "u32")
    want = oracle.sort_keys(x, "u32")
    assert np.array_equal(got, want)


def host_threads():
    """Host cores this process may run on (the oracle's multi-threaded form
    uses all of them)."""
    import os
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


@pytest.mark.parametrize("dt", ["i32", "f32"])
@pytest.mark.parametrize("dist", list(inputs.DISTRIBUTIONS))
def test_full_size_against_oracle(ns, dt, dist):
    """The 2^28-key workloads of each dtype and distribution, in the launch
    configuration the benchmark times, compared element by element with the
    oracle (its multi-threaded form, which equals the serial sort: the
    oracle's own tests check that)."""
    n = 1 << 28
    x = inputs.keys(n, dt, dist, seed=2)
    got = gpu_sort(ns, x, dt)
    torch.cuda.empty_cache()
    want = oracle.sort_keys_par(x, dt, host_threads())
    del x
    assert np.array_equal(got, want)


def test_full_size_pairs_against_oracle(ns):
    """2^27 float32 Normal(0,1) keys with 0.1% IEEE specials, payload = index."""
    n = 1 << 27
    k, v = inputs.normal_pairs(n, seed=0)
    ko, vo = gpu_pairs(ns, k, v, "f32")
    wk, wv = oracle.sort_pairs(k, v, "f32")
    assert np.array_equal(ko, wk)
    assert np.array_equal(vo, wv)


# ---- dependent launches ------------------------------------------------------

def test_sort_captured_in_a_cuda_graph(ns):
    """nsort_keys and nsort_pairs captured into one CUDA graph (their
    partition and merge kernels are dependent launches) and replayed on new
    data give the oracle's result."""
    n = 3 * 16384 + 11
    x = torch.empty(n, dtype=torch.int32, device="cuda")
    y = torch.empty_like(x)
    kv, vv = torch.empty_like(x), torch.empty_like(x)
    ko, vo = torch.empty_like(x), torch.empty_like(x)
    tk = ns.scratch(ns.KIND_KEYS, n)
    tp = ns.scratch(ns.KIND_PAIRS, n)
    s = torch.cuda.Stream()
    x.zero_()
    kv.zero_()
    vv.zero_()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):      # one-time set-up (shared-memory opt-ins) before capture
        assert ns.nsort_keys(x, y, n, DT["f32"], tk, tk.numel(), s) == ns.OK
        assert ns.nsort_pairs(kv, vv, ko, vo, n, DT["u32"], tp, tp.numel(), s) == ns.OK
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        assert ns.nsort_keys(x, y, n, DT["f32"], tk, tk.numel(), s) == ns.OK
        assert ns.nsort_pairs(kv, vv, ko, vo, n, DT["u32"], tp, tp.numel(), s) == ns.OK
    for seed in (1, 2):
        bits = inputs.keys(n, "f32", "dup16", seed=seed)
        kb = inputs.keys(n, "u32", "zipf", seed=seed)
        vb = np.arange(n, dtype=np.uint32)
        x.copy_(dev(bits))
        kv.copy_(dev(kb))
        vv.copy_(dev(vb))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(host(y), oracle.sort_keys(bits, "f32"))
        wk, wv = oracle.sort_pairs(kb, vb, "u32")
        assert np.array_equal(host(ko), wk) and np.array_equal(host(vo), wv)


def test_plain_launches_give_the_same_result(ns, tmp_path):
    """NSORT_NO_PDL=1 (read once per process) selects plain launches; a
    child process sorting that way matches the oracle."""
    import subprocess
    import sys
    import textwrap
    root = __import__("os").path.dirname(__import__("os").path.dirname(__file__))
    code = textwrap.dedent("""
        import sys, numpy as np, torch
        sys.path.insert(0, %r)
        import oracle
        from paper_2409_03970_gb300 import inputs, nsort
        n = (1 << 20) + 77
        bits = inputs.keys(n, "i32", "uniform", seed=3)
        x = torch.from_numpy(bits.view(np.int32)).cuda()
        tmp = nsort.scratch(nsort.KIND_KEYS, n)
        assert nsort.nsort_keys(x, x, n, nsort.I32, tmp, tmp.numel()) == nsort.OK
        assert np.array_equal(x.cpu().numpy().view(np.uint32), oracle.sort_keys(bits, "i32"))
        print("ok")
    """ % root)
    env = dict(__import__("os").environ, NSORT_NO_PDL="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
