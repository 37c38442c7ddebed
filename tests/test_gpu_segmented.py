"""GPU parity of nsort_segmented against the CPU oracle (bit for bit):
every length bin (one thread, one warp, one CTA, multi-level), every
tuning configuration, keys and stable pairs, empty segments, in-place,
malformed offsets, CUDA-graph capture and replay, and the on-GPU sorting
networks checked exhaustively by the 0-1 principle through the one-thread
bin."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2409_03970_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"u32": 0, "i32": 1, "f32": 2}
CONFIGS = [dict(block_threads=b, tiny_width=w, small_ipt=i, blocks_per_sm=0)
           for b, w, i in itertools.product((256, 512), (8, 16), (8, 16))]


@pytest.fixture(scope="module")
def ns():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03970_gb300 import build, nsort
    build.build()
    nsort.lib()
    yield nsort
    nsort.nsort_segmented_set_config()


def dev(a, dtype=np.int32):
    return torch.from_numpy(np.ascontiguousarray(a).view(dtype)).cuda()


def mixed_offsets(seed, extra=()):
    """Lengths covering every bin and its edges, plus log-uniform ones."""
    edges = [0, 1, 2, 7, 8, 9, 15, 16, 17, 255, 256, 257, 511, 512, 513, 4095, 4096, 4097,
             8191, 8192, 8193, 16383, 16384, 16385, 32767, 32768, 32769, 40000, 65536,
             100_003]
    rnd = np.diff(inputs.segment_offsets(300, seed=seed, max_len=65536))
    lens = np.array(list(edges) + list(rnd) + list(extra), dtype=np.int64)
    rng_perm = inputs.counter_u64(seed, 7, 0, lens.size).argsort()
    lens = lens[rng_perm]
    off = np.zeros(lens.size + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    return off


def run_seg(ns, keys, off, dt, vals=None, inplace=False):
    n, nseg = keys.size, off.size - 1
    kt = dev(keys)
    ko = kt if inplace else torch.empty_like(kt)
    vt = vo = None
    if vals is not None:
        vt = dev(vals)
        vo = vt if inplace else torch.empty_like(vt)
    ot = dev(off, np.int64)
    kind = ns.KIND_SEGMENTED if vals is None else ns.KIND_SEGMENTED_PAIRS
    tmp = ns.scratch(kind, n, nseg)
    rc = ns.nsort_segmented(kt, ko, vt, vo, ot, nseg, n, DT[dt], tmp, tmp.numel())
    assert rc == ns.OK, ns.lib().nsort_last_error()
    assert ns.nsort_device_status(tmp) == ns.OK
    k = ko.cpu().numpy().view(np.uint32)
    return k if vals is None else (k, vo.cpu().numpy().view(np.uint32))


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: f"nt{c['block_threads']}-w{c['tiny_width']}-ipt{c['small_ipt']}")
def test_keys_all_bins_all_configs(ns, cfg):
    assert ns.nsort_segmented_set_config(**cfg) == ns.OK
    off = mixed_offsets(1)
    x = inputs.keys(int(off[-1]), "u32", "uniform", seed=1)
    np.testing.assert_array_equal(run_seg(ns, x, off, "u32"), oracle.sort_segmented(x, off, "u32"))


@pytest.mark.parametrize("cfg", [CONFIGS[0], CONFIGS[-1]], ids=["nt256-w8-ipt8", "nt512-w16-ipt16"])
@pytest.mark.parametrize("dt", ["u32", "i32", "f32"])
def test_pairs_all_bins_stable(ns, cfg, dt):
    assert ns.nsort_segmented_set_config(**cfg) == ns.OK
    off = mixed_offsets(2)
    n = int(off[-1])
    k = inputs.keys(n, dt, "dup16", seed=2)                       # heavy ties: stability
    v = np.arange(n, dtype=np.uint32)
    ko, vo = run_seg(ns, k, off, dt, vals=v)
    wk, wv = oracle.sort_segmented(k, off, dt, vals=v)
    np.testing.assert_array_equal(ko, wk)
    np.testing.assert_array_equal(vo, wv)


@pytest.mark.parametrize("dist", ["uniform", "sorted", "reverse", "zipf"])
def test_keys_distributions_f32(ns, dist):
    ns.nsort_segmented_set_config()
    off = mixed_offsets(3)
    x = inputs.keys(int(off[-1]), "f32", dist, seed=3)
    np.testing.assert_array_equal(run_seg(ns, x, off, "f32"), oracle.sort_segmented(x, off, "f32"))


def test_pairs_ieee_specials_in_place(ns):
    ns.nsort_segmented_set_config()
    off = mixed_offsets(4)
    n = int(off[-1])
    k, v = inputs.normal_pairs(n, seed=4, special_per_mille=50)
    ko, vo = run_seg(ns, k, off, "f32", vals=v, inplace=True)
    wk, wv = oracle.sort_segmented(k, off, "f32", vals=v)
    np.testing.assert_array_equal(ko, wk)
    np.testing.assert_array_equal(vo, wv)


def test_empty_and_single_segments(ns):
    ns.nsort_segmented_set_config()
    for lens in ([0], [0, 0, 0], [5], [0, 1, 0], [70000], [0, 70000, 0]):
        off = np.zeros(len(lens) + 1, np.int64)
        np.cumsum(lens, out=off[1:])
        x = inputs.keys(int(off[-1]), "i32", "uniform", seed=len(lens))
        np.testing.assert_array_equal(run_seg(ns, x, off, "i32"), oracle.sort_segmented(x, off, "i32"))


def test_malformed_offsets_reported(ns):
    ns.nsort_segmented_set_config()
    x = dev(inputs.keys(1000, "u32", "uniform", seed=5))
    out = torch.empty_like(x)
    for bad in ([0, 600, 500, 1000], [1, 500, 1000], [0, 500, 999]):
        off = dev(np.array(bad, np.int64), np.int64)
        tmp = ns.scratch(ns.KIND_SEGMENTED, 1000, len(bad) - 1)
        rc = ns.nsort_segmented(x, out, None, None, off, len(bad) - 1, 1000, 0, tmp, tmp.numel())
        assert rc == ns.OK
        assert ns.nsort_device_status(tmp) == ns.EINVAL


def test_zero_one_principle_16_input_network_on_gpu(ns):
    """All 2^16 0-1 inputs of length 16, one segment each, through the
    one-thread bin (tiny_width 16): every segment must come out sorted."""
    assert ns.nsort_segmented_set_config(tiny_width=16) == ns.OK
    x = np.arange(1 << 16, dtype=np.uint32)
    bits = ((x[:, None] >> np.arange(16, dtype=np.uint32)) & 1).astype(np.uint32).ravel()
    off = np.arange(0, bits.size + 1, 16, dtype=np.int64)
    y = run_seg(ns, bits, off, "u32").reshape(-1, 16)
    assert np.all(y[:, :-1] <= y[:, 1:])
    np.testing.assert_array_equal(y.sum(axis=1), bits.reshape(-1, 16).sum(axis=1))


def test_zero_one_principle_8_input_network_on_gpu(ns):
    assert ns.nsort_segmented_set_config(tiny_width=8) == ns.OK
    x = np.arange(1 << 8, dtype=np.uint32)
    bits = ((x[:, None] >> np.arange(8, dtype=np.uint32)) & 1).astype(np.uint32).ravel()
    off = np.arange(0, bits.size + 1, 8, dtype=np.int64)
    y = run_seg(ns, bits, off, "u32").reshape(-1, 8)
    assert np.all(y[:, :-1] <= y[:, 1:])
    np.testing.assert_array_equal(y.sum(axis=1), bits.reshape(-1, 8).sum(axis=1))


def test_cuda_graph_capture_and_replay(ns):
    """One nsort_segmented captured into a CUDA graph, replayed on new keys
    copied into the captured input buffer before each replay: every replay
    sorts the data it finds there."""
    ns.nsort_segmented_set_config()
    off = mixed_offsets(6)
    n, nseg = int(off[-1]), off.size - 1
    kt, ot = dev(inputs.keys(n, "u32", "uniform", seed=6)), dev(off, np.int64)
    ko = torch.empty_like(kt)
    tmp = ns.scratch(ns.KIND_SEGMENTED, n, nseg)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):           # warm up (lazy module loading) outside the capture
        assert ns.nsort_segmented(kt, ko, None, None, ot, nseg, n, 0, tmp, tmp.numel(), s) == ns.OK
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rc = ns.nsort_segmented(kt, ko, None, None, ot, nseg, n, 0, tmp, tmp.numel(), s)
    assert rc == ns.OK
    for seed, dist in ((7, "uniform"), (8, "dup16"), (9, "reverse")):
        x = inputs.keys(n, "u32", dist, seed=seed)
        kt.copy_(dev(x))
        ko.zero_()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint32),
                                      oracle.sort_segmented(x, off, "u32"))
        assert ns.nsort_device_status(tmp) == ns.OK


def test_batch_of_the_benchmark_shape(ns):
    """2,000 log-uniform segments of 1..65536 keys (the shape of the
    100,000-segment benchmark, at a size the serial oracle sorts in a
    second)."""
    ns.nsort_segmented_set_config()
    off = inputs.segment_offsets(2000, seed=9)
    x = inputs.keys(int(off[-1]), "u32", "uniform", seed=9)
    np.testing.assert_array_equal(run_seg(ns, x, off, "u32"), oracle.sort_segmented(x, off, "u32"))


def oracle_segmented_threaded(x, off, dt):
    """oracle.sort_segmented applied to contiguous groups of whole segments
    on all host cores.  Segments are sorted independently, so sorting each
    group on its own (offsets rebased to the group) is the same computation
    as one call over the batch."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    try:
        threads = max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        threads = max(1, os.cpu_count() or 1)
    n, nseg = int(off[-1]), off.size - 1
    cuts = np.searchsorted(off, np.linspace(0, n, threads + 1)[1:-1])
    bounds = [0] + sorted(set(int(c) for c in cuts if 0 < c < nseg)) + [nseg]
    out = np.empty_like(x)

    def run(i):
        s0, s1 = bounds[i], bounds[i + 1]
        k0, k1 = int(off[s0]), int(off[s1])
        out[k0:k1] = oracle.sort_segmented(x[k0:k1], off[s0:s1 + 1] - k0, dt)

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(run, range(len(bounds) - 1)))
    return out


def test_full_benchmark_batch_against_oracle(ns):
    """The batched benchmark workload at its full size: 100,000 log-uniform
    segments of 1..65536 uniform u32 keys (about 5.9e8 keys), in one
    persistent launch with the default tuning, compared element by element
    with the oracle."""
    ns.nsort_segmented_set_config()
    off = inputs.segment_offsets(100_000, seed=0)
    x = inputs.keys(int(off[-1]), "u32", "uniform", seed=0)
    got = run_seg(ns, x, off, "u32")
    torch.cuda.empty_cache()
    want = oracle_segmented_threaded(x, off, "u32")
    assert np.array_equal(got, want)
