"""CPU-side checks of libnsort: it builds for sm_103a, loads, exports every
function include/nsort.h declares, and its host logic (plans, scratch sizes,
argument validation) behaves — all without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_2409_03970_gb300 import build as nbuild
from paper_2409_03970_gb300 import nsort

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    nbuild.build()
    return nsort.lib()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(nsort_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("nsort_keys", "nsort_pairs", "nsort_temp_bytes", "nsort_plan",
                 "nsort_status_string", "nsort_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(nsort.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(raw, n)]
    assert missing == []


def test_plan_pass_counts(lib):
    prev = nsort.nsort_testing_set_four_way_min(nsort.FOUR_WAY_NEVER)
    try:
        passes, st, mt = nsort.nsort_plan(nsort.KIND_KEYS, 1 << 28)
        assert st & (st - 1) == 0 and mt > 0          # run lengths double from a power of two
        # one tile sort + ceil(log2(2^28 / tile)) merge passes of one level
        levels = 28 - st.bit_length() + 1
        assert passes == 1 + levels
        assert nsort.nsort_plan(nsort.KIND_KEYS, 1)[0] == 1
        assert nsort.nsort_plan(nsort.KIND_KEYS, st)[0] == 1
        assert nsort.nsort_plan(nsort.KIND_KEYS, st + 1)[0] == 2
        assert nsort.nsort_plan(nsort.KIND_KEYS, 3 * st)[0] == 3
        # four-way passes merge two levels each, after a one-level pass when
        # the number of levels is odd
        nsort.nsort_testing_set_four_way_min(0)
        assert nsort.nsort_plan(nsort.KIND_KEYS, 1 << 28)[0] == 1 + levels % 2 + levels // 2
        assert nsort.nsort_plan(nsort.KIND_KEYS, st + 1)[0] == 2      # one level
        assert nsort.nsort_plan(nsort.KIND_KEYS, 3 * st)[0] == 2      # two levels: one pass
        assert nsort.nsort_plan(nsort.KIND_KEYS, 5 * st)[0] == 3      # three: two passes
        # pairs and 64-bit keys merge one level a pass
        p2, st2, _ = nsort.nsort_plan(nsort.KIND_PAIRS, 1 << 27)
        assert p2 == 1 + (27 - st2.bit_length() + 1)
        p3, st3, _ = nsort.nsort_plan(nsort.KIND_KEYS, 1 << 27, nsort.U64)
        assert p3 == 1 + (27 - st3.bit_length() + 1)
    finally:
        nsort.nsort_testing_set_four_way_min(prev)


def test_temp_bytes(lib):
    _, st, mt = nsort.nsort_plan(nsort.KIND_KEYS, 1 << 20)
    assert nsort.nsort_temp_bytes(nsort.KIND_KEYS, st) == 0          # one tile: no scratch
    n = 1 << 20
    tb = nsort.nsort_temp_bytes(nsort.KIND_KEYS, n)
    # one ping-pong copy, the status word, one splitter per merge tile of the
    # pass with the most tiles (tiles never span two run pairs) and every
    # 64th key of a pass's output
    assert 4 * n <= tb <= 4 * n + 8 * (n // mt + n // (2 * st) + 3) + 4 * (n // 64 + 2) + 1280
    tp = nsort.nsort_temp_bytes(nsort.KIND_PAIRS, n)
    _, pst, pmt = nsort.nsort_plan(nsort.KIND_PAIRS, n)
    assert 8 * n <= tp <= 8 * n + 8 * (n // pmt + n // (2 * pst) + 3) + 4 * (n // 64 + 2) + 1280
    assert nsort.nsort_temp_bytes(99, n) == 0


def test_temp_bytes_four_way(lib):
    # four-way passes add the level-one sample records (8 bytes per 64 keys)
    # and the tile boundaries (4 x 8 bytes per tile of about 3968 keys, plus
    # one record per group of four runs: at most one per 3641 keys)
    n = 1 << 24
    prev = nsort.nsort_testing_set_four_way_min(nsort.FOUR_WAY_NEVER)
    try:
        two = nsort.nsort_temp_bytes(nsort.KIND_KEYS, n)
        nsort.nsort_testing_set_four_way_min(0)
        four = nsort.nsort_temp_bytes(nsort.KIND_KEYS, n)
        # pairs and 64-bit keys are unaffected
        pairs = nsort.nsort_temp_bytes(nsort.KIND_PAIRS, n)
        wide = nsort.nsort_temp_bytes(nsort.KIND_KEYS, n, 0, nsort.U64)
        nsort.nsort_testing_set_four_way_min(nsort.FOUR_WAY_NEVER)
        assert pairs == nsort.nsort_temp_bytes(nsort.KIND_PAIRS, n)
        assert wide == nsort.nsort_temp_bytes(nsort.KIND_KEYS, n, 0, nsort.U64)
    finally:
        nsort.nsort_testing_set_four_way_min(prev)
    extra = four - two
    assert 8 * (n // 64) <= extra <= 8 * (n // 64 + 2) + 32 * (n // 3600 + 2) + 512


def test_argument_validation_needs_no_gpu(lib):
    big = 1 << 20
    # bad dtype, NULL pointers, misaligned pointers, too little scratch, too many keys:
    # all rejected on the host before any CUDA call
    assert nsort.nsort_keys(0x1000, 0x1000, 10, 7, 0, 0, 0) == nsort.EINVAL
    assert nsort.nsort_keys(0, 0x1000, 10, nsort.U32, 0, 0, 0) == nsort.EINVAL
    assert nsort.nsort_keys(0x1002, 0x1000, 10, nsort.U32, 0, 0, 0) == nsort.EINVAL
    assert nsort.nsort_keys(0x1000, 0x2000, big, nsort.U32, 0, 0, 0) == nsort.ENOMEM
    assert nsort.nsort_keys(0x1000, 0x2000, big, nsort.U32, 0x100000, 64, 0) == nsort.ENOMEM
    assert nsort.nsort_keys(0x1000, 0x2000, 1 << 41, nsort.U32, 0, 0, 0) == nsort.EINVAL
    assert nsort.nsort_keys(0, 0, 0, nsort.U32, 0, 0, 0) == nsort.OK        # n = 0: no-op
    assert nsort.nsort_pairs(0x1000, 0, 0x2000, 0x3000, 10, nsort.U32, 0, 0, 0) == nsort.EINVAL
    assert nsort.nsort_pairs(0x1000, 0x4000, 0x2000, 0x3000, big, nsort.F32, 0, 0, 0) == nsort.ENOMEM
    for s in range(7):
        assert lib.nsort_status_string(s)


def test_binding_rejects_host_tensors(lib):
    """The binding passes device addresses only: a CPU tensor (whose host
    address a kernel would be handed) is refused before the call."""
    torch = pytest.importorskip("torch")
    x = torch.zeros(16, dtype=torch.int32)
    with pytest.raises(ValueError):
        nsort.nsort_keys(x, x, 16, nsort.I32, None, 0, 0)
    with pytest.raises(ValueError):
        nsort.nsort_pairs(0x1000, x, 0x2000, 0x3000, 16, nsort.I32, None, 0, 0)


# ---- column-sort networks of the ablation (include/nsort_ablation.h) ----

FAMILIES = {"bitonic": nsort.NET_BITONIC, "oddeven": nsort.NET_ODDEVEN, "best": nsort.NET_BEST}


def test_library_networks_have_table1_sizes(lib, golden):
    for n, bit, oe, amin, amax in golden("table1_comparators.txt"):
        n = int(n)
        assert len(nsort.nsort_network(nsort.NET_BITONIC, n)) == int(bit)
        assert len(nsort.nsort_network(nsort.NET_ODDEVEN, n)) == int(oe)
        assert int(amin) <= len(nsort.nsort_network(nsort.NET_BEST, n)) <= int(amax)
    assert len(nsort.nsort_network(nsort.NET_BEST, 16)) == 60
    assert len(nsort.nsort_network(nsort.NET_BEST, 32)) == 185


@pytest.mark.parametrize("family", list(FAMILIES))
def test_library_networks_sort_by_zero_one_principle(lib, family):
    """The lists the device column sorts are generated from, checked on all
    0-1 inputs (widths 4-16) and by composition (width 32)."""
    from oracle import networks as N
    f = FAMILIES[family]
    for w in (4, 8, 16):
        net = nsort.nsort_network(f, w)
        assert all(0 <= lo < hi < w for lo, hi in net)
        assert N.zero_one_failures_sorter(net, w) == 0
    lower, upper, merge = N.split_halves(nsort.nsort_network(f, 32), 32)
    assert N.zero_one_failures_sorter(lower, 16) == 0
    assert N.zero_one_failures_sorter(upper, 16) == 0
    assert N.zero_one_failures_merger(merge, 16) == 0


def test_library_networks_are_the_named_networks(lib):
    """Same comparators as the oracle's independently written generators;
    the best 16-input network is Green's, comparator for comparator."""
    from oracle import networks as N
    for w in (4, 8, 16, 32):
        assert set(nsort.nsort_network(nsort.NET_BITONIC, w)) == set(N.bitonic_sorter(w))
        assert set(nsort.nsort_network(nsort.NET_ODDEVEN, w)) == set(N.odd_even_sorter(w))
        assert set(nsort.nsort_network(nsort.NET_BEST, w)) == set(N.best_sorter(w))
    assert nsort.nsort_network(nsort.NET_BEST, 16) == N.green16()
    assert N.depth(nsort.nsort_network(nsort.NET_BEST, 16)) == 10


def test_ablation_argument_validation_needs_no_gpu(lib):
    assert nsort.nsort_network(3, 16) is None
    assert nsort.nsort_network(nsort.NET_BEST, 12) is None
    assert nsort.nsort_network_apply(0x1000, 0x1000, 4, nsort.NET_BEST, 12, 0) == nsort.EINVAL
    assert nsort.nsort_network_apply(0x1000, 0x1000, 4, 7, 16, 0) == nsort.EINVAL
    assert nsort.nsort_network_apply(0, 0, 0, nsort.NET_BEST, 16, 0) == nsort.OK
    assert nsort.nsort_network_apply(0, 0x1000, 4, nsort.NET_BEST, 16, 0) == nsort.EINVAL
    # run must be ipt * 2^L (L <= 5) or 512 * ipt
    assert nsort.nsort_runs(0x1000, 0x1000, 100, nsort.NET_BEST, 16, 24, 0) == nsort.EINVAL
    assert nsort.nsort_runs(0x1000, 0x1000, 100, nsort.NET_BEST, 16, 1024, 0) == nsort.EINVAL
    assert nsort.nsort_runs(0x1000, 0x1000, 100, nsort.NET_BEST, 12, 12, 0) == nsort.EINVAL
    assert nsort.nsort_runs(0x1000, 0x1000, 1 << 41, nsort.NET_BEST, 16, 16, 0) == nsort.EINVAL
    assert nsort.nsort_runs(0, 0, 100, nsort.NET_BEST, 16, 16, 0) == nsort.EINVAL
    assert nsort.nsort_runs(0, 0, 0, nsort.NET_BEST, 16, 8192, 0) == nsort.OK


def test_merge_runs_argument_validation_needs_no_gpu(lib):
    H, S, R = nsort.MERGE_HYBRID, nsort.MERGE_SHUFFLE, nsort.MERGE_SERIAL
    bad = [(100, 8, H, 16), (100, 512, H, 16), (100, 24, S, 16), (100, 512, S, 16),
           (100, 4, R, 16), (100, 8192, R, 16), (100, 16, 3, 16), (100, 16, H, 12),
           (100, 0, S, 16), (1 << 41, 16, H, 16)]
    for n, run, m, ipt in bad:
        assert nsort.nsort_merge_runs(0x1000, 0x1000, n, run, m, ipt, 0) == nsort.EINVAL, (run, m)
    assert nsort.nsort_merge_runs(0, 0, 0, 16, H, 16, 0) == nsort.OK
    assert nsort.nsort_merge_runs(0, 0x1000, 10, 16, H, 16, 0) == nsort.EINVAL
    assert nsort.merge_run_lengths(H, 16) == [16, 32, 64, 128, 256]
    assert nsort.merge_run_lengths(S, 4) == [1, 2, 4, 8, 16, 32, 64]
    assert nsort.merge_run_lengths(R, 4)[0] == 2 and nsort.merge_run_lengths(R, 4)[-1] == 1024


def test_64bit_keys_plan_scratch_and_validation(lib):
    p, st, mt = nsort.nsort_plan(nsort.KIND_KEYS, 1 << 27, nsort.U64)
    assert (st, mt) == (4096, 1920) and p == 1 + (27 - 12)
    assert nsort.nsort_plan(nsort.KIND_KEYS, 4096, nsort.F64)[0] == 1
    assert nsort.nsort_plan(nsort.KIND_KEYS, 4097, nsort.I64)[0] == 2
    n = 1 << 20
    t64 = nsort.nsort_temp_bytes(nsort.KIND_KEYS, n, 0, nsort.U64)
    assert 8 * n <= t64 <= 8 * n + 8 * (n // 1920 + n // 8192 + 3) + 8 * (n // 64 + 2) + 1280
    assert nsort.nsort_temp_bytes(nsort.KIND_KEYS, 4096, 0, nsort.U64) == 0    # one tile
    # 64-bit keys: nsort_keys only, 8-byte aligned pointers
    assert nsort.nsort_keys(0x1004, 0x2000, 1 << 20, nsort.U64, 0x100000, t64, 0) == nsort.EINVAL
    assert nsort.nsort_keys(0x1000, 0x2000, 1 << 20, nsort.F64, 0x100000, t64 - 8, 0) == nsort.ENOMEM
    assert nsort.nsort_pairs(0x1000, 0x3000, 0x2000, 0x4000, 10, nsort.U64, 0, 0, 0) == nsort.EINVAL
    assert nsort.nsort_segmented(0x1000, 0x2000, 0, 0, 0x3000, 1, 10, nsort.I64, 0x4000, 1 << 20,
                                 0) == nsort.EINVAL
    assert nsort.nsort_keys(0x1000, 0x2000, 10, 6, 0, 0, 0) == nsort.EINVAL
    with pytest.raises(nsort.NsortError):
        nsort.nsort_plan(nsort.KIND_PAIRS, 100, nsort.U64)
