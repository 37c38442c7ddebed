"""GPU checks of the column-sort networks and of the ablation sorts
(include/nsort_ablation.h), through the C ABI.

The networks (bitonic, odd-even, best; widths 4, 8, 16, 32; Sec. 2.3,
Table 1) are run by the device on every 0-1 input of widths 4 to 16 (a
network sorts everything iff it sorts every 0-1 input), and on 0-1 inputs
that fix one half plus random words at width 32.  nsort_runs (the
in-register sort of Table 2 and the block sort, for every family and keys
per thread) is compared bit for bit with the oracle's sort of each run.
"""
import numpy as np
import pytest

import oracle
from paper_2409_03970_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FAMILIES = {"bitonic": 0, "oddeven": 1, "best": 2}
IPTS = [4, 8, 16, 32]


@pytest.fixture(scope="module")
def ns():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03970_gb300 import build, nsort
    build.build()
    nsort.lib()
    return nsort


def dev(bits):
    return torch.from_numpy(np.ascontiguousarray(bits, dtype=np.uint32).view(np.int32)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint32)


def apply_net(ns, groups_2d, family, width):
    g = groups_2d.shape[0]
    x = dev(groups_2d.reshape(-1))
    out = torch.empty_like(x)
    rc = ns.nsort_network_apply(x, out, g, FAMILIES[family], width, 0)
    assert rc == ns.OK, ns.lib().nsort_last_error()
    torch.cuda.synchronize()
    return host(out).reshape(g, width)


def all_zero_one(width):
    x = np.arange(1 << width, dtype=np.uint64)
    return ((x[:, None] >> np.arange(width, dtype=np.uint64)) & 1).astype(np.uint32)


def oracle_runs(bits, run):
    n = bits.size
    offs = np.arange(0, n, run, dtype=np.int64)
    offs = np.append(offs, n) if n else np.zeros(1, np.int64)
    return oracle.sort_segmented(bits, offs, "u32")


@pytest.mark.parametrize("family", list(FAMILIES))
@pytest.mark.parametrize("width", [4, 8, 16])
def test_network_sorts_every_zero_one_input(ns, family, width):
    x = all_zero_one(width)
    out = apply_net(ns, x, family, width)
    # sorted, and the number of ones of each group kept
    assert np.all(out[:, :-1] <= out[:, 1:])
    np.testing.assert_array_equal(out.sum(axis=1), x.sum(axis=1))


@pytest.mark.parametrize("family", list(FAMILIES))
def test_network_32_on_zero_one_halves(ns, family):
    """All 2^16 patterns of one half against fixed patterns of the other."""
    half = all_zero_one(16)
    fixed = [np.zeros(16, np.uint32), np.ones(16, np.uint32),
             np.tile(np.array([0, 1], np.uint32), 8),
             (inputs.counter_u32(11, 0, 0, 16) & 1).astype(np.uint32)]
    rows = []
    for f in fixed:
        rows.append(np.hstack([half, np.broadcast_to(f, half.shape)]))
        rows.append(np.hstack([np.broadcast_to(f, half.shape), half]))
    x = np.ascontiguousarray(np.vstack(rows))
    out = apply_net(ns, x, family, 32)
    assert np.all(out[:, :-1] <= out[:, 1:])
    np.testing.assert_array_equal(out.sum(axis=1), x.sum(axis=1))


@pytest.mark.parametrize("family", list(FAMILIES))
@pytest.mark.parametrize("width", [4, 8, 16, 32])
def test_network_matches_oracle_on_random_words(ns, family, width):
    g = 4099
    bits = inputs.counter_u32(12, width, 0, g * width)
    bits[::7] = bits[::7] & 0xF            # duplicates
    out = apply_net(ns, bits.reshape(g, width), family, width)
    np.testing.assert_array_equal(out.reshape(-1), oracle_runs(bits, width))


def run_cases():
    for family in FAMILIES:
        for ipt in IPTS:
            for lv in range(6):
                yield family, ipt, ipt << lv
            yield family, ipt, 512 * ipt


@pytest.mark.parametrize("family,ipt,run", list(run_cases()))
def test_runs_match_oracle(ns, family, ipt, run):
    """Several tiles and a ragged last run; duplicates and the largest key
    (the value the kernels pad with) among the inputs."""
    n = 3 * 512 * ipt + 777
    bits = inputs.counter_u32(13, ipt, 0, n)
    bits[::5] = bits[::5] % 97
    bits[3::101] = 0xFFFFFFFF
    x = dev(bits)
    out = torch.empty_like(x)
    rc = ns.nsort_runs(x, out, n, FAMILIES[family], ipt, run, 0)
    assert rc == ns.OK, ns.lib().nsort_last_error()
    np.testing.assert_array_equal(host(out), oracle_runs(bits, run))


@pytest.mark.parametrize("ipt", IPTS)
@pytest.mark.parametrize("n", [1, 5, 511, 4097])
def test_runs_short_inputs_in_place_and_misaligned(ns, ipt, n):
    bits = inputs.counter_u32(14, n, 0, n)
    for run in (ipt, 32 * ipt, 512 * ipt):
        buf = dev(np.concatenate([np.zeros(1, np.uint32), bits]))
        x = buf[1:]                                   # 4-byte aligned only
        rc = ns.nsort_runs(x, x, n, ns.NET_BEST, ipt, run, 0)
        assert rc == ns.OK, ns.lib().nsort_last_error()
        np.testing.assert_array_equal(host(x), oracle_runs(bits, run))


def test_block_sort_best16_equals_production_tile_sort(ns):
    """nsort_runs with the best network, 16 keys per thread and whole
    tiles runs the production tile sort's code: its output is the oracle's
    sort of each 8192-key tile, like the first stage of nsort_keys."""
    n = 1 << 20
    bits = inputs.keys(n, "u32", "uniform", seed=15)
    x = dev(bits)
    out = torch.empty_like(x)
    assert ns.nsort_runs(x, out, n, ns.NET_BEST, 16, 8192, 0) == ns.OK
    np.testing.assert_array_equal(host(out), oracle_runs(bits, 8192))


# ---- mergers of Table 3 (nsort_merge_runs) --------------------------------

MERGERS = {"hybrid": 0, "shuffle": 1, "serial": 2}


def merge_cases():
    from paper_2409_03970_gb300 import nsort as N     # run-length rule only, no library call
    for m, code in MERGERS.items():
        for ipt in IPTS:
            for run in N.merge_run_lengths(code, ipt):
                yield m, ipt, run


@pytest.mark.parametrize("method,ipt,run", list(merge_cases()))
def test_merge_runs_match_oracle(ns, method, ipt, run):
    """Input sorted in runs of `run` by the oracle; the output must be the
    oracle's sort of each run of 2 run (several tiles, ragged end)."""
    n = 3 * 512 * ipt + 777
    bits = inputs.counter_u32(16, ipt, 0, n)
    bits[::3] = bits[::3] % 61
    bits[5::97] = 0xFFFFFFFF
    x = dev(oracle_runs(bits, run))
    out = torch.empty_like(x)
    rc = ns.nsort_merge_runs(x, out, n, run, MERGERS[method], ipt, 0)
    assert rc == ns.OK, ns.lib().nsort_last_error()
    np.testing.assert_array_equal(host(out), oracle_runs(bits, 2 * run))


@pytest.mark.parametrize("method", list(MERGERS))
@pytest.mark.parametrize("n", [1, 7, 600, 20000])
def test_merge_runs_in_place_short_inputs(ns, method, n):
    ipt, run = 8, 16
    bits = inputs.counter_u32(17, n, 0, n)
    buf = dev(np.concatenate([np.zeros(1, np.uint32), oracle_runs(bits, run)]))
    x = buf[1:]
    rc = ns.nsort_merge_runs(x, x, n, run, MERGERS[method], ipt, 0)
    assert rc == ns.OK, ns.lib().nsort_last_error()
    np.testing.assert_array_equal(host(x), oracle_runs(bits, 2 * run))
