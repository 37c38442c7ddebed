"""Pins of the comparator networks of Sec. 2.3 / 2.4 (oracle/networks.py).

Counts against the paper's Table 1 and Table 3 merge lengths (golden
fixtures), correctness by the 0-1 principle, exhaustively.
"""
import numpy as np
import pytest

from oracle import networks as N
from paper_2409_03970_gb300 import inputs


def test_table1_counts(golden):
    for n, bit, oe, amin, amax in golden("table1_comparators.txt"):
        n = int(n)
        assert len(N.bitonic_sorter(n)) == int(bit)
        assert len(N.odd_even_sorter(n)) == int(oe)
        if n == 16:
            g = N.green16()
            assert int(amin) <= len(g) <= int(amax)
            assert len(g) == 60


def test_green16_depth_and_shape():
    g = N.green16()
    assert N.depth(g) == 10
    assert all(0 <= lo < hi < 16 for lo, hi in g)


def test_green16_zero_one_exhaustive():
    assert N.zero_one_failures_sorter(N.green16(), 16) == 0


@pytest.mark.parametrize("n", [2, 4, 8, 16])
def test_symmetric_sorters_zero_one_exhaustive(n):
    assert N.zero_one_failures_sorter(N.bitonic_sorter(n), n) == 0
    assert N.zero_one_failures_sorter(N.odd_even_sorter(n), n) == 0


def test_flip_mergers(golden):
    for m, count in golden("table3_merge_lengths.txt"):
        m = int(m)
        net = N.flip_merger(m)
        assert len(net) == int(count)
        assert N.zero_one_failures_merger(net, m) == 0


def test_networks_sort_random_words():
    x = inputs.counter_u32(4, 0, 0, 16 * 4096).reshape(4096, 16)
    np.testing.assert_array_equal(N.apply(N.green16(), x), np.sort(x, axis=1))
    y = inputs.counter_u32(5, 0, 0, 32 * 512).reshape(512, 32)
    np.testing.assert_array_equal(N.apply(N.bitonic_sorter(32), y), np.sort(y, axis=1))
    np.testing.assert_array_equal(N.apply(N.odd_even_sorter(32), y), np.sort(y, axis=1))


def test_verifier_catches_a_dropped_comparator():
    g = N.green16()
    for drop in (0, 31, 45, 59):
        broken = g[:drop] + g[drop + 1:]
        assert N.zero_one_failures_sorter(broken, 16) > 0
    m = N.flip_merger(16)
    assert N.zero_one_failures_merger(m[1:], 16) > 0


def test_best_sorters_within_table1(golden):
    for n, _bit, _oe, amin, amax in golden("table1_comparators.txt"):
        n = int(n)
        assert int(amin) <= len(N.best_sorter(n)) <= int(amax)
    assert len(N.best32()) == 185          # the upper bound of Table 1, n = 32


@pytest.mark.parametrize("make", [lambda: N.bitonic_sorter(32), lambda: N.odd_even_sorter(32),
                                  N.best32], ids=["bitonic", "oddeven", "best"])
def test_32_input_sorters_by_composition(make):
    """A network that first sorts each half and then merges any two sorted
    halves sorts everything (0-1 principle, applied to the two phases):
    each half's prefix is checked on all 2^16 0-1 inputs, the rest on all
    17 x 17 pairs of sorted 0-1 halves."""
    lower, upper, merge = N.split_halves(make(), 32)
    assert N.zero_one_failures_sorter(lower, 16) == 0
    assert N.zero_one_failures_sorter(upper, 16) == 0
    assert N.zero_one_failures_merger(merge, 16) == 0


def test_composition_check_catches_a_dropped_merge_comparator():
    lower, upper, merge = N.split_halves(N.best32(), 32)
    for drop in (0, 20, 64):
        assert N.zero_one_failures_merger(merge[:drop] + merge[drop + 1:], 16) > 0
