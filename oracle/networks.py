"""Comparator networks of the paper, as data — TEST INFRASTRUCTURE ONLY.

The paper's column sort (Sec. 2.3) sorts each column of an R x W register
tile with a sorting network, and its mergers (Sec. 2.4) are bitonic merging
networks.  Table 1 counts the comparators of bitonic, odd-even and
"asymmetric" (best-known) sorting networks for n = 4, 8, 16, 32.  This module
holds those networks as lists of comparators and an exhaustive verifier
based on the 0-1 principle (a comparator network sorts every input iff it
sorts every 0-1 input; it merges two sorted runs iff it merges every pair of
sorted 0-1 runs).

A comparator is a pair (lo, hi) with lo < hi: afterwards v[lo] <= v[hi].

Nothing here is imported by the product path; the CUDA column sort carries
its own copy of the 16-input network, checked on the GPU through the public
API (tests/test_gpu_networks.py).
"""
from __future__ import annotations

import itertools

import numpy as np


# --- the 16-input network ------------------------------------------------

def green16():
    """M. W. Green's 16-input sorting network: 60 comparators, depth 10.

    This is the "best" 16-input network the paper adopts for its column sort
    (Sec. 2.3, Table 1 row n=16, "55~60").  The first four layers compare
    every wire with the wire whose index differs in one bit (a 4-cube); six
    more layers finish the sort.
    """
    net = []
    for k in range(4):
        for i in range(16):
            if not i & (1 << k):
                net.append((i, i | (1 << k)))
    net += [(5, 10), (6, 9), (3, 12), (13, 14), (7, 11), (1, 2), (4, 8)]
    net += [(1, 4), (7, 13), (2, 8), (11, 14), (5, 6), (9, 10)]
    net += [(2, 4), (11, 13), (3, 8), (7, 12)]
    net += [(6, 8), (10, 12), (3, 5), (7, 9)]
    net += [(3, 4), (5, 6), (7, 8), (9, 10), (11, 12)]
    net += [(6, 7), (8, 9)]
    return net


# --- symmetric networks of Table 1 ---------------------------------------

def flip_merger(m: int, base: int = 0):
    """Merging network for two sorted runs of length m (m a power of two) on
    wires [base, base+2m).

    Sec. 2.4's bitonic merger written in the "asymmetric" (flip) form: the
    first layer compares wire i with wire 2m-1-i, which merges two ascending
    runs without reversing one of them; after it, each half is cleaned by
    half-cleaner layers at distances m/2, m/4, ..., 1.  m * log2(2m)
    comparators.
    """
    net = [(base + i, base + 2 * m - 1 - i) for i in range(m)]
    d = m // 2
    while d >= 1:
        for i in range(2 * m):
            if not i & d:
                net.append((base + i, base + i + d))
        d //= 2
    return net


def bitonic_sorter(n: int):
    """Bitonic sorting network on n = 2^k wires (Table 1, "Bitonic"), built
    from flip mergers of growing width: (n/2) * k * (k+1) / 2 comparators."""
    net = []
    m = 1
    while m < n:
        for base in range(0, n, 2 * m):
            net += flip_merger(m, base)
        m *= 2
    return net


def _odd_even_merge(wires):
    """Batcher's odd-even merge of the two sorted halves of `wires`: merge
    the even-indexed and the odd-indexed subsequences recursively, then
    compare each odd wire with the next even one."""
    n = len(wires)
    if n == 2:
        return [(wires[0], wires[1])]
    net = _odd_even_merge(wires[0::2]) + _odd_even_merge(wires[1::2])
    for i in range(1, n - 1, 2):
        net.append((wires[i], wires[i + 1]))
    return net


def odd_even_sorter(n: int):
    """Batcher's odd-even merge sorting network on n = 2^k wires (Table 1,
    "Odd-even")."""
    def rec(wires):
        if len(wires) <= 1:
            return []
        h = len(wires) // 2
        return rec(wires[:h]) + rec(wires[h:]) + _odd_even_merge(wires)
    return rec(list(range(n)))


def best32():
    """The fewest-comparator 32-input network Table 1 bounds from above
    (n = 32, "135~185"): Green's network on each half, then Batcher's
    odd-even merge of the two sorted halves, 2 * 60 + 65 = 185
    comparators."""
    upper = [(lo + 16, hi + 16) for lo, hi in green16()]
    return green16() + upper + _odd_even_merge(list(range(32)))


def best_sorter(n: int):
    """Table 1's "Asymmetric Network" column for n = 4, 8, 16, 32: the
    odd-even networks for 4 and 8 (5 and 19 comparators, the fewest
    possible), Green's network for 16, best32() for 32."""
    if n in (4, 8):
        return odd_even_sorter(n)
    return {16: green16, 32: best32}[n]()


# --- analysis -----------------------------------------------------------

def depth(net) -> int:
    """Number of parallel layers when each comparator is placed as early as
    its two wires allow."""
    level = {}
    d = 0
    for lo, hi in net:
        lv = max(level.get(lo, 0), level.get(hi, 0)) + 1
        level[lo] = level[hi] = lv
        d = max(d, lv)
    return d


def apply(net, values):
    """Runs the network on each row of `values` (shape (..., n))."""
    v = np.array(values, copy=True)
    for lo, hi in net:
        a = v[..., lo].copy()
        b = v[..., hi].copy()
        v[..., lo] = np.minimum(a, b)
        v[..., hi] = np.maximum(a, b)
    return v


def zero_one_failures_sorter(net, n: int) -> int:
    """Counts the 0-1 inputs (all 2^n of them) that the network leaves
    unsorted.  Bit-sliced: wire w holds bit w of every input x."""
    x = np.arange(1 << n, dtype=np.uint32)
    wires = [((x >> w) & 1).astype(bool) for w in range(n)]
    for lo, hi in net:
        a, b = wires[lo], wires[hi]
        wires[lo], wires[hi] = a & b, a | b
    bad = np.zeros(1 << n, dtype=bool)
    for w in range(n - 1):
        bad |= wires[w] & ~wires[w + 1]
    return int(bad.sum())


def split_halves(net, n: int):
    """Splits a network on n wires into the longest prefix whose comparators
    each stay inside one half and the rest: (lower-half prefix, upper-half
    prefix shifted to wires [0, n/2), suffix)."""
    h = n // 2
    k = 0
    while k < len(net) and (net[k][1] < h or net[k][0] >= h):
        k += 1
    lower = [c for c in net[:k] if c[1] < h]
    upper = [(lo - h, hi - h) for lo, hi in net[:k] if lo >= h]
    return lower, upper, net[k:]


def zero_one_failures_merger(net, m: int) -> int:
    """Counts the pairs of sorted 0-1 runs (a zeros then ones, b likewise;
    (m+1)^2 pairs) that the network fails to merge into one sorted run."""
    fails = 0
    for za, zb in itertools.product(range(m + 1), repeat=2):
        v = np.array([0] * za + [1] * (m - za) + [0] * zb + [1] * (m - zb))
        out = apply(net, v)
        if np.any(out[:-1] > out[1:]):
            fails += 1
    return fails
