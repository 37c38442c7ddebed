"""Pins of the CPU oracle against things other than itself.

Each function of oracle.c is checked against an independent source: the
IEEE 754 totalOrder table (tests/golden), numpy's own integer and float
comparisons, numpy's library sorts in the cases where they compute the same
thing, a textbook insertion sort on every small input, invariants and closed
forms.  test_planted_mistakes compiles deliberately broken copies of
oracle.c and checks that these pins catch each one.
"""
import itertools
import os
import re

import numpy as np
import pytest

import oracle
from paper_2409_03970_gb300 import inputs


# --- independent references ------------------------------------------------

def insertion_sort_pairs(items, less):
    """Textbook stable insertion sort: an element moves left only past
    strictly greater elements."""
    out = []
    for it in items:
        j = len(out)
        while j > 0 and less(it, out[j - 1]):
            j -= 1
        out.insert(j, it)
    return out


def f32_less_nonnan(a_bits, b_bits):
    """IEEE order of two non-NaN binary32 values by Python float comparison,
    with -0 below +0 (totalOrder)."""
    a = np.uint32(a_bits).view(np.float32)
    b = np.uint32(b_bits).view(np.float32)
    if a == b:
        return bool(np.signbit(a)) and not bool(np.signbit(b))
    return bool(a < b)


LESS = {
    "u32": lambda a, b: int(a) < int(b),
    "i32": lambda a, b: int(np.uint32(a).view(np.int32)) < int(np.uint32(b).view(np.int32)),
    "f32": f32_less_nonnan,
}

ALPHABET = {  # four bit patterns per dtype, used for brute force
    "u32": [0x00000000, 0x00000007, 0x80000000, 0xFFFFFFFF],
    "i32": [0x80000000, 0xFFFFFFFF, 0x00000000, 0x7FFFFFFF],       # -2^31, -1, 0, 2^31-1
    "f32": [0xBFC00000, 0x80000000, 0x00000000, 0x40000000],       # -1.5, -0, +0, 2
}


# --- key map -------------------------------------------------------------

def test_key_u32_is_identity():
    x = inputs.counter_u32(1, 0, 0, 4096)
    np.testing.assert_array_equal(oracle.key(x, "u32"), x)


def test_key_i32_matches_signed_order():
    x = np.concatenate([inputs.counter_u32(2, 0, 0, 2000),
                        np.array([0, 1, 0x7FFFFFFF, 0x80000000, 0x80000001, 0xFFFFFFFF], np.uint32)])
    k = oracle.key(x, "i32")
    s = x.view(np.int32).astype(np.int64)
    a, b = np.meshgrid(np.arange(x.size), np.arange(x.size), indexing="ij")
    np.testing.assert_array_equal(k[a] < k[b], s[a] < s[b])


def test_key_f32_golden_total_order(golden):
    rows = golden("f32_total_order.txt")
    bits = np.array([int(r[0], 16) for r in rows], dtype=np.uint32)
    k = oracle.key(bits, "f32").astype(np.int64)
    assert np.all(np.diff(k) > 0), "IEEE totalOrder table is not strictly increasing"


def test_key_f32_matches_float_compare_without_nan():
    x = inputs.counter_u32(3, 0, 0, 3000)
    f = x.view(np.float32)
    x = x[~np.isnan(f)]
    f = x.view(np.float32).astype(np.float64)
    k = oracle.key(x, "f32").astype(np.int64)
    a, b = np.meshgrid(np.arange(x.size), np.arange(x.size), indexing="ij")
    ne = f[a] != f[b]
    np.testing.assert_array_equal((k[a] < k[b])[ne], (f[a] < f[b])[ne])


@pytest.mark.slow
def test_key_f32_exhaustive_total_order_and_bijection():
    """All 2^32 patterns, enumerated in IEEE totalOrder (negative patterns
    from 0xFFFFFFFF down to 0x80000000, then 0x00000000 up to 0x7FFFFFFF):
    the key must be strictly increasing along the enumeration, which also
    makes it a bijection.  The int32 key is checked the same way along the
    signed order (0x80000000 up to 0xFFFFFFFF, then 0 up to 0x7FFFFFFF)."""
    step = 1 << 27

    def walk(dtype, segments):
        last = None
        for start, stop, inc in segments:            # each: arange(start, stop, inc)
            for lo in range(start, stop, inc * step):
                hi = lo + inc * step
                hi = min(hi, stop) if inc > 0 else max(hi, stop)
                b = np.arange(lo, hi, inc, dtype=np.int64).astype(np.uint32)
                k = oracle.key(b, dtype)
                assert np.all(k[1:] > k[:-1]), (dtype, hex(lo))
                if last is not None:
                    assert k[0] > last, (dtype, hex(lo))
                last = k[-1]

    walk("f32", [(0xFFFFFFFF, 0x7FFFFFFF, -1), (0, 0x80000000, 1)])
    walk("i32", [(0x80000000, 0x100000000, 1), (0, 0x80000000, 1)])


# --- brute force on tiny inputs ----------------------------------------

@pytest.mark.parametrize("dtype", ["u32", "i32", "f32"])
def test_all_permutations_against_insertion_sort(dtype):
    base = [0x3F800000, 0xBF800000, 0x00000000, 0x80000000, 0x40490FDB, 0xC0490FDB, 0x00000001]
    if dtype != "f32":
        base = [0, 1, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFF, 12345, 0xDEADBEEF]
    for n in range(0, 8):
        for perm in itertools.permutations(base[:n]):
            x = np.array(perm, dtype=np.uint32)
            got = oracle.sort_keys(x, dtype)
            want = insertion_sort_pairs(list(perm), LESS[dtype])
            assert got.tolist() == want, (dtype, perm)


@pytest.mark.parametrize("dtype", ["u32", "i32", "f32"])
def test_all_words_pairs_stable_against_insertion_sort(dtype):
    alpha = ALPHABET[dtype]
    less = LESS[dtype]
    for n in range(0, 8):
        for word in itertools.product(range(4), repeat=n):
            k = np.array([alpha[w] for w in word], dtype=np.uint32)
            v = np.arange(n, dtype=np.uint32)
            ko, vo = oracle.sort_pairs(k, v, dtype)
            want = insertion_sort_pairs(list(zip(k.tolist(), v.tolist())),
                                        lambda a, b: less(a[0], b[0]))
            assert list(zip(ko.tolist(), vo.tolist())) == want, (dtype, word)


# --- library routines that compute the same thing ------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 17, 1000, 4097, 65536 + 3])
def test_matches_numpy_sorts(n):
    x = inputs.keys(n, "u32", "uniform", seed=n)
    np.testing.assert_array_equal(oracle.sort_keys(x, "u32"), np.sort(x))
    s = x.view(np.int32)
    np.testing.assert_array_equal(oracle.sort_keys(x, "i32").view(np.int32), np.sort(s))
    # float32 without NaN and without -0: numpy's float order is totalOrder there
    f = inputs.keys(n, "f32", "uniform", seed=n)
    f = np.where(f == np.uint32(0x80000000), np.uint32(0), f)
    np.testing.assert_array_equal(oracle.sort_keys(f, "f32").view(np.float32),
                                  np.sort(f.view(np.float32)))
    # stable pairs with heavy duplicates: numpy's stable argsort is the definition
    d = inputs.keys(n, "i32", "dup16", seed=n)
    v = inputs.counter_u32(n, 5, 0, n)
    perm = np.argsort(d.view(np.int32), kind="stable")
    ko, vo = oracle.sort_pairs(d, v, "i32")
    np.testing.assert_array_equal(ko, d[perm])
    np.testing.assert_array_equal(vo, v[perm])


# --- invariants and closed forms ------------------------------------------

def _sorted_in_key_order(bits, dtype):
    if dtype == "u32":
        return np.all(bits[:-1] <= bits[1:])
    if dtype == "i32":
        s = bits.view(np.int32)
        return np.all(s[:-1] <= s[1:])
    with np.errstate(invalid="ignore"):
        f = bits.view(np.float32).astype(np.float64)
    a, b = f[:-1], f[1:]
    nan_a, nan_b = np.isnan(a), np.isnan(b)
    sa, sb = np.signbit(a), np.signbit(b)
    ok = np.where(nan_a | nan_b,
                  # -NaN first, +NaN last
                  (nan_a & sa) | (nan_b & ~sb),
                  (a < b) | ((a == b) & ~(~sa & sb)))
    return np.all(ok)


@pytest.mark.parametrize("dtype", ["u32", "i32", "f32"])
@pytest.mark.parametrize("dist", list(inputs.DISTRIBUTIONS))
def test_invariants_all_distributions(dtype, dist):
    n = 20000 + 7
    x = inputs.keys(n, dtype, dist, seed=11)
    y = oracle.sort_keys(x, dtype)
    assert _sorted_in_key_order(y, dtype)
    np.testing.assert_array_equal(np.sort(y), np.sort(x))      # same multiset of patterns


@pytest.mark.parametrize("threads", [1, 2, 3, 8, 16])
@pytest.mark.parametrize("dist", ["uniform", "dup16", "reverse"])
def test_multithreaded_oracle_equals_the_serial_one(threads, dist):
    """The CPU baseline's multi-threaded form (chunk sorts, pairwise merges)
    returns exactly the serial oracle's result, including ragged chunks and
    more threads than keys."""
    for n in (0, 1, 5, 17, 20_011):
        for dt in ("u32", "i32", "f32"):
            x = inputs.keys(n, dt, dist, seed=n + threads)
            np.testing.assert_array_equal(oracle.sort_keys_par(x, dt, threads),
                                          oracle.sort_keys(x, dt))


def test_multithreaded_oracle_rejects_bad_arguments():
    x = inputs.keys(10, "u32", "uniform", seed=1)
    for dt, threads in (("u32", 0), ("u32", 257)):
        with pytest.raises(RuntimeError):
            oracle.sort_keys_par(x, dt, threads)
    with pytest.raises(ValueError):
        oracle.sort_keys_par(x, "u64", 2)


def test_pairs_with_ieee_specials_invariants():
    n = 50000
    k, v = inputs.normal_pairs(n, seed=3, special_per_mille=20)
    ko, vo = oracle.sort_pairs(k, v, "f32")
    assert _sorted_in_key_order(ko, "f32")
    np.testing.assert_array_equal(ko, k[vo])                    # payload travels with its key
    np.testing.assert_array_equal(np.sort(vo), v)               # permutation
    eq = ko[:-1] == ko[1:]
    assert np.all(vo[:-1][eq] < vo[1:][eq])                     # stable (payload = index)
    # every NaN pattern sorts to an end: -NaN first, +NaN last
    f = ko.view(np.float32)
    nn = np.isnan(f)
    neg = np.signbit(f)
    first_non_negnan = np.argmax(~(nn & neg))
    assert not np.any((nn & neg)[first_non_negnan:])


def test_closed_forms():
    n = 4096
    s = inputs.keys(n, "u32", "sorted", seed=5)
    np.testing.assert_array_equal(oracle.sort_keys(s, "u32"), s)          # sorted -> identity
    r = inputs.keys(n, "u32", "reverse", seed=5)
    assert len(np.unique(r)) == n
    np.testing.assert_array_equal(oracle.sort_keys(r, "u32"), r[::-1])    # reverse -> reversal
    d = inputs.keys(n, "i32", "dup16", seed=5)
    y = oracle.sort_keys(d, "i32")
    vals, counts = np.unique(d.view(np.int32), return_counts=True)
    np.testing.assert_array_equal(y.view(np.int32), np.repeat(vals, counts))
    assert oracle.sort_keys(np.zeros(0, np.uint32), "u32").size == 0


def test_segmented_matches_per_segment_and_rejects_bad_offsets():
    off = np.array([0, 0, 1, 5, 5, 300, 1000], dtype=np.int64)
    x = inputs.keys(int(off[-1]), "f32", "uniform", seed=9)
    v = np.arange(x.size, dtype=np.uint32)
    ko, vo = oracle.sort_segmented(x, off, "f32", vals=v)
    for a, b in zip(off[:-1], off[1:]):
        kk, vv = oracle.sort_pairs(x[a:b], v[a:b], "f32")
        np.testing.assert_array_equal(ko[a:b], kk)
        np.testing.assert_array_equal(vo[a:b], vv)
        assert np.all((vo[a:b] >= a) & (vo[a:b] < b))                    # segments never mix
    with pytest.raises(RuntimeError):
        oracle.sort_segmented(x, np.array([0, 600, 500, 1000], np.int64), "f32")


# --- 64-bit keys -------------------------------------------------------------

def f64_less_nonnan(a_bits, b_bits):
    """IEEE order of two non-NaN binary64 values by numpy comparison, with
    -0 below +0 (totalOrder)."""
    a = np.uint64(a_bits).view(np.float64)
    b = np.uint64(b_bits).view(np.float64)
    if a == b:
        return bool(np.signbit(a)) and not bool(np.signbit(b))
    return bool(a < b)


LESS64 = {
    "u64": lambda a, b: int(a) < int(b),
    "i64": lambda a, b: int(np.uint64(a).view(np.int64)) < int(np.uint64(b).view(np.int64)),
    "f64": f64_less_nonnan,
}

ALPHABET64 = {
    "u64": [0x0, 0x7, 0x8000000000000000, 0xFFFFFFFFFFFFFFFF],
    "i64": [0x8000000000000000, 0xFFFFFFFFFFFFFFFF, 0x0, 0x7FFFFFFFFFFFFFFF],   # min, -1, 0, max
    "f64": [0xBFF8000000000000, 0x8000000000000000, 0x0, 0x4000000000000000],   # -1.5, -0, +0, 2
}


def f64_edge_patterns():
    """Every sign x exponent edge x mantissa edge combination of binary64."""
    exps = [0, 1, 2, 1022, 1023, 1024, 2045, 2046, 2047]
    mants = [0, 1, 2, (1 << 51) - 1, 1 << 51, (1 << 51) + 1, (1 << 52) - 1]
    out = [(sg << 63) | (e << 52) | m for sg in (0, 1) for e in exps for m in mants]
    return np.array(out, dtype=np.uint64)


def test_key64_u64_identity_and_i64_signed_order():
    x = inputs.keys64(4096, "u64", "specials", seed=3)
    np.testing.assert_array_equal(oracle.key64(x, "u64"), x)
    edges = np.array([-(1 << 63), -2, -1, 0, 1, (1 << 63) - 1], dtype=np.int64)
    v = np.concatenate([x.view(np.int64), edges])
    k = oracle.key64(v.view(np.uint64), "i64")
    order_k = np.argsort(k, kind="stable")
    order_v = np.argsort(v, kind="stable")
    np.testing.assert_array_equal(v[order_k], v[order_v])


def test_key64_f64_golden_total_order(golden):
    rows = golden("f64_total_order.txt")
    bits = np.array([int(r[0], 16) for r in rows], dtype=np.uint64)
    k = oracle.key64(bits, "f64")
    assert np.all(k[1:] > k[:-1])


def test_key64_f64_matches_float_compare_without_nan():
    pats = np.concatenate([f64_edge_patterns(), inputs.keys64(2000, "f64", "uniform", seed=4)])
    f = pats.view(np.float64)
    pats = pats[~np.isnan(f)]
    k = oracle.key64(pats, "f64")
    # sort by (value, sign) with numpy, then the keys must be strictly increasing
    f = pats.view(np.float64)
    order = np.lexsort((~np.signbit(f), f))
    ks = k[order]
    uniq = np.unique(pats).size == pats.size
    assert uniq
    assert np.all(ks[1:] > ks[:-1])


def test_key64_f64_nans_beyond_the_infinities():
    pats = f64_edge_patterns()
    f = pats.view(np.float64)
    k = oracle.key64(pats, "f64")
    kninf = oracle.key64(np.array([0xFFF0000000000000], np.uint64), "f64")[0]
    kpinf = oracle.key64(np.array([0x7FF0000000000000], np.uint64), "f64")[0]
    nan = np.isnan(f)
    neg = np.signbit(f)
    assert np.all(k[nan & neg] < kninf)
    assert np.all(k[nan & ~neg] > kpinf)


@pytest.mark.parametrize("dtype", list(ALPHABET64))
def test_sort64_all_words_against_insertion_sort(dtype):
    less = LESS64[dtype]
    for n in range(0, 7):
        for word in itertools.product(ALPHABET64[dtype], repeat=n):
            bits = np.array(word, dtype=np.uint64)
            want = insertion_sort_pairs(list(word), less)
            np.testing.assert_array_equal(oracle.sort_keys64(bits, dtype),
                                          np.array(want, dtype=np.uint64))


@pytest.mark.parametrize("n", [1, 2, 3, 17, 1000, 65537])
def test_sort64_matches_numpy(n):
    x = inputs.keys64(n, "u64", "uniform", seed=n)
    np.testing.assert_array_equal(oracle.sort_keys64(x, "u64"), np.sort(x))
    np.testing.assert_array_equal(oracle.sort_keys64(x, "i64").view(np.int64),
                                  np.sort(x.view(np.int64)))
    f = inputs.keys64(n, "f64", "uniform", seed=n)      # no NaN, no -0
    np.testing.assert_array_equal(oracle.sort_keys64(f, "f64").view(np.float64),
                                  np.sort(f.view(np.float64)))


@pytest.mark.parametrize("dtype", ["u64", "i64", "f64"])
@pytest.mark.parametrize("dist", ["uniform", "sorted", "reverse", "dup16", "specials"])
def test_sort64_invariants_and_closed_forms(dtype, dist):
    x = inputs.keys64(20000, dtype, dist, seed=5)
    out = oracle.sort_keys64(x, dtype)
    k = oracle.key64(out, dtype)
    assert np.all(k[1:] >= k[:-1])                                    # non-decreasing
    np.testing.assert_array_equal(np.sort(out), np.sort(x))           # a permutation
    if dist == "sorted":
        np.testing.assert_array_equal(out, x)                         # identity
    if dist == "reverse" and np.unique(x).size == x.size:
        np.testing.assert_array_equal(out, x[::-1])                   # reversal


# --- planted mistakes -------------------------------------------------------

MUTATIONS = {
    # a wrong tie rule: takes from the right run on equal keys (unstable)
    "tie_rule": (r"if \(orc_key\(src_k\[j\], dtype\) < orc_key\(src_k\[i\], dtype\)\)",
                 "if (orc_key(src_k[j], dtype) <= orc_key(src_k[i], dtype))"),
    # float map without the complement of negatives
    "f32_negatives": (r"return ~bits;", "return bits;"),
    # signed map without the sign flip
    "i32_sign": (r"return bits \^ 0x80000000u;\n    if \(dtype == ORC_F32\)",
                 "return bits;\n    if (dtype == ORC_F32)"),
    # drops the left run's tail
    "lost_tail": (r"while \(i < mid\) \{", "while (0) {"),
    # off-by-one in the run width
    "run_width": (r"uint64_t mid = lo \+ width < n \? lo \+ width : n;",
                  "uint64_t mid = lo + width + 1 < n ? lo + width + 1 : n;"),
    # 64-bit float map without the complement of negatives
    "f64_negatives": (r"if \(bits & sign\)\n            return ~bits;",
                      "if (bits & sign)\n            return bits;"),
    # 64-bit signed map without the sign flip
    "i64_sign": (r"return bits \^ sign;\n    if \(dtype == ORC_F64\)",
                 "return bits;\n    if (dtype == ORC_F64)"),
    # 64-bit merge drops the left run's tail
    "lost_tail64": (r"while \(i < mid\)\n        dst\[o\+\+\] = src\[i\+\+\];",
                    "while (0)\n        dst[o++] = src[i++];"),
    # 64-bit merge takes from the wrong run
    "merge64_order": (r"if \(orc_key64\(src\[j\], dtype\) < orc_key64\(src\[i\], dtype\)\)",
                      "if (orc_key64(src[j], dtype) > orc_key64(src[i], dtype))"),
}


def _pins(orc):
    """A compact replay of the pins above against one oracle copy; returns
    the names of the pins that fail."""
    failed = []
    x = inputs.keys(5000, "u32", "uniform", seed=1)
    if not np.array_equal(orc.sort_keys(x, "u32"), np.sort(x)):
        failed.append("numpy_u32")
    if not np.array_equal(orc.sort_keys(x, "i32").view(np.int32), np.sort(x.view(np.int32))):
        failed.append("numpy_i32")
    bits = np.array([0xBF800000, 0x80000000, 0x00000000, 0x3F800000], np.uint32)
    if not np.all(np.diff(orc.key(bits, "f32").astype(np.int64)) > 0):
        failed.append("f32_table")
    d = inputs.keys(5000, "u32", "dup16", seed=1)
    v = np.arange(d.size, dtype=np.uint32)
    ko, vo = orc.sort_pairs(d, v, "u32")
    perm = np.argsort(d, kind="stable")
    if not (np.array_equal(ko, d[perm]) and np.array_equal(vo, v[perm])):
        failed.append("stable_pairs")
    y = inputs.keys64(5000, "u64", "uniform", seed=1)
    if not np.array_equal(orc.sort_keys64(y, "u64"), np.sort(y)):
        failed.append("numpy_u64")
    if not np.array_equal(orc.sort_keys64(y, "i64").view(np.int64), np.sort(y.view(np.int64))):
        failed.append("numpy_i64")
    b64 = np.array([0xBFF0000000000000, 0x8000000000000000, 0x0, 0x3FF0000000000000], np.uint64)
    k64 = orc.key64(b64, "f64")
    if not np.all(k64[1:] > k64[:-1]):
        failed.append("f64_table")
    return failed


def test_pins_pass_on_the_real_oracle():
    assert _pins(oracle.default()) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistakes(tmp_path, name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    pat, rep = MUTATIONS[name]
    mutated, count = re.subn(pat, rep, src, count=1)
    assert count == 1, f"mutation {name} did not apply"
    c = tmp_path / f"oracle_{name}.c"
    c.write_text(mutated)
    lib = oracle.compile_source(str(c), str(tmp_path / f"lib_{name}.so"))
    assert _pins(oracle.Oracle(lib)) != [], f"planted mistake {name} went unnoticed"
