"""Seeded synthetic inputs, shared by the tests, the benchmark and smoke().

This module holds none of the sort's arithmetic: it only draws numbers.  The
paper sorts "random integers" (Sec. 3); the other workloads (signed and
float keys, duplicates, Zipf, stable pairs with IEEE special values, uneven
segments, a request stream) are synthetic stand-ins with the shapes and
value distributions of the benchmark configurations.

Every number comes from one counter-based generator, so any element can be
recomputed from (seed, stream, index) alone, on any machine:

    base(seed, stream) = mix64(seed * 2^16 + stream + 1)
    x(seed, stream, i) = mix64(base + (i + 1) * 0x9E3779B97F4A7C15)

where mix64 is the splitmix64 finaliser (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014):
z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB;
z ^= z >> 31 (all mod 2^64).  A 32-bit draw is the high half of x.

All key arrays are returned as numpy uint32 bit patterns; ``as_dtype`` views
them as uint32 / int32 / float32.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
CHUNK = 1 << 22

KEY_DTYPES = ("u32", "i32", "f32")
DISTRIBUTIONS = ("uniform", "sorted", "reverse", "dup16", "zipf")

# streams: independent sub-sequences of one seed
S_KEYS, S_PICK, S_DUP, S_SPECIAL, S_LEN, S_ZIPF, S_NORMAL2, S_SERVE = range(8)


def mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def _base(seed: int, stream: int) -> np.uint64:
    v = np.array([(int(seed) & 0xFFFFFFFFFFFF) * 65536 + int(stream) + 1], dtype=np.uint64)
    return mix64(v)[0]


def counter_u64(seed: int, stream: int, lo: int, hi: int) -> np.ndarray:
    """x(seed, stream, i) for i in [lo, hi)."""
    idx = np.arange(lo, hi, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _base(seed, stream) + (idx + np.uint64(1)) * GOLDEN
    return mix64(z)


def counter_u32(seed: int, stream: int, lo: int, hi: int) -> np.ndarray:
    return (counter_u64(seed, stream, lo, hi) >> np.uint64(32)).astype(np.uint32)


def unit_double(x: np.ndarray) -> np.ndarray:
    """Uniform double in [0, 1) from the top 53 bits."""
    return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _int_bits_to_dtype(bits: np.ndarray, dtype: str) -> np.ndarray:
    """Maps 32-bit integer draws to key patterns of `dtype`.  u32 / i32: the
    draw itself (every 2^32 pattern is possible).  f32: the draw read as an
    int32, converted to float32 and scaled by 2^-31, i.e. U[-1, 1) — no NaN,
    no infinity."""
    if dtype in ("u32", "i32"):
        return bits.astype(np.uint32, copy=False)
    if dtype == "f32":
        f = bits.view(np.int32).astype(np.float32) * np.float32(2.0 ** -31)
        return f.view(np.uint32)
    raise ValueError(f"unknown key dtype {dtype!r}")


def as_dtype(bits: np.ndarray, dtype: str) -> np.ndarray:
    return bits.view({"u32": np.uint32, "i32": np.int32, "f32": np.float32}[dtype])


def _zipf_cdf(ranks: int) -> np.ndarray:
    w = 1.0 / np.arange(1, ranks + 1, dtype=np.float64)
    c = np.cumsum(w)
    return c / c[-1]


def keys(n: int, dtype: str = "u32", dist: str = "uniform", seed: int = 0,
         zipf_ranks: int = 1 << 20) -> np.ndarray:
    """n key bit patterns (uint32) of the given dtype and distribution.

    uniform : one 32-bit draw per element (float32: U[-1, 1)).
    sorted  : ascending in the dtype's order without any sorting step:
              element i is drawn inside the i-th of n equal slices of the
              32-bit range (signed order for i32, then scaled to U[-1,1) for
              f32; int-to-float rounding keeps the order).
    reverse : the sorted sequence, last element first.
    dup16   : 16 values drawn as for uniform; each element picks one of them.
    zipf    : Zipf(s=1) ranks over `zipf_ranks` values by inverse CDF (binary
              search on the prefix sums of 1/r); rank r's value is the 32-bit
              draw of stream S_ZIPF at index r, so frequent values are
              scattered over the key range.
    """
    if dtype not in KEY_DTYPES:
        raise ValueError(f"unknown key dtype {dtype!r}")
    if dist not in DISTRIBUTIONS:
        raise ValueError(f"unknown distribution {dist!r}")
    out = np.empty(n, dtype=np.uint32)
    if n == 0:
        return out
    if dist == "dup16":
        table = _int_bits_to_dtype(counter_u32(seed, S_DUP, 0, 16), dtype)
    if dist == "zipf":
        cdf = _zipf_cdf(zipf_ranks)
    for lo in range(0, n, CHUNK):
        hi = min(n, lo + CHUNK)
        if dist == "uniform":
            out[lo:hi] = _int_bits_to_dtype(counter_u32(seed, S_KEYS, lo, hi), dtype)
        elif dist in ("sorted", "reverse"):
            if dist == "sorted":
                i = np.arange(lo, hi, dtype=np.uint64)
            else:
                i = np.uint64(n - 1) - np.arange(lo, hi, dtype=np.uint64)
            # slice i of [0, 2^32): [floor(i 2^32 / n), floor((i+1) 2^32 / n))
            start = (i << np.uint64(32)) // np.uint64(n)
            stop = ((i + np.uint64(1)) << np.uint64(32)) // np.uint64(n)
            width = np.maximum(stop - start, np.uint64(1))
            jit = counter_u64(seed, S_KEYS, lo, hi) % width
            v = (start + jit).astype(np.uint32)
            if dtype in ("i32", "f32"):
                v = v ^ np.uint32(0x80000000)      # ascending in signed order
            out[lo:hi] = _int_bits_to_dtype(v, dtype)
        elif dist == "dup16":
            pick = counter_u32(seed, S_PICK, lo, hi) & np.uint32(15)
            out[lo:hi] = table[pick]
        elif dist == "zipf":
            u = unit_double(counter_u64(seed, S_KEYS, lo, hi))
            r = np.searchsorted(cdf, u, side="right")
            r = np.minimum(r, zipf_ranks - 1).astype(np.uint64) + np.uint64(1)
            z = mix64(_base(seed, S_ZIPF) + r * GOLDEN)
            out[lo:hi] = _int_bits_to_dtype((z >> np.uint64(32)).astype(np.uint32), dtype)
    return out


KEY64_DTYPES = ("u64", "i64", "f64")
DISTRIBUTIONS64 = ("uniform", "sorted", "reverse", "dup16", "specials")

# IEEE binary64 specials: -0, +0, +Inf, -Inf, +qNaN, -qNaN, +sNaN,
# smallest subnormal, -DBL_MAX
SPECIALS_F64 = np.array([0x8000000000000000, 0x0000000000000000, 0x7FF0000000000000,
                         0xFFF0000000000000, 0x7FF8000000000000, 0xFFF8000000000000,
                         0x7FF0000000000001, 0x0000000000000001, 0xFFEFFFFFFFFFFFFF],
                        dtype=np.uint64)


def _int64_bits_to_dtype(bits: np.ndarray, dtype: str) -> np.ndarray:
    """64-bit draws to key patterns: u64 / i64 the draw itself; f64 the draw
    read as an int64, converted to float64 and scaled by 2^-63 (U[-1, 1))."""
    if dtype in ("u64", "i64"):
        return bits.astype(np.uint64, copy=False)
    if dtype == "f64":
        return (bits.view(np.int64).astype(np.float64) * (2.0 ** -63)).view(np.uint64)
    raise ValueError(f"unknown 64-bit key dtype {dtype!r}")


def keys64(n: int, dtype: str = "u64", dist: str = "uniform", seed: int = 0) -> np.ndarray:
    """n 64-bit key patterns (uint64) of the given dtype and distribution.

    uniform  : one 64-bit draw per element (float64: U[-1, 1)).
    sorted   : ascending in the dtype's order without a sorting step: element
               i is i * floor(2^64 / n) plus a draw below that step (signed
               order for i64, then scaled for f64).
    reverse  : the sorted sequence, last element first.
    dup16    : 16 values drawn as for uniform; each element picks one.
    specials : uniform, with about 1/1000 of the positions replaced by one
               of SPECIALS_F64 (f64) or by 0, 1, 2^63 - 1, 2^63, 2^64 - 1
               (u64 / i64), chosen by draw(S_SPECIAL, i).
    """
    if dtype not in KEY64_DTYPES:
        raise ValueError(f"unknown 64-bit key dtype {dtype!r}")
    if dist not in DISTRIBUTIONS64:
        raise ValueError(f"unknown distribution {dist!r}")
    out = np.empty(n, dtype=np.uint64)
    if n == 0:
        return out
    edges = np.array([0, 1, 0x7FFFFFFFFFFFFFFF, 0x8000000000000000, 0xFFFFFFFFFFFFFFFF],
                     dtype=np.uint64)
    table = _int64_bits_to_dtype(counter_u64(seed, S_DUP, 0, 16), dtype)
    step = np.uint64(min((1 << 64) // n, (1 << 64) - 1))
    for lo in range(0, n, CHUNK):
        hi = min(n, lo + CHUNK)
        if dist in ("uniform", "specials"):
            v = _int64_bits_to_dtype(counter_u64(seed, S_KEYS, lo, hi), dtype)
            if dist == "specials":
                h = counter_u64(seed, S_SPECIAL, lo, hi)
                sp = (h % np.uint64(1000)) == np.uint64(0)
                sel = h >> np.uint64(40)
                if dtype == "f64":
                    rep = SPECIALS_F64[(sel % np.uint64(SPECIALS_F64.size)).astype(np.int64)]
                else:
                    rep = edges[(sel % np.uint64(edges.size)).astype(np.int64)]
                v = np.where(sp, rep, v)
            out[lo:hi] = v
        elif dist in ("sorted", "reverse"):
            if dist == "sorted":
                i = np.arange(lo, hi, dtype=np.uint64)
            else:
                i = np.uint64(n - 1) - np.arange(lo, hi, dtype=np.uint64)
            with np.errstate(over="ignore"):
                v = i * step + counter_u64(seed, S_KEYS, lo, hi) % max(step, np.uint64(1))
            if dtype in ("i64", "f64"):
                v = v ^ np.uint64(0x8000000000000000)   # ascending in signed order
            out[lo:hi] = _int64_bits_to_dtype(v, dtype)
        else:   # dup16
            out[lo:hi] = table[counter_u32(seed, S_PICK, lo, hi) & np.uint32(15)]
    return out


# IEEE binary32 specials used by the stable-pairs workload
SPECIALS_F32 = np.array([0x80000000, 0x00000000, 0x7F800000, 0xFF800000,
                         0x7FC00000, 0xFFC00000, 0x7F800001], dtype=np.uint32)


def normal_pairs(n: int, seed: int = 0, special_per_mille: int = 1):
    """float32 keys ~ Normal(0, 1) with about `special_per_mille`/1000 of the
    positions replaced by one of SPECIALS_F32 (-0, +0, +Inf, -Inf, +qNaN,
    -qNaN, +sNaN), each paired with a uint32 payload equal to its index.

    Box-Muller in double from two counter uniforms u1 in (0, 1], u2 in
    [0, 1): z = sqrt(-2 ln u1) cos(2 pi u2), rounded to float32.  A position
    i is special when draw(S_SPECIAL, i) mod 1000 < special_per_mille; the
    special is SPECIALS_F32[(draw >> 40) mod 7].  Many keys repeat (float32
    rounding and the specials), so equal keys exercise stability."""
    k = np.empty(n, dtype=np.uint32)
    for lo in range(0, n, CHUNK):
        hi = min(n, lo + CHUNK)
        u1 = 1.0 - unit_double(counter_u64(seed, S_KEYS, lo, hi))
        u2 = unit_double(counter_u64(seed, S_NORMAL2, lo, hi))
        z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
        kb = z.astype(np.float32).view(np.uint32)
        h = counter_u64(seed, S_SPECIAL, lo, hi)
        sp = (h % np.uint64(1000)) < np.uint64(special_per_mille)
        kb = np.where(sp, SPECIALS_F32[((h >> np.uint64(40)) % np.uint64(7)).astype(np.int64)], kb)
        k[lo:hi] = kb
    v = np.arange(n, dtype=np.uint32)
    return k, v


def segment_offsets(nseg: int, seed: int = 0, max_len: int = 65536,
                    min_len: int = 1) -> np.ndarray:
    """int64 CSR offsets (nseg+1 entries) of nseg segments whose lengths are
    log-uniform: L = clamp(floor(2^(log2(max_len) * u)), min_len, max_len)."""
    u = unit_double(counter_u64(seed, S_LEN, 0, nseg))
    lg = math.log2(max_len)
    lens = np.floor(np.exp2(lg * u)).astype(np.int64)
    lens = np.clip(lens, min_len, max_len)
    off = np.zeros(nseg + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    return off
