"""CPU oracle for the NEON-MS sort — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (``libnsort`` and its
Python binding) never imports it, and the two share no code.

Two parts:

* ``oracle.c`` (loaded here through ctypes): the plain definition of what the
  method computes — a stable ascending sort of 32-bit keys (paper Sec. 2.1),
  written as a textbook bottom-up merge sort, plus the order-preserving key
  map for int32 / float32 keys (IEEE 754-2008 totalOrder for float32), and
  the same for 64-bit keys (uint64 / int64 / float64).  A multi-threaded
  form of the same sort (chunk sorts, then pairwise merges) gives the CPU
  baseline's second figure; the tests check it against the serial one.
* ``networks.py``: the comparator networks the paper compares in Table 1
  (bitonic, odd-even, the 60-comparator 16-input network) and the merging
  networks of Sec. 2.4, as data, with an exhaustive 0-1-principle verifier.

Every function is pinned by ``tests/test_oracle.py`` / ``tests/test_networks.py``
against things other than itself (brute force, textbook insertion sort, IEEE
comparisons by numpy, the paper's Table 1 counts, closed forms).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

DTYPES = {"u32": 0, "i32": 1, "f32": 2}
DTYPES64 = {"u64": 3, "i64": 4, "f64": 5}

_lock = threading.Lock()
_lib = None


def compile_source(src: str, out: str) -> str:
    """Compiles a C source of the oracle into a shared library with gcc
    (plain C, portable: no target-specific flags)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-pthread", "-shared", "-fPIC", "-o", tmp,
                           src])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Builds oracle/_build/liboracle.so when missing or older than oracle.c."""
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        compile_source(_SRC, _LIB_PATH)
    return _LIB_PATH


def _dt(dtype: str) -> int:
    if dtype not in DTYPES:
        raise ValueError(f"unknown key dtype {dtype!r}; expected one of {sorted(DTYPES)}")
    return DTYPES[dtype]


def _dt64(dtype: str) -> int:
    if dtype not in DTYPES64:
        raise ValueError(f"unknown 64-bit key dtype {dtype!r}; expected one of {sorted(DTYPES64)}")
    return DTYPES64[dtype]


def _u64(a) -> np.ndarray:
    a = np.ascontiguousarray(a)
    if a.dtype.itemsize != 8:
        raise TypeError(f"expected a 64-bit array, got {a.dtype}")
    return a.view(np.uint64)


def _u32(a) -> np.ndarray:
    a = np.ascontiguousarray(a)
    if a.dtype.itemsize != 4:
        raise TypeError(f"expected a 32-bit array, got {a.dtype}")
    return a.view(np.uint32)


def _p(a: np.ndarray, ty=ctypes.c_uint32):
    return a.ctypes.data_as(ctypes.POINTER(ty))


class Oracle:
    """ctypes view of one compiled copy of oracle.c."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.orc_key.argtypes = [ctypes.c_uint32, ctypes.c_int]
        lib.orc_key.restype = ctypes.c_uint32
        lib.orc_key_array.argtypes = [u32p, u32p, ctypes.c_uint64, ctypes.c_int]
        lib.orc_key_array.restype = None
        lib.orc_sort_keys.argtypes = [u32p, u32p, ctypes.c_uint64, ctypes.c_int]
        lib.orc_sort_keys.restype = ctypes.c_int
        lib.orc_sort_keys_par.argtypes = [u32p, u32p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int]
        lib.orc_sort_keys_par.restype = ctypes.c_int
        lib.orc_sort_pairs.argtypes = [u32p, u32p, u32p, u32p, ctypes.c_uint64, ctypes.c_int]
        lib.orc_sort_pairs.restype = ctypes.c_int
        lib.orc_sort_segmented.argtypes = [u32p, u32p, u32p, u32p, i64p,
                                           ctypes.c_uint64, ctypes.c_int]
        lib.orc_sort_segmented.restype = ctypes.c_int
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.orc_key64.argtypes = [ctypes.c_uint64, ctypes.c_int]
        lib.orc_key64.restype = ctypes.c_uint64
        lib.orc_key64_array.argtypes = [u64p, u64p, ctypes.c_uint64, ctypes.c_int]
        lib.orc_key64_array.restype = None
        lib.orc_sort_keys64.argtypes = [u64p, u64p, ctypes.c_uint64, ctypes.c_int]
        lib.orc_sort_keys64.restype = ctypes.c_int
        self.lib = lib
        self.path = path

    def key(self, bits, dtype: str) -> np.ndarray:
        """The order-preserving unsigned key of each 32-bit pattern."""
        b = _u32(np.atleast_1d(bits))
        out = np.empty_like(b)
        self.lib.orc_key_array(_p(b), _p(out), b.size, _dt(dtype))
        return out

    def sort_keys(self, bits, dtype: str) -> np.ndarray:
        """The input bit patterns (uint32 view) in ascending key order."""
        b = _u32(bits)
        out = np.empty_like(b)
        rc = self.lib.orc_sort_keys(_p(b), _p(out), b.size, _dt(dtype))
        if rc != 0:
            raise RuntimeError(f"orc_sort_keys failed ({rc})")
        return out

    def sort_keys_par(self, bits, dtype: str, threads: int) -> np.ndarray:
        """sort_keys on `threads` host threads (chunk sorts, then pairwise
        merges): the CPU baseline's multi-threaded figure."""
        b = _u32(bits)
        out = np.empty_like(b)
        rc = self.lib.orc_sort_keys_par(_p(b), _p(out), b.size, _dt(dtype), int(threads))
        if rc != 0:
            raise RuntimeError(f"orc_sort_keys_par failed ({rc})")
        return out

    def key64(self, bits, dtype: str) -> np.ndarray:
        """The order-preserving unsigned key of each 64-bit pattern."""
        b = _u64(np.atleast_1d(bits))
        out = np.empty_like(b)
        self.lib.orc_key64_array(_p(b, ctypes.c_uint64), _p(out, ctypes.c_uint64), b.size,
                                 _dt64(dtype))
        return out

    def sort_keys64(self, bits, dtype: str) -> np.ndarray:
        """The input 64-bit patterns (uint64 view) in ascending key order."""
        b = _u64(bits)
        out = np.empty_like(b)
        rc = self.lib.orc_sort_keys64(_p(b, ctypes.c_uint64), _p(out, ctypes.c_uint64), b.size,
                                      _dt64(dtype))
        if rc != 0:
            raise RuntimeError(f"orc_sort_keys64 failed ({rc})")
        return out

    def sort_pairs(self, bits, vals, dtype: str):
        """Stable key/value sort.  Returns (keys, vals) as uint32 arrays."""
        b = _u32(bits)
        v = _u32(vals)
        if v.size != b.size:
            raise ValueError("keys and values differ in length")
        ko = np.empty_like(b)
        vo = np.empty_like(v)
        rc = self.lib.orc_sort_pairs(_p(b), _p(v), _p(ko), _p(vo), b.size, _dt(dtype))
        if rc != 0:
            raise RuntimeError(f"orc_sort_pairs failed ({rc})")
        return ko, vo

    def sort_segmented(self, bits, offsets, dtype: str, vals=None):
        """Sorts each segment [offsets[s], offsets[s+1]) on its own (stable).
        Returns keys, or (keys, vals) when vals is given."""
        b = _u32(bits)
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        if off.size < 1 or off[-1] != b.size:
            raise ValueError("offsets must have nseg+1 entries ending at len(keys)")
        ko = np.empty_like(b)
        if vals is not None:
            v = _u32(vals)
            vo = np.empty_like(v)
            vp, vop = _p(v), _p(vo)
        else:
            vo = None
            vp = vop = None
        rc = self.lib.orc_sort_segmented(_p(b), vp, _p(ko), vop, _p(off, ctypes.c_int64),
                                         off.size - 1, _dt(dtype))
        if rc != 0:
            raise RuntimeError(f"orc_sort_segmented failed ({rc})")
        return ko if vals is None else (ko, vo)


def default() -> Oracle:
    global _lib
    with _lock:
        if _lib is None:
            _lib = Oracle(build())
    return _lib


def key(bits, dtype: str) -> np.ndarray:
    return default().key(bits, dtype)


def sort_keys(bits, dtype: str) -> np.ndarray:
    return default().sort_keys(bits, dtype)


def sort_keys_par(bits, dtype: str, threads: int) -> np.ndarray:
    return default().sort_keys_par(bits, dtype, threads)


def sort_pairs(bits, vals, dtype: str):
    return default().sort_pairs(bits, vals, dtype)


def sort_segmented(bits, offsets, dtype: str, vals=None):
    return default().sort_segmented(bits, offsets, dtype, vals)


def key64(bits, dtype: str) -> np.ndarray:
    return default().key64(bits, dtype)


def sort_keys64(bits, dtype: str) -> np.ndarray:
    return default().sort_keys64(bits, dtype)
