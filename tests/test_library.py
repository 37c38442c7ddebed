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
    passes, st, mt = nsort.nsort_plan(nsort.KIND_KEYS, 1 << 28)
    assert st & (st - 1) == 0 and mt > 0          # run lengths double from a power of two
    # one tile sort + ceil(log2(2^28 / tile)) merge passes
    assert passes == 1 + (28 - st.bit_length() + 1)
    assert nsort.nsort_plan(nsort.KIND_KEYS, 1)[0] == 1
    assert nsort.nsort_plan(nsort.KIND_KEYS, st)[0] == 1
    assert nsort.nsort_plan(nsort.KIND_KEYS, st + 1)[0] == 2
    assert nsort.nsort_plan(nsort.KIND_KEYS, 3 * st)[0] == 3
    p2, st2, _ = nsort.nsort_plan(nsort.KIND_PAIRS, 1 << 27)
    assert p2 == 1 + (27 - st2.bit_length() + 1)


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
    assert 8 * n <= tp <= 8 * n + 8 * (n // pmt + n // (2 * pst) + 3) + 1024
    assert nsort.nsort_temp_bytes(99, n) == 0


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
