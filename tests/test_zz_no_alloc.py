"""The allocation-free key sort (nsort_keys_noalloc), for callers that cannot
allocate device memory — their memory belongs to another allocator, or a
cudaMalloc could block or synchronise where they run.  Its scratch is a fixed
array inside the library, shared by every call on a device.

Each case calls it through the C ABI and checks the result bit for bit
against the oracle and against nsort_keys (the entry point that takes a
caller-provided scratch buffer).  Two calls in a row, with different sizes
and key types, make the second start from what the first left in the shared
array.  The other cases take the paths through that array that the first
two do not: a sort within one tile (no scratch), an output 4 bytes past a
16-byte boundary (the staged-load merge passes) and an in-place sort.  After
each call nsort_keys_noalloc_status reports the call's device status.

This file is collected last, so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import oracle
from paper_2409_03970_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = {0: "u32", 1: "i32", 2: "f32"}


@pytest.fixture(scope="module")
def ns():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03970_gb300 import build, nsort
    build.build()
    nsort.lib()
    return nsort


def _noalloc(ns, bits, code, offset=0, inplace=False):
    """nsort_keys_noalloc on bits placed `offset` words into a fresh device
    buffer; returns the output as uint32."""
    n = bits.size
    x = torch.from_numpy(np.concatenate([np.zeros(offset, np.uint32), bits]).view(np.int32))
    x = x.cuda()[offset:]
    out = x if inplace else torch.empty(n + offset, dtype=torch.int32, device="cuda")[offset:]
    rc = ns.nsort_keys_noalloc(x, out, n, code)
    assert rc == ns.OK, ns.lib().nsort_last_error()
    assert ns.nsort_keys_noalloc_status() == ns.OK
    return out.cpu().numpy().view(np.uint32)


def _with_scratch(ns, bits, code):
    n = bits.size
    x = torch.from_numpy(bits.view(np.int32)).cuda()
    out = torch.empty_like(x)
    tmp = ns.scratch(ns.KIND_KEYS, n)
    rc = ns.nsort_keys(x, out, n, code, tmp, tmp.numel())
    assert rc == ns.OK, ns.lib().nsort_last_error()
    return out.cpu().numpy().view(np.uint32)


def _check(ns, bits, code, **kw):
    got = _noalloc(ns, bits, code, **kw)
    want = oracle.sort_keys(bits, NAMES[code])
    assert np.array_equal(got, want)
    assert np.array_equal(got, _with_scratch(ns, bits, code))


def test_noalloc_matches_oracle_and_nsort_keys_on_two_calls_in_a_row(ns):
    first = inputs.keys(ns.NOALLOC_MAX_KEYS, "u32", "uniform", seed=21)       # the maximum size
    k, _ = inputs.normal_pairs(300_001, seed=22, special_per_mille=20)        # smaller, float keys
    _check(ns, first, ns.U32)
    _check(ns, k, ns.F32)


@pytest.mark.parametrize("n", [1, 5000, 16384])
def test_noalloc_within_one_tile(ns, n):
    """No merge pass and no scratch: the status word is still cleared."""
    _check(ns, inputs.keys(n, "i32", "dup16", seed=n), ns.I32)


def test_noalloc_output_off_a_16_byte_boundary(ns):
    """4 bytes past a 16-byte boundary: the merge passes stage their loads
    instead of using bulk copies."""
    _check(ns, inputs.keys(200_003, "f32", "zipf", seed=23), ns.F32, offset=1)


def test_noalloc_in_place(ns):
    _check(ns, inputs.keys(123_457, "u32", "reverse", seed=24), ns.U32, inplace=True)


def test_noalloc_rejects_sizes_above_its_maximum(ns):
    x = torch.zeros(16, dtype=torch.int32, device="cuda")
    rc = ns.nsort_keys_noalloc(x, x, ns.NOALLOC_MAX_KEYS + 1, ns.U32)
    assert rc == ns.ENOMEM
    assert "maximum" in ns.lib().nsort_last_error().decode()
