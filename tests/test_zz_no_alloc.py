"""The allocation-free key sort (nsort_keys_noalloc), for callers that cannot
allocate device memory — their memory belongs to another allocator, or a
cudaMalloc could block or synchronise where they run.  Its scratch is a fixed
array inside the library, shared by every call on a device.

The test calls it twice in a row through the C ABI, with different sizes and
key types so that the second call starts from what the first left in the
shared array, and checks each result bit for bit against nsort_keys (the
entry point that takes a caller-provided scratch buffer).  This file is
collected last, so that a run stopping at the first failure has already run
every other test."""
import numpy as np
import pytest

from paper_2409_03970_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ns():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03970_gb300 import build, nsort
    build.build()
    nsort.lib()
    return nsort


def _sorted_both_ways(ns, bits, code):
    n = bits.size
    x = torch.from_numpy(bits.view(np.int32)).cuda()
    out_noalloc = torch.empty_like(x)
    rc = ns.nsort_keys_noalloc(x, out_noalloc, n, code)
    assert rc == ns.OK, ns.lib().nsort_last_error()
    out_ref = torch.empty_like(x)
    tmp = ns.scratch(ns.KIND_KEYS, n)
    rc = ns.nsort_keys(x, out_ref, n, code, tmp, tmp.numel())
    assert rc == ns.OK, ns.lib().nsort_last_error()
    torch.cuda.synchronize()
    return out_noalloc.cpu().numpy(), out_ref.cpu().numpy()


def test_noalloc_matches_nsort_keys_on_two_calls_in_a_row(ns):
    first = inputs.keys(ns.NOALLOC_MAX_KEYS, "u32", "uniform", seed=21)       # the maximum size
    k, _ = inputs.normal_pairs(300_001, seed=22, special_per_mille=20)        # smaller, float keys
    for bits, code in ((first, ns.U32), (k, ns.F32)):
        got, want = _sorted_both_ways(ns, bits, code)
        assert np.array_equal(got, want)


def test_noalloc_rejects_sizes_above_its_maximum(ns):
    x = torch.zeros(16, dtype=torch.int32, device="cuda")
    rc = ns.nsort_keys_noalloc(x, x, ns.NOALLOC_MAX_KEYS + 1, ns.U32)
    assert rc == ns.ENOMEM
    assert "maximum" in ns.lib().nsort_last_error().decode()
