"""Failure detection without a GPU fault: the library's in-kernel waits are
bounded.  nsort_selftest_wait runs the same wait helpers the merge pass and
the segmented sort use (an mbarrier wait and a completion-counter wait) on
events that never happen; both give up after the given limit, the kernel
records NSORT_ETIMEOUT in the scratch status word and returns normally, and
the context keeps working."""
import time

import numpy as np
import pytest

import oracle
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


def test_bounded_waits_give_up_and_report(ns):
    tmp = torch.empty(1024, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    assert ns.nsort_selftest_wait(tmp, limit_us=20_000) == ns.OK
    assert ns.nsort_device_status(tmp) == ns.ETIMEOUT
    elapsed = time.perf_counter() - t0
    assert 0.03 <= elapsed < 5.0          # two 20 ms waits, then the kernel returned
    # the context is still usable and exact
    n = 100_003
    x = inputs.keys(n, "f32", "uniform", seed=31)
    xt = torch.from_numpy(x.view(np.int32)).cuda()
    out = torch.empty_like(xt)
    sc = ns.scratch(ns.KIND_KEYS, n)
    assert ns.nsort_keys(xt, out, n, ns.F32, sc, sc.numel()) == ns.OK
    assert ns.nsort_device_status(sc) == ns.OK
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), oracle.sort_keys(x, "f32"))


def test_status_word_reports_ok_after_normal_sorts(ns):
    n = 1 << 20
    x = torch.from_numpy(inputs.keys(n, "u32", "uniform", seed=32).view(np.int32)).cuda()
    out = torch.empty_like(x)
    sc = ns.scratch(ns.KIND_KEYS, n)
    assert ns.nsort_keys(x, out, n, ns.U32, sc, sc.numel()) == ns.OK
    assert ns.nsort_device_status(sc) == ns.OK
