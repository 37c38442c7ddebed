"""Host-side policy of the sort server, checked without a GPU: the FIFO
admission with co-batching of small requests and large requests one at a
time, and the first-fit scratch arena (nsort_policy_* hooks, no CUDA
calls)."""
import pytest

from paper_2409_03970_gb300 import build as nbuild
from paper_2409_03970_gb300 import nsort

K, P = nsort.KIND_KEYS, nsort.KIND_PAIRS


@pytest.fixture(scope="module", autouse=True)
def lib():
    nbuild.build()
    return nsort.lib()


def test_fifo_head_runs_alone_when_large():
    q = [(1, K, 0, 1 << 20), (2, K, 0, 100), (3, K, 0, 200)]
    assert nsort.policy_pick_batch(q, batch_max_keys=1 << 16) == [1]


def test_small_head_collects_same_class_in_arrival_order():
    q = [(1, K, 0, 100), (2, K, 1, 100), (3, P, 0, 100), (4, K, 0, 1 << 20), (5, K, 0, 300),
         (6, K, 0, 5)]
    # same kind and dtype as the head, small, arrival order; others wait
    assert nsort.policy_pick_batch(q, batch_max_keys=1 << 16) == [1, 5, 6]
    assert nsort.policy_pick_batch(q[1:], batch_max_keys=1 << 16) == [2]
    assert nsort.policy_pick_batch(q[2:], batch_max_keys=1 << 16) == [3]


def test_batch_limits_and_disabled_batching():
    q = [(i, K, 0, 1000) for i in range(1, 11)]
    assert nsort.policy_pick_batch(q, 1 << 16, max_batch=4) == [1, 2, 3, 4]
    assert nsort.policy_pick_batch(q, 1 << 16, max_batch_keys=3500) == [1, 2, 3]
    assert nsort.policy_pick_batch(q, 0) == [1]                    # batching off: plain FIFO
    assert nsort.policy_pick_batch([], 1 << 16) == []


def test_large_requests_run_one_at_a_time():
    L = nsort.SERVE_LARGE_MIN_KEYS
    q = [(1, K, 0, L), (2, P, 0, 4 * L), (3, K, 0, L - 1), (4, K, 0, 100), (5, K, 0, 50)]
    # no large request running: plain FIFO, the large head runs alone
    assert nsort.policy_pick_batch(q, 1 << 16, large_min_keys=L) == [1]
    # one running: the large ones wait and the first smaller request goes ahead
    assert nsort.policy_pick_batch(q, 1 << 16, large_min_keys=L, large_running=True) == [3]
    # a small one that goes ahead still collects its class behind it
    assert nsort.policy_pick_batch(q[:2] + q[3:], 1 << 16, large_min_keys=L,
                                   large_running=True) == [4, 5]
    # only large requests wait: nothing may start
    assert nsort.policy_pick_batch(q[:2], 1 << 16, large_min_keys=L, large_running=True) == []
    # without a large-size limit the flag changes nothing
    assert nsort.policy_pick_batch(q, 1 << 16, large_running=True) == [1]


def test_arena_first_fit_coalescing_and_exhaustion():
    cap = 1 << 20
    ops = [1000, 300_000, 500_000,     # 0, 1, 2: allocate (1000 rounds up to 1024)
           -2,                         # 3: release op 1
           200_000,                    # 4: fits in the hole left by op 1
           400_000,                    # 5: does not fit anywhere
           -1, -5, -3,                 # 6, 7, 8: release everything
           cap]                        # 9: the whole arena again (coalesced)
    r = nsort.policy_arena_replay(cap, ops)
    assert r[0] == 0 and r[1] == 1024 and r[2] == 1024 + 300_032
    assert r[4] == 1024                # first fit reuses the hole
    assert r[5] == -1
    assert r[9] == 0


def test_arena_rejects_bad_release():
    with pytest.raises(nsort.NsortError):
        nsort.policy_arena_replay(1 << 20, [100, -5])
