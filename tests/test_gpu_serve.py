"""GPU tests of the sort server (nsort_ctx_* / nsort_submit / poll / wait):
a mixed stream of key and pair requests of many sizes and dtypes, checked
bit for bit against the oracle; every result identical alone (plain FIFO,
one at a time) and in the mix (co-batched, overlapping); admission under a
memory budget that fits one request at a time; error paths."""
import numpy as np
import pytest

import oracle
from paper_2409_03970_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"u32": 0, "i32": 1, "f32": 2}


@pytest.fixture(scope="module")
def ns():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03970_gb300 import build, nsort
    build.build()
    nsort.lib()
    return nsort


def make_requests(count, seed, lo=10, hi=20):
    """(kind, dtype, keys, vals) with sizes log-uniform in [2^lo, 2^hi] and the
    dtype mix {u32, i32, f32 keys, f32 key + u32 value}."""
    u = inputs.unit_double(inputs.counter_u64(seed, inputs.S_SERVE, 0, count))
    pick = inputs.counter_u32(seed, inputs.S_SERVE + 1, 0, count) % 4
    reqs = []
    for i in range(count):
        n = int(2 ** (lo + (hi - lo) * u[i]))
        mode = ["u32", "i32", "f32", "pairs"][int(pick[i])]
        if mode == "pairs":
            k, v = inputs.normal_pairs(n, seed=seed * 1000 + i, special_per_mille=10)
            reqs.append(("pairs", "f32", k, v))
        else:
            reqs.append(("keys", mode, inputs.keys(n, mode, "uniform", seed=seed * 1000 + i), None))
    return reqs


def run_all(ns, reqs, streams, batch_max_keys, budget=1 << 31, sequential=False):
    outs, tickets = [], []
    with ns.SortServer(0, budget, streams, batch_max_keys) as srv:
        bufs = []
        for kind, dt, k, v in reqs:
            kt = torch.from_numpy(k.view(np.int32)).cuda()
            ko = torch.empty_like(kt)
            vt = vo = None
            if v is not None:
                vt = torch.from_numpy(v.view(np.int32)).cuda()
                vo = torch.empty_like(vt)
            bufs.append((kt, ko, vt, vo))
        torch.cuda.synchronize()
        for (kind, dt, k, v), (kt, ko, vt, vo) in zip(reqs, bufs):
            t = srv.submit(kt, ko, vt, vo, n=k.size, dtype=DT[dt])
            tickets.append(t)
            if sequential:
                assert srv.wait(t) == ns.OK
        timings = []
        for t in tickets:
            assert srv.wait(t, 120000) == ns.OK
            done, tm = srv.poll(t)
            assert done and tm["status"] == ns.OK
            timings.append(tm)
        for (kt, ko, vt, vo) in bufs:
            outs.append((ko.cpu().numpy().view(np.uint32),
                         None if vo is None else vo.cpu().numpy().view(np.uint32)))
    return outs, timings


def test_mixed_stream_matches_oracle_and_is_the_same_alone(ns):
    reqs = make_requests(120, seed=1)
    mixed, tm = run_all(ns, reqs, streams=8, batch_max_keys=1 << 16)
    assert any(t["batched"] for t in tm) and not all(t["batched"] for t in tm)
    for (kind, dt, k, v), (ko, vo) in zip(reqs, mixed):
        if v is None:
            np.testing.assert_array_equal(ko, oracle.sort_keys(k, dt))
        else:
            wk, wv = oracle.sort_pairs(k, v, dt)
            np.testing.assert_array_equal(ko, wk)
            np.testing.assert_array_equal(vo, wv)
    alone, tm2 = run_all(ns, reqs, streams=1, batch_max_keys=0, sequential=True)
    assert not any(t["batched"] for t in tm2)
    for (a_k, a_v), (m_k, m_v) in zip(alone, mixed):
        np.testing.assert_array_equal(a_k, m_k)
        if a_v is not None:
            np.testing.assert_array_equal(a_v, m_v)


def test_admission_waits_for_memory(ns):
    n = 1 << 20
    need = ns.nsort_temp_bytes(ns.KIND_KEYS, n)
    reqs = [("keys", "u32", inputs.keys(n, "u32", "uniform", seed=s), None) for s in range(4)]
    outs, tm = run_all(ns, reqs, streams=4, batch_max_keys=0, budget=need + 4096)
    for (kind, dt, k, v), (ko, _) in zip(reqs, outs):
        np.testing.assert_array_equal(ko, oracle.sort_keys(k, dt))
    tm = sorted(tm, key=lambda t: t["t_admit"])
    for a, b in zip(tm, tm[1:]):
        assert b["t_admit"] >= a["t_done"] - 1e-3       # one request's scratch at a time


def test_error_paths(ns):
    with ns.SortServer(0, 1 << 20, 2, 0) as srv:
        x = torch.zeros(1 << 22, dtype=torch.int32, device="cuda")
        with pytest.raises(ns.NsortError) as e:            # scratch larger than the budget
            srv.submit(x, x)
        assert e.value.status == ns.ENOMEM
        with pytest.raises(ns.NsortError) as e:
            srv.poll(12345)
        assert e.value.status == ns.ENOTFOUND
        assert srv.wait(12345, 10) == ns.ENOTFOUND
        t = srv.submit(x[:0], x[:0])                        # n = 0 completes at once
        assert srv.poll(t)[0]


def test_admitted_requests_overlap_and_match_alone(ns):
    """Continuous batching admits a request while others are on the GPU: a
    large request and one just below the size from which requests run one
    at a time, on different stream slots and submitted back to back, are
    both admitted before either completes (their admit-to-done intervals
    overlap), and each result equals the oracle's."""
    big, small = 1 << 26, ns.SERVE_LARGE_MIN_KEYS - 1
    reqs = [("keys", "u32", inputs.keys(big, "u32", "uniform", seed=31), None),
            ("keys", "f32", inputs.keys(small, "f32", "zipf", seed=32), None)]
    budget = ns.nsort_temp_bytes(ns.KIND_KEYS, big) + ns.nsort_temp_bytes(ns.KIND_KEYS, small) \
        + (1 << 20)
    outs, tm = run_all(ns, reqs, streams=2, batch_max_keys=0, budget=budget)
    assert not any(t["batched"] for t in tm)
    assert max(t["t_admit"] for t in tm) < min(t["t_done"] for t in tm)
    for (kind, dt, k, v), (ko, _) in zip(reqs, outs):
        np.testing.assert_array_equal(ko, oracle.sort_keys(k, dt))


def test_large_requests_run_one_at_a_time(ns):
    """Requests of at least SERVE_LARGE_MIN_KEYS keys fill the GPU by
    themselves and run one at a time, in arrival order, even with free
    slots and memory: the next one is enqueued behind the running one.  The
    second request here reads the first one's output as its input, so it
    returns the oracle's result only if it ran after the first completed;
    a smaller request submitted last still runs beside them."""
    n = 1 << 23
    x = torch.from_numpy(inputs.keys(n, "u32", "uniform", seed=33).view(np.int32)).cuda()
    y, z = torch.empty_like(x), torch.empty_like(x)
    m = ns.SERVE_LARGE_MIN_KEYS // 4
    small = inputs.keys(m, "f32", "dup16", seed=34)
    s_in = torch.from_numpy(small.view(np.int32)).cuda()
    s_out = torch.empty_like(s_in)
    budget = 3 * ns.nsort_temp_bytes(ns.KIND_KEYS, n) + (1 << 20)
    with ns.SortServer(0, budget, 4, 0) as srv:
        torch.cuda.synchronize()
        t1 = srv.submit(x, y, n=n, dtype=DT["u32"])
        t2 = srv.submit(y, z, n=n, dtype=DT["u32"])
        t3 = srv.submit(s_in, s_out, n=m, dtype=DT["f32"])
        tms = []
        for t in (t1, t2, t3):
            assert srv.wait(t, 120000) == ns.OK
            done, tm = srv.poll(t)
            assert done and tm["status"] == ns.OK
            tms.append(tm)
    want = oracle.sort_keys(x.cpu().numpy().view(np.uint32), "u32")
    np.testing.assert_array_equal(y.cpu().numpy().view(np.uint32), want)
    np.testing.assert_array_equal(z.cpu().numpy().view(np.uint32), want)
    np.testing.assert_array_equal(s_out.cpu().numpy().view(np.uint32), oracle.sort_keys(small, "f32"))
    assert tms[0]["t_done"] <= tms[1]["t_done"]
    # the smaller request was admitted before the second large one completed
    assert tms[2]["t_admit"] < tms[1]["t_done"]
