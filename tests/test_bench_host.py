"""Host-side rules of bench.py, checked without a GPU: the measured peak and
its fallback, the roofline traffic that must go null once the kernel's
sources change after the counters were taken, and the defaults (one GPU, at
least three warm-up steps, the 2^28-key workload)."""
import importlib.util
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture()
def bench():
    spec = importlib.util.spec_from_file_location("bench_host", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_defaults_are_one_gpu_full_workload_with_three_warmups(bench, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.impl == "nsort" and a.log2n == 28 and a.dtype == "u32"
    assert a.warmup >= 3 and a.steps >= 1


def test_peak_from_measured_file_else_fallback(bench, tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_peaks() == {"hbm_gbs": 6800.0, "source": "fallback"}
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6678.5, "bf16_tflops": 1}))
    assert bench.load_peaks() == {"hbm_gbs": 6678.5, "source": "measured"}


def test_committed_traffic_is_plausible(bench):
    """Each committed figure is the DRAM bytes read and written by one merge
    launch at the n it was captured at: each at most the algorithmic read
    (or write) of that n plus a few percent, and above zero.  It names the
    profile it came from and the sources its hash covers."""
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for kernel, word in (("merge_keys", 4),):
        t = d[kernel]
        n = t["captured_n"]
        assert 0 < t["read_bytes"] <= word * n * 1.05
        assert 0 < t["write_bytes"] <= word * n * 1.05
        assert os.path.exists(os.path.join(ROOT, t["profile"]))
        assert all(os.path.exists(os.path.join(ROOT, f)) for f in t["sources"])


def test_traffic_goes_null_when_a_source_changes(bench, tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("int a = 1;  // version 1\n/* the kernel */\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    entry = {"captured_n": 1 << 28, "read_bytes": 1 << 30, "write_bytes": 1 << 30,
             "sources": ["kernel.cu"], "source_sha": bench.source_hash(["kernel.cu"])}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"merge_keys": entry}))
    assert bench.load_traffic("merge_keys")["read_bytes"] == 1 << 30
    assert bench.load_traffic("merge_pairs") is None
    # a comment edit leaves the code, and the counters, as they were
    src.write_text("int a = 1;  // version 2\n\n/* the kernel,\n   commented */\n")
    assert bench.load_traffic("merge_keys")["read_bytes"] == 1 << 30
    # a code edit does not
    src.write_text("int a = 2;  // version 2\n")
    assert bench.load_traffic("merge_keys") is None
