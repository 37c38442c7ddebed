"""The multi-process path of bench.py on CPU: two ranks over gloo.

With N > 1 every rank sorts its own array (replicas, no data-path
collective); the step time is the max over ranks, the value counts the keys
of all ranks, and only rank 0 runs the CPU reference arm and prints.  These
tests drive that host logic with world_size 2 over the gloo backend on
127.0.0.1, without a GPU."""
import importlib.util
import io
import multiprocessing as mp
import os
import socket
import types
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, local_ms, n, out):
    import torch.distributed as dist
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        bench = load_bench()
        assert bench.dist_env() == (rank, rank, world)
        bench.barrier(world)
        ms, value = bench.replica_throughput(local_ms[rank], n, world, device="cpu")
        bench.barrier(world)
        # the reference arm: rank 0 alone runs it; the others return at once
        args = types.SimpleNamespace(dtype="u32", warmup=0, steps=1, gpus=world, log2n=12)
        buf = io.StringIO()
        if rank != 0:
            with redirect_stdout(buf):
                bench.run_reference(args, rank, world)
        out.put((rank, ms, value, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def run_ranks(world, local_ms, n):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, world, port, local_ms, n, q))
             for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(got)


def test_two_ranks_take_the_slowest_time_and_count_all_keys():
    n = 1 << 28
    got = run_ranks(2, [6.5, 7.25], n)
    for rank, ms, value, printed in got:
        assert ms == 7.25                                  # max over ranks
        assert value == pytest.approx(2 * n / 7.25e-3 / 1e9)
        assert printed == ""                               # rank 1 printed nothing


def test_single_rank_needs_no_process_group():
    bench = load_bench()
    ms, value = bench.replica_throughput(4.0, 1000, 1, device="cpu")
    assert ms == 4.0 and value == pytest.approx(1000 / 4e-3 / 1e9)
