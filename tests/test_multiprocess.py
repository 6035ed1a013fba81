"""The multi-process (N > 1) host logic of the benchmark on CPU: two gloo ranks.

`bench.py --gpus N` runs one independent CipherTensor per rank (weak scaling,
no collective on the data path); the only cross-rank steps are the barrier,
the max over ranks of each timed region and the whole-job throughput, and
only rank 0 prints (the reference arm runs on rank 0 alone).
"""
import contextlib
import importlib.util
import io
import os
import socket
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        dist.barrier()
        ms = b.max_over_ranks(times[rank], dist, "cpu")
        out.put((rank, ms, b.job_throughput(world, 64, 20, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_units():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [10.0, 12.5]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 12.5                            # the slowest rank bounds the job
        assert value == pytest.approx(2 * 64 * 20 / 12.5e-3)  # both ranks' pairs over that time


def test_single_process_needs_no_collective():
    b = _bench()
    assert b.max_over_ranks(7.0, None, "cpu") == 7.0
    assert b.job_throughput(1, 64, 20, 500.0) == pytest.approx(64 * 20 / 0.5)


def test_reference_arm_runs_on_rank_zero_only():
    b = _bench()
    old = os.environ.get("RANK")
    os.environ["RANK"] = "1"
    try:
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            assert b.run_reference(types.SimpleNamespace(steps=1, warmup=0, gpus=2)) is None
        assert buf.getvalue() == ""  # no work, no line: rank 0 prints the job's line
    finally:
        if old is None:
            del os.environ["RANK"]
        else:
            os.environ["RANK"] = old
