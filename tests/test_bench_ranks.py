"""Host logic of bench.py's multi-rank run, on CPU: two gloo ranks agree on the slowest
rank's time, the whole-job rate counts every rank's units, and only rank 0 of the
reference arm prints."""
import io
import os
import socket
import sys
import contextlib

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = bench.max_over_ranks(times[rank], dist)
    dist.barrier()
    q.put((rank, got, bench.whole_job_rate(1_000_000_000, world, 2, got * 1e3)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [0.5, 2.0]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.0, 2.0]
    # 2 ranks x 2 steps x 1 G units in 2 s: 2 G units/s
    assert all(abs(o[2] - 2.0) < 1e-12 for o in out)


def test_single_process_helpers():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert abs(bench.whole_job_rate(2_400_000_000, 1, 20, 1353.2) - 2.4e9 * 20 / 1.3532 / 1e9) < 1e-9


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(argparse.Namespace(workload=bench.DEFAULT_WORKLOAD, gpus=2, steps=1, warmup=0))
    assert buf.getvalue() == ""
