"""Host logic of the multi-rank bench path on CPU: two gloo ranks with
different timed regions agree on the slowest time and on the whole-job value;
the reference arm's extra ranks exit without work."""
import argparse
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        value, ms_max = bench.replica_throughput(10.0 + 5.0 * rank, cells=1000, steps=4, dist=dist)
        out.put((rank, value, ms_max))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms_max in res:
        assert ms_max == 15.0
        assert value == pytest.approx(1000 * 4 * 2 / 0.015)


def test_single_process_value():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.replica_throughput(20.0, cells=1000, steps=4)
    assert ms == 20.0 and value == pytest.approx(1000 * 4 / 0.020)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(gpus=2, steps=1, warmup=1)
    assert bench.run_reference(args) == 0
