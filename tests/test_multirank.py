"""Multi-rank host logic of the bench on CPU (gloo, world size 2).

Each rank transforms its own replica (weak scaling, no data-path
collective); the only collectives are the barrier and the max-over-ranks
reduction of the step time, which these tests run with the gloo backend."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(dist, 1.5 + rank, "cpu")  # rank 1 is the slow one
    value = bench.job_gflops(world, 8.0e9, ms)
    dist.barrier()
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in results:
        assert ms == 2.5  # every rank reports the slowest rank's time
        assert abs(value - 2 * 8.0e9 / 2.5e-3 / 1e9) < 1e-6


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(argparse.Namespace(steps=1, warmup=0)) == 0
    assert capsys.readouterr().out == ""
