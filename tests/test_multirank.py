"""The benchmark's multi-rank bookkeeping on CPU ranks (gloo, world size 2):
the job's time is the slowest rank's, the job's throughput counts every
rank's units, and under a multi-rank launch only rank 0 runs the oracle
arm.  (One GPU per process; every rank runs its own replica of the step.)"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) s on the device and 2 (r + 1) s end to end for 10 steps
        value, e2e, t_max = bench.job_rates(10, world, 1.0 * (rank + 1), 2.0 * (rank + 1), dist, "cpu")
        q.put((rank, value, e2e, t_max))
    finally:
        dist.destroy_process_group()


def test_job_rates_take_the_slowest_rank_over_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, value, e2e, t_max in out:
        assert t_max == 2.0                 # the slowest rank's device time, on every rank
        assert value == pytest.approx(2 * 10 / 2.0)
        assert e2e == pytest.approx(2 * 10 / 4.0)


def test_single_process_rates():
    value, e2e, t_max = bench.job_rates(5, 1, 0.5, 1.0)
    assert (value, e2e, t_max) == (10.0, 5.0, 0.5)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, gpus = 1, 0, 2

    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""
