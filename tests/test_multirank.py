"""The multi-rank path on CPU ranks (gloo, world size 2): the benchmark's
bookkeeping (the job's time is the slowest rank's; only rank 0 runs the
oracle arm) and home-atom sharding (each rank's share of E, F and sigma,
summed by one all-reduce, gives the whole structure's result)."""
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
        # rank r took (r + 1) s on the device and 2 (r + 1) s end to end
        t_max, t_e2e = bench.max_over_ranks([1.0 * (rank + 1), 2.0 * (rank + 1)], dist, "cpu")
        q.put((rank, t_max, t_e2e))
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_ranks_over_gloo():
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
    for rank, t_max, t_e2e in out:
        assert (t_max, t_e2e) == (2.0, 4.0)   # the slowest rank's times, on every rank


def test_single_process_times():
    assert bench.max_over_ranks([0.5, 1.0]) == [0.5, 1.0]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, gpus = 1, 0, 2

    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""


# ---------------------------------------------------------------- sharding
class _SharePlan:
    """Stand-in for a plan over a home-atom range: per home atom A a pair
    gradient g_A on the pair (A, A+1), the share of E, F and sigma that the
    items of A give (F_A += g, F_(A+1) -= g, virial g (x) d), so that shares
    of disjoint ranges add up exactly as the library's do."""

    def __init__(self, w, home):
        self.n, self.home = w.n, home

    def evaluate(self, lattice, positions):
        import numpy as np
        E, F, W = 0.0, np.zeros((self.n, 3)), np.zeros((3, 3))
        for A in range(*self.home):
            g = np.array([A + 1.0, -0.5 * A, 0.25]) / self.n
            d = np.asarray(positions[(A + 1) % self.n]) - np.asarray(positions[A])
            E -= 1.0 / (A + 2.0)
            F[A] += g
            F[(A + 1) % self.n] -= g
            W += np.outer(g, d)
        return E, F, -W / 10.0

    def close(self):
        pass


def _shard_worker(rank, world, port, q):
    import numpy as np
    from paper_2412_11081_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pos = np.random.default_rng(0).normal(size=(7, 3))
        from types import SimpleNamespace
        with shard.ShardedPlan(SimpleNamespace(n=7, species=np.zeros(7)), rank, world,
                               plan_factory=lambda w, home: _SharePlan(w, home)) as sp:
            E, F, S = sp.evaluate(np.eye(3), pos)
            q.put((rank, sp.home, E, F.tolist(), S.tolist()))
    finally:
        dist.destroy_process_group()


def test_home_ranges_partition_the_atoms():
    from paper_2412_11081_gb300 import shard
    for n, world in ((7, 2), (1000, 8), (1080, 3), (5, 5)):
        r = shard.home_ranges(n, world)
        assert r[0][0] == 0 and r[-1][1] == n and all(a < b for a, b in r)
        assert all(r[k][1] == r[k + 1][0] for k in range(world - 1))
        assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1
    with pytest.raises(ValueError):
        shard.home_ranges(3, 4)


def test_sharded_shares_sum_to_the_whole_over_gloo():
    """Two CPU ranks, each with half of the home atoms: after the all-reduce
    both hold the single-process result."""
    import numpy as np
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    pos = np.random.default_rng(0).normal(size=(7, 3))
    from types import SimpleNamespace
    E0, F0, S0 = _SharePlan(SimpleNamespace(n=7), (0, 7)).evaluate(np.eye(3), pos)
    assert [o[1] for o in out] == [(0, 3), (3, 7)]
    for _, _, E, F, S in out:
        assert abs(E - E0) <= 1e-15 * abs(E0)
        assert np.allclose(F, F0, rtol=0, atol=1e-15) and np.allclose(S, S0, rtol=0, atol=1e-15)
