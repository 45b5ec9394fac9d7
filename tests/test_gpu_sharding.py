"""Home-atom sharding on the GPU: two processes share one GPU, each with a
plan over half of the home atoms (hfx_options home_begin / home_end), and a
gloo all-reduce of their shares gives the single-process E, F and sigma.
The processes never wait on each other inside a kernel: the only exchange
is the host-side all-reduce after both evaluations."""
import os
import socket

import numpy as np
import pytest

from paper_2412_11081_gb300 import hfx, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, prec, q):
    import torch.distributed as dist
    from paper_2412_11081_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        w = inputs.si_supercell(1)
        with shard.ShardedPlan(w, rank, world, precision=prec) as sp:
            E, F, S = sp.evaluate(w.lattice, w.positions)
            q.put((rank, sp.home, E, F, S))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("prec", [hfx.HFX_FP64, hfx.HFX_BF16X6])
def test_two_processes_each_with_half_the_home_atoms(prec):
    w = inputs.si_supercell(1)
    with hfx.Plan(w, precision=prec) as p:
        E0, F0, S0 = p.evaluate(w.lattice, w.positions)
    world, port = 2, _free_port()
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, prec, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in range(world)), key=lambda o: o[0])
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [(0, 4), (4, 8)]
    rel = lambda a, b: float(np.max(np.abs(np.asarray(a) - b)) / np.max(np.abs(b)))
    for _, _, E, F, S in out:
        assert abs(E - E0) <= 1e-12 * abs(E0)
        assert rel(F, F0) <= 1e-12 and rel(S, S0) <= 1e-12
