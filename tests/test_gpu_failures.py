"""Failure detection without a GPU fault.

* Allocation failures: a plan whose allocation hook (hfx_options alloc /
  free) refuses memory reports HFX_ERR_OOM, gives back everything it took,
  and a plan whose per-call store cannot grow stays usable once memory is
  available again.
* Bounded waits: the tensor-core pipelines wait on mbarriers with a limit of
  one second of wall time.  The test-only switch
  HFX_TEST_STALL_Q2_PRODUCER=1 keeps the second product's producer warp from
  issuing its copies, so the consumers' waits run out; the call must return
  HFX_ERR_TIMEOUT (no trap, no hang) and the same plan must evaluate
  correctly afterwards.
"""
import numpy as np
import pytest

from paper_2412_11081_gb300 import hfx, inputs

pytestmark = pytest.mark.gpu


def rel(a, ref):
    a, ref = np.asarray(a, float), np.asarray(ref, float)
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


class CountingAllocator:
    """Device memory from PyTorch's caching allocator, with a budget of
    allocations after which it refuses (returns 0)."""

    def __init__(self, budget=10 ** 9):
        import torch
        self.torch = torch
        self.budget = budget
        self.live = {}
        self.allocs = 0
        self.frees = 0

    def alloc(self, n):
        if self.allocs >= self.budget:
            return 0
        self.allocs += 1
        p = self.torch.cuda.caching_allocator_alloc(n, 0, self.torch.cuda.current_stream())
        self.live[int(p)] = n
        return int(p)

    def free(self, p, n):
        self.frees += 1
        assert self.live.pop(p) == n
        self.torch.cuda.caching_allocator_delete(p)

    def hooks(self):
        return (self.alloc, self.free)


def test_plan_creation_out_of_memory_gives_back_what_it_took():
    pytest.importorskip("torch")
    w = inputs.diamond8()
    for budget in (0, 5, 30):
        a = CountingAllocator(budget)
        with pytest.raises(hfx.HfxError) as ei:
            hfx.Plan(w, allocator=a.hooks())
        assert ei.value.status == 2, (budget, ei.value)
        assert not a.live and a.frees == a.allocs, budget


def test_evaluation_out_of_memory_leaves_the_plan_usable():
    pytest.importorskip("torch")
    w = inputs.diamond8()
    a = CountingAllocator()
    with hfx.Plan(w, allocator=a.hooks()) as p:
        a.budget = a.allocs          # the per-call stores cannot grow any more
        with pytest.raises(hfx.HfxError) as ei:
            p.evaluate(w.lattice, w.positions)
        assert ei.value.status == 2
        a.budget = 10 ** 9
        E, F, S = p.evaluate(w.lattice, w.positions)
    with hfx.Plan(w) as q:
        ref = q.evaluate(w.lattice, w.positions)
    assert abs(E - ref[0]) <= 1e-12 * abs(ref[0]) and rel(F, ref[1]) <= 1e-12
    assert not a.live


@pytest.mark.parametrize("prec", [hfx.HFX_BF16X3, hfx.HFX_BF16X6])
def test_stalled_pipeline_wait_runs_out_and_plan_recovers(prec, monkeypatch):
    w = inputs.diamond8()
    with hfx.Plan(w, precision=prec) as p:
        ref = p.evaluate(w.lattice, w.positions)
        monkeypatch.setenv("HFX_TEST_STALL_Q2_PRODUCER", "1")
        with pytest.raises(hfx.HfxError) as ei:
            p.evaluate(w.lattice, w.positions)
        assert ei.value.status == 4, ei.value
        monkeypatch.delenv("HFX_TEST_STALL_Q2_PRODUCER")
        E, F, S = p.evaluate(w.lattice, w.positions)
    assert abs(E - ref[0]) <= 1e-12 * abs(ref[0]) and rel(F, ref[1]) <= 1e-12 and rel(S, ref[2]) <= 1e-12
