"""hfx_energy_force_stress_noalloc against hfx_energy_force_stress, through the C ABI.

The no-allocation entry point serves callers that cannot allocate device
memory while they evaluate: hosts whose device memory belongs to their own
pool after start-up, and real-time loops that forbid allocation after
initialisation.  Its per-call scratch is a fixed 64 MiB array inside the
library instead of plan buffers grown with cudaMalloc.  This file is
collected last, so a run that stops at its first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2412_11081_gb300 import hfx, inputs

pytestmark = pytest.mark.gpu
TOL = 1e-10   # the FP64 parity tolerance of the other GPU tests


def rel(a, ref):
    a, ref = np.asarray(a, float), np.asarray(ref, float)
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


def assert_same(got, ref):
    assert abs(got[0] - ref[0]) <= TOL * abs(ref[0])
    assert rel(got[1], ref[1]) <= TOL
    assert rel(got[2], ref[2]) <= TOL


def workload():
    # 8-atom diamond cell with D cut at 10 A: its Y and V blocks fit the array
    return inputs.cut_density(inputs.diamond8(), 10.0)


def test_noalloc_matches_allocating_entry_point_two_calls_in_a_row():
    w = workload()
    with hfx.Plan(w) as p:
        ref = p.evaluate(w.lattice, w.positions)
        first = p.evaluate_noalloc(w.lattice, w.positions)
        second = p.evaluate_noalloc(w.lattice, w.positions)
        assert_same(first, ref)
        assert_same(second, ref)
        # a moved geometry (within the skin): both entry points again
        q = w.positions + np.random.default_rng(2).normal(0.0, 0.02, w.positions.shape)
        ref2 = p.evaluate(w.lattice, q)
        assert_same(p.evaluate_noalloc(w.lattice, q), ref2)
        assert_same(p.evaluate_noalloc(w.lattice, q), ref2)


def test_noalloc_as_the_first_call_of_a_plan():
    w = workload()
    with hfx.Plan(w) as p:
        got = [p.evaluate_noalloc(w.lattice, w.positions) for _ in range(2)]
        ref = p.evaluate(w.lattice, w.positions)
    for g in got:
        assert_same(g, ref)


def test_noalloc_rejects_work_beyond_the_array_and_plan_stays_usable():
    w = inputs.si_supercell(1)   # 8 atoms, n_ao 13, n_abf 50: Y blocks need far more than 64 MiB
    with hfx.Plan(w) as p:
        with pytest.raises(hfx.HfxError) as ei:
            p.evaluate_noalloc(w.lattice, w.positions)
        assert ei.value.status == 6 and "scratch" in str(ei.value)
        E, F, S = p.evaluate(w.lattice, w.positions)
        assert np.isfinite(E)


def test_noalloc_refuses_split_precision_plans():
    w = workload()
    with hfx.Plan(w, precision=hfx.HFX_BF16X6) as p:
        with pytest.raises(hfx.HfxError) as ei:
            p.evaluate_noalloc(w.lattice, w.positions)
        assert ei.value.status == 6


def test_noalloc_calls_no_allocation_hook():
    """With counting hooks in hfx_options, the entry point neither allocates
    nor frees (the allocating entry point, by contrast, grows its stores)."""
    torch = pytest.importorskip("torch")
    calls = {"alloc": 0, "free": 0}

    def alloc(n):
        calls["alloc"] += 1
        return int(torch.cuda.caching_allocator_alloc(n, 0, torch.cuda.current_stream()))

    def free(ptr, n):
        calls["free"] += 1
        torch.cuda.caching_allocator_delete(ptr)

    w = workload()
    with hfx.Plan(w, allocator=(alloc, free)) as p:
        made = calls["alloc"]
        assert made > 0
        got = [p.evaluate_noalloc(w.lattice, w.positions) for _ in range(2)]
        assert calls == {"alloc": made, "free": 0}
        ref = p.evaluate(w.lattice, w.positions)
        assert calls["alloc"] > made
    for g in got:
        assert_same(g, ref)


def test_noalloc_stale_pair_lists_are_refused_and_plan_stays_usable():
    """Atoms moved by skin/2 or more need new pair lists, which allocate: the
    entry point refuses with HFX_ERR_PAIRLIST_STALE and writes nothing; the
    allocating entry point rebuilds the lists, after which it runs again."""
    w = workload()
    with hfx.Plan(w, skin=0.5) as p:
        p.evaluate_noalloc(w.lattice, w.positions)
        q = w.positions.copy()
        q[3] += np.array([0.3, 0.0, 0.0])   # 0.3 A >= skin / 2
        with pytest.raises(hfx.HfxError) as ei:
            p.evaluate_noalloc(w.lattice, q)
        assert ei.value.status == 5
        ref = p.evaluate(w.lattice, q)
        assert_same(p.evaluate_noalloc(w.lattice, q), ref)
