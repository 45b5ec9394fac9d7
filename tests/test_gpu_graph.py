"""CUDA-graph replay of a frozen plan (hfx_options.graph).

With frozen pair lists and screening decisions (freeze_lists), every call
after the first is a fixed sequence of launches whose inputs (positions and
lattice) sit in device memory: the second call records it into a CUDA graph
and later calls launch the graph.  Replayed results must equal those of a
plan that launches every kernel, at new positions and a new (strained)
lattice alike, in both precisions.
"""
import numpy as np
import pytest

from paper_2412_11081_gb300 import hfx, inputs

pytestmark = pytest.mark.gpu


def rel(a, ref):
    a, ref = np.asarray(a, float), np.asarray(ref, float)
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


def geometries(w, n=4):
    out = [(w.lattice, g) for g in inputs.geometry_sequence(w, n, seed=5, amp=0.005)]
    eps = np.array([[2e-4, 1e-4, 0.0], [1e-4, -1e-4, 0.0], [0.0, 0.0, 1.5e-4]])
    Fm = np.eye(3) + eps
    out.append((w.lattice @ Fm.T, w.positions @ Fm.T))   # a strained cell, within the skin
    return out


@pytest.mark.parametrize("prec", [hfx.HFX_FP64, hfx.HFX_BF16X6])
@pytest.mark.parametrize("case", ["diamond8", "si8_passes"])
def test_graph_replay_equals_direct_launches(prec, case):
    w = inputs.diamond8() if case == "diamond8" else inputs.si_supercell(1)
    chunk = 3 if case == "si8_passes" else 0
    geo = geometries(w)
    with hfx.Plan(w, precision=prec, freeze_lists=True, home_chunk=chunk) as p:
        ref = [p.evaluate(L, x) for L, x in geo]
    replayed = []
    with hfx.Plan(w, precision=prec, freeze_lists=True, home_chunk=chunk, graph=True) as p:
        got = []
        for L, x in geo:
            got.append(p.evaluate(L, x, stats=True))
            replayed.append(p.stats.graph_replayed)
        # per-stage timing evaluates without the graph, with the same result
        p.set_timing(True)
        timed = p.evaluate(*geo[1], stats=True)
        assert p.stats.graph_replayed == 0 and p.stats.ms_total > 0
        p.set_timing(False)
        again = p.evaluate(*geo[1], stats=True)
        assert p.stats.graph_replayed == 1 and p.stats.kernel_launches > 0
    assert replayed == [0] + [1] * (len(geo) - 1)
    for (E, F, S), (E0, F0, S0) in zip(got, ref):
        assert abs(E - E0) <= 1e-12 * abs(E0) and rel(F, F0) <= 1e-12 and rel(S, S0) <= 1e-12
    for res in (timed, again):
        assert abs(res[0] - ref[1][0]) <= 1e-12 * abs(ref[1][0]) and rel(res[1], ref[1][1]) <= 1e-12


def test_graph_needs_a_frozen_plan():
    """Without frozen lists every call may re-screen, so nothing is recorded."""
    w = inputs.diamond8()
    with hfx.Plan(w, graph=True) as p:
        for _ in range(3):
            p.evaluate(w.lattice, w.positions, stats=True)
            assert p.stats.graph_replayed == 0
