"""hfx_plan_autotune: it times the first product's Y-ring shapes, the item
order and the row tiles per CTA of the Y build and the Q2 GEMM, keeps the
fastest, and leaves the results unchanged (the candidates differ only in
launch shape; the order of FP64 atomic additions is the only difference)."""
import os

import numpy as np
import pytest

from paper_2412_11081_gb300 import hfx, inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def two_species():
    rng = np.random.default_rng(11)
    pos = np.array([[0.0, 0.0, 0.0], [1.7, 1.7, 0.0], [1.7, 0.0, 1.7], [0.0, 1.7, 1.7]]) + rng.normal(0, 0.05, (4, 3))
    w = inputs.tiny_model([5, 9], [14, 40], [0, 1, 0, 1], np.eye(3) * 3.4, pos, r_c=2.3, seed=13)
    return inputs.cut_density(w, 4.5)


@pytest.mark.parametrize("prec", [hfx.HFX_BF16X6, hfx.HFX_BF16X3])
@pytest.mark.parametrize("case", ["si8", "two_species"])
def test_autotune_keeps_results_and_picks_the_fastest(case, prec):
    w = inputs.si_supercell(1) if case == "si8" else two_species()
    with hfx.Plan(w, precision=prec) as p:
        E0, F0, S0 = p.evaluate(w.lattice, w.positions)
        rep = p.autotune(w.lattice, w.positions, reps=2)
        assert rep["candidates"] >= 2
        assert 0 < rep["best_ms"] <= rep["default_ms"]
        assert rep["t1_rows_per_slot"] >= 1 and rep["t1_slots"] >= 2
        assert rep["t1_home_order"] in (0, 1, 2)
        assert rep["y_tiles_per_cta"] in (1, 2) and rep["q2_tiles_per_cta"] in (1, 2, 3)
        assert rep["candidates"] >= 4   # ring shapes, item order, two tile counts
        E1, F1, S1 = p.evaluate(w.lattice, w.positions)
    assert abs(E1 - E0) <= 1e-12 * abs(E0) and rel(F1, F0) <= 1e-12 and rel(S1, S0) <= 1e-12


@pytest.mark.parametrize("prec", [hfx.HFX_BF16X6, hfx.HFX_BF16X3])
@pytest.mark.parametrize("case", ["si8", "two_species"])
@pytest.mark.parametrize("shape", ["1", "3"])
def test_one_row_tile_per_cta_equals_two(case, prec, shape, monkeypatch):
    """The Y build and the Q2 GEMM with one 128-row tile per CTA (more stages,
    two accumulators), and the Q2 GEMM with two tiles in one CTA per SM and
    a deeper pipeline (shape 3), give the results of two tiles per CTA: each tile runs
    the same K steps in the same order."""
    w = inputs.si_supercell(1) if case == "si8" else two_species()
    with hfx.Plan(w, precision=prec) as p:
        ref = p.evaluate(w.lattice, w.positions)
    monkeypatch.setenv("HFX_Y_TILES", "1")
    monkeypatch.setenv("HFX_Q2_TILES", shape)
    with hfx.Plan(w, precision=prec) as p:
        got = p.evaluate(w.lattice, w.positions)
        rep = p.autotune(w.lattice, w.positions, reps=1)
        assert rep["y_tiles_per_cta"] in (1, 2) and rep["q2_tiles_per_cta"] in (1, 2, 3)
    assert abs(got[0] - ref[0]) <= 1e-12 * abs(ref[0])
    assert rel(got[1], ref[1]) <= 1e-12 and rel(got[2], ref[2]) <= 1e-12


def test_autotune_without_tunable_kernel_and_bad_arguments():
    w = inputs.diamond8()
    with hfx.Plan(w, precision=hfx.HFX_FP64) as p:
        assert p.autotune(w.lattice, w.positions, reps=1)["candidates"] == 0
        with pytest.raises(hfx.HfxError) as ei:
            p.autotune(w.lattice, w.positions, reps=0)
        assert ei.value.status == 1
