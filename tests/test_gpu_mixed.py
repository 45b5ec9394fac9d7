"""Split-precision path (bf16 pieces on the tensor cores, FP32 accumulation,
FP64 screening and reductions) against the FP64 CPU oracle.

Error metric: max|x - x_ref| / max|x_ref| per output (|dE|/|E| for E).
Every case is held to the 1e-5 relative contract.  HFX_BF16X6 keeps every
piece product down to 2^-24 of the operands and meets it everywhere.
HFX_BF16X3 drops the products below 2^-16 of them: it meets the contract on
the unperturbed cells, but not on the two-species cell (2.1e-5 in F from its
second product) nor on every jittered si64 geometry (up to 1.8e-5 in sigma);
those cases are marked as expected failures (strict: they must keep
failing, so a change that brings BF16X3 within the contract shows up) and
print the error they measure.
"""
import json
import os

import numpy as np
import pytest

from oracle import evaluate
from paper_2412_11081_gb300 import hfx, inputs

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
SPLITS = [hfx.HFX_BF16X6, hfx.HFX_BF16X3]
BOUND = 1e-5   # the relative force/stress/energy contract of the split precisions
BF16X3_MISSES = pytest.mark.xfail(strict=True, reason="BF16X3 exceeds the 1e-5 contract here (two-piece operands)")


def rel(a, ref):
    a, ref = np.asarray(a, float), np.asarray(ref, float)
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


def run(w, prec, **kw):
    with hfx.Plan(w, precision=prec, **kw) as p:
        E, F, S = p.evaluate(w.lattice, w.positions, stats=True)
        return E, F, S, p.stats.as_dict()


def tiny_periodic(seed=7):
    rng = np.random.default_rng(seed)
    pos = np.array([[0.1, 0.2, 0.0], [1.5, 1.7, 1.4]]) + rng.normal(0, 0.05, (2, 3))
    w = inputs.tiny_model([2, 3], [3, 4], [0, 1], np.eye(3) * 3.2, pos, r_c=1.3, seed=seed)
    return inputs.cut_density(w, 3.5)


@pytest.mark.parametrize("prec", SPLITS)
@pytest.mark.parametrize("case", ["tiny", "diamond8"])
def test_mixed_small_cells(case, prec):
    w = tiny_periodic() if case == "tiny" else inputs.diamond8()
    r = evaluate(w)
    E, F, S, st = run(w, prec)
    b = BOUND
    assert abs(E - r.E) <= b * abs(r.E)
    assert rel(F, r.F) <= b, rel(F, r.F)
    assert rel(S, r.sigma) <= b, rel(S, r.sigma)
    # screening is FP64 on both sides: the same items are contracted
    assert st["triplets"] == r.counts["triplets"] and st["term2_pairs"] == r.counts["term2_pairs"]


def two_species_cell(seed=13):
    """Four atoms of two species with different block shapes (n_ao 5 / 9,
    n_abf 14 / 40): consecutive B of one item change n_abf(B) and the items
    change n_ao(F), which the tcgen05 first product pads per B."""
    rng = np.random.default_rng(11)
    pos = np.array([[0.0, 0.0, 0.0], [1.7, 1.7, 0.0], [1.7, 0.0, 1.7], [0.0, 1.7, 1.7]]) + rng.normal(0, 0.05, (4, 3))
    w = inputs.tiny_model([5, 9], [14, 40], [0, 1, 0, 1], np.eye(3) * 3.4, pos, r_c=2.3, seed=seed)
    return inputs.cut_density(w, 4.5)


@pytest.mark.parametrize("prec", [hfx.HFX_BF16X6, pytest.param(hfx.HFX_BF16X3, marks=BF16X3_MISSES)])
def test_mixed_two_species_shapes(prec):
    """BF16X6 meets 1e-5 here too.  BF16X3 does not on this cell: its
    second product (R2 and Z from two-piece Y, the 2^-16 piece product
    dropped) leaves about 2e-5 in F on its own."""
    w = two_species_cell()
    r = evaluate(w)
    E, F, S, st = run(w, prec)
    eE, eF, eS = abs(E - r.E) / abs(r.E), rel(F, r.F), rel(S, r.sigma)
    print(f"two-species cell, precision {prec}: errE {eE:.2e} errF {eF:.2e} errS {eS:.2e}")
    assert st["triplets"] == r.counts["triplets"] and st["term2_pairs"] == r.counts["term2_pairs"]
    assert eE <= BOUND and eF <= BOUND and eS <= BOUND


@pytest.mark.parametrize("prec", SPLITS)
def test_mixed_si64_full_size(prec):
    """The 64-atom Si-like supercell of the benchmark against the stored oracle."""
    ref = json.load(open(os.path.join(HERE, "golden", "si64_oracle.json")))
    w = inputs.si_supercell(2)
    E, F, S, st = run(w, prec)
    b = BOUND
    eF, eS, eE = rel(F, ref["F"]), rel(S, ref["sigma"]), abs(E - ref["E"]) / abs(ref["E"])
    print(f"precision {prec}: errE {eE:.2e} errF {eF:.2e} errS {eS:.2e}")
    assert eE <= b and eF <= b and eS <= b
    assert st["triplets"] == ref["counts"]["triplets"]


@pytest.mark.parametrize("prec", [hfx.HFX_BF16X6, pytest.param(hfx.HFX_BF16X3, marks=BF16X3_MISSES)])
def test_split_precisions_on_jittered_si64_geometries(prec):
    """The first four geometries of the benchmark's jittered si64 sequence,
    against the FP64 GPU path (itself within 1e-10 of the oracle).  BF16X6
    stays within 1e-5 on each.  BF16X3 reaches about 1.8e-5 in sigma on some
    of them (its two-piece operands leave 2^-16-level errors in both
    exchange products); the benchmark takes it as its headline only where it
    meets 1e-5 on these geometries."""
    w = inputs.si_supercell(2)
    geoms = inputs.geometry_sequence(w, 4)
    with hfx.Plan(w, precision=hfx.HFX_FP64) as p0:
        refs = [p0.evaluate(w.lattice, g) for g in geoms]
    worst = 0.0
    with hfx.Plan(w, precision=prec) as p:
        for k, g in enumerate(geoms):
            E, F, S = p.evaluate(w.lattice, g)
            E0, F0, S0 = refs[k]
            eE, eF, eS = abs(E - E0) / abs(E0), rel(F, F0), rel(S, S0)
            print(f"precision {prec} geometry {k}: errE {eE:.2e} errF {eF:.2e} errS {eS:.2e}")
            worst = max(worst, eE, eF, eS)
    assert worst <= BOUND, worst


def test_mixed_anisotropic_gradient_blocks():
    w = tiny_periodic(seed=9)
    rng = np.random.default_rng(4)
    Gp = [rng.standard_normal(g.shape) for g in w.G]
    e = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    import dataclasses
    from oracle import Options
    r = evaluate(w, dataclasses.replace(Options.from_theta(w.theta), aniso=(Gp, e)))
    E, F, S, _ = run(w, hfx.HFX_BF16X6, aniso=(Gp, e))
    assert rel(F, r.F) <= 1e-5 and rel(S, r.sigma) <= 1e-5


def test_mixed_each_exchange_product_alone():
    w = tiny_periodic(seed=3)
    import dataclasses
    from oracle import Options
    for terms in (1, 2):
        r = evaluate(w, dataclasses.replace(Options.from_theta(w.theta), terms=terms))
        E, F, S, _ = run(w, hfx.HFX_BF16X6, terms=terms)
        assert abs(E - r.E) <= 1e-5 * abs(r.E)
        assert rel(F, r.F) <= 1e-5 and rel(S, r.sigma) <= 1e-5


@pytest.mark.parametrize("prec", SPLITS)
def test_first_product_kernels_agree(prec, monkeypatch):
    """The tcgen05 first product and the warp-level MMA one (selected at plan
    creation by HFX_T1_KERNEL) on the same cell: both within the contract of
    the oracle."""
    w = inputs.diamond8()
    r = evaluate(w)
    for kern in ("umma", "mma"):
        monkeypatch.setenv("HFX_T1_KERNEL", kern)
        E, F, S, _ = run(w, prec)
        eE, eF, eS = abs(E - r.E) / abs(r.E), rel(F, r.F), rel(S, r.sigma)
        print(f"first product {kern}, precision {prec}: errE {eE:.2e} errF {eF:.2e} errS {eS:.2e}")
        assert eE <= BOUND and eF <= BOUND and eS <= BOUND, kern


def test_auxiliary_basis_beyond_tcgen05_kernel(monkeypatch):
    """n_abf = 66/70 (> 64 rows of the tcgen05 tiles): the plan takes the
    warp-level MMA first product; forcing the tcgen05 kernel is rejected."""
    rng = np.random.default_rng(21)
    pos = np.array([[0.1, 0.2, 0.0], [1.5, 1.7, 1.4]]) + rng.normal(0, 0.05, (2, 3))
    w = inputs.cut_density(inputs.tiny_model([3, 4], [66, 70], [0, 1], np.eye(3) * 3.2, pos, r_c=1.3, seed=21), 3.5)
    r = evaluate(w)
    E, F, S, _ = run(w, hfx.HFX_BF16X6)
    assert abs(E - r.E) <= 1e-5 * abs(r.E) and rel(F, r.F) <= 1e-5 and rel(S, r.sigma) <= 1e-5
    monkeypatch.setenv("HFX_T1_KERNEL", "umma")
    with pytest.raises(hfx.HfxError) as ei:
        run(w, hfx.HFX_BF16X6)
    assert ei.value.status == 6


@pytest.mark.parametrize("prec", SPLITS)
def test_mixed_everything_screened_out(prec):
    """No kept pair, triplet or term-2 pair: every split kernel sees empty
    lists and the result is exactly zero."""
    w = tiny_periodic()
    th = dict(C=1e30, dC=1e30, V=1e30, dV=1e30, D=1e30, CS=1e30)
    with hfx.Plan(w, precision=prec, theta=th) as p:
        E, F, S = p.evaluate(w.lattice, w.positions, stats=True)
        st = p.stats.as_dict()
    assert E == 0.0 and not np.asarray(F).any() and not np.asarray(S).any()
    assert st["triplets"] == 0 and st["term2_pairs"] == 0


@pytest.mark.parametrize("prec", SPLITS)
def test_mixed_single_atom_cell_self_images_only(prec):
    """One atom per cell: every pair is a self-image, F = 0 to rounding and
    E, sigma within the split's bound of the oracle."""
    w = inputs.cut_density(inputs.tiny_model([3], [5], [0], np.eye(3) * 2.9, np.array([[0.2, 0.1, 0.3]]),
                                             r_c=1.6, seed=5), 6.0)
    r = evaluate(w)
    E, F, S, _ = run(w, prec)
    assert np.max(np.abs(F)) <= 1e-10 * abs(r.E)
    assert abs(E - r.E) <= BOUND * abs(r.E) and rel(S, r.sigma) <= BOUND
