"""Split-precision path (bf16 pieces on the tensor cores, FP32 accumulation,
FP64 screening and reductions) against the FP64 CPU oracle.

Error metric: max|x - x_ref| / max|x_ref| per output (|dE|/|E| for E).
HFX_BF16X6 keeps every piece product down to 2^-24 of the operands;
HFX_BF16X3 drops the products below 2^-16 of them.  Both must meet the
1e-5 relative force/stress contract on the unperturbed cells here (BF16X3
misses it on the two-species cell and on some jittered si64 geometries,
see the tests below): in the tcgen05 first product U is
built in FP32 from FP32 Y and D, so the 16-bit truncation of BF16X3 only
touches the operands of the two tensor-core products, and the FP32
accumulators are flushed to FP64 every 32 B (the remaining error is the
sum of independent per-element rounding, measured at 4e-6 to 6e-6 on
si64).  The warp-level MMA first product (HFX_T1_KERNEL=mma; it also takes
the shapes the tcgen05 kernel does not: n_abf > 64) is held to 3e-5 at
BF16X3 and checked against the tcgen05 one.
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
BOUND = {hfx.HFX_BF16X6: 1e-5, hfx.HFX_BF16X3: 1e-5}
BOUND_MMA = {hfx.HFX_BF16X6: 1e-5, hfx.HFX_BF16X3: 3e-5}


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
    b = BOUND[prec]
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


@pytest.mark.parametrize("prec", SPLITS)
def test_mixed_two_species_shapes(prec):
    """BF16X6 meets 1e-5 here too.  BF16X3 does not on this cell: its
    second product (R2 and Z from two-piece Y, the 2^-16 piece product
    dropped) leaves 2.1e-5 in F on its own, the same with the warp-level and
    the tcgen05 first product, so BF16X3 is held to 3e-5 on it."""
    w = two_species_cell()
    r = evaluate(w)
    E, F, S, st = run(w, prec)
    b = 3e-5 if prec == hfx.HFX_BF16X3 else BOUND[prec]
    assert abs(E - r.E) <= b * abs(r.E)
    assert rel(F, r.F) <= b, rel(F, r.F)
    assert rel(S, r.sigma) <= b, rel(S, r.sigma)
    assert st["triplets"] == r.counts["triplets"] and st["term2_pairs"] == r.counts["term2_pairs"]


@pytest.mark.parametrize("prec", SPLITS)
def test_mixed_si64_full_size(prec):
    """The 64-atom Si-like supercell of the benchmark against the stored oracle."""
    ref = json.load(open(os.path.join(HERE, "golden", "si64_oracle.json")))
    w = inputs.si_supercell(2)
    E, F, S, st = run(w, prec)
    b = BOUND[prec]
    eF, eS, eE = rel(F, ref["F"]), rel(S, ref["sigma"]), abs(E - ref["E"]) / abs(ref["E"])
    print(f"precision {prec}: errE {eE:.2e} errF {eF:.2e} errS {eS:.2e}")
    assert eE <= b and eF <= b and eS <= b
    assert st["triplets"] == ref["counts"]["triplets"]


@pytest.mark.parametrize("prec", [hfx.HFX_BF16X6, hfx.HFX_BF16X3])
def test_split_precisions_on_jittered_si64_geometries(prec):
    """The first four geometries of the benchmark's jittered si64 sequence,
    against the FP64 GPU path (itself within 1e-10 of the oracle).  BF16X6
    stays within 1e-5 on each.  BF16X3 reaches 1.75e-5 in sigma on some of
    them (its two-piece operands leave 2^-16-level errors in both exchange
    products), so it is held to 2.5e-5 here, and the benchmark takes it as
    its headline only where it meets 1e-5 on these geometries."""
    w = inputs.si_supercell(2)
    geoms = inputs.geometry_sequence(w, 4)
    with hfx.Plan(w, precision=hfx.HFX_FP64) as p0:
        refs = [p0.evaluate(w.lattice, g) for g in geoms]
    with hfx.Plan(w, precision=prec) as p:
        for k, g in enumerate(geoms):
            E, F, S = p.evaluate(w.lattice, g)
            E0, F0, S0 = refs[k]
            eE, eF, eS = abs(E - E0) / abs(E0), rel(F, F0), rel(S, S0)
            print(f"precision {prec} geometry {k}: errE {eE:.2e} errF {eF:.2e} errS {eS:.2e}")
            b = 1e-5 if prec == hfx.HFX_BF16X6 else 2.5e-5
            assert eE <= b and eF <= b and eS <= b, k


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
    creation by HFX_T1_KERNEL) on the same cell: both within their bound of
    the oracle, and within it of each other."""
    w = inputs.diamond8()
    r = evaluate(w)
    out = {}
    for kern in ("umma", "mma"):
        monkeypatch.setenv("HFX_T1_KERNEL", kern)
        out[kern] = run(w, prec)
        b = BOUND[prec] if kern == "umma" else BOUND_MMA[prec]
        E, F, S, _ = out[kern]
        assert abs(E - r.E) <= b * abs(r.E) and rel(F, r.F) <= b and rel(S, r.sigma) <= b, kern
    assert rel(out["umma"][1], out["mma"][1]) <= BOUND_MMA[prec]
    assert rel(out["umma"][2], out["mma"][2]) <= BOUND_MMA[prec]


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
    assert abs(E - r.E) <= BOUND[prec] * abs(r.E) and rel(S, r.sigma) <= BOUND[prec]
