"""Split-precision path (bf16 pieces on the tensor cores, FP32 accumulation,
FP64 screening and reductions) against the FP64 CPU oracle.

Error metric: max|x - x_ref| / max|x_ref| per output (|dE|/|E| for E).
HFX_BF16X6 keeps every piece product down to 2^-24 of the operands, so its
error is set by FP32 accumulation (~1e-6): it must meet the 1e-5 relative
force/stress contract.  HFX_BF16X3 drops the products below 2^-16 of the
operands (~3 * 2^-18 relative per product), which puts it at the contract;
it is held to 3e-5 and reported, not used for the contract.
"""
import json
import os

import numpy as np
import pytest

from oracle import evaluate
from paper_2412_11081_gb300 import hfx, inputs

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
BOUND = {hfx.HFX_BF16X6: 1e-5, hfx.HFX_BF16X3: 3e-5}


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


@pytest.mark.parametrize("prec", [hfx.HFX_BF16X6, hfx.HFX_BF16X3])
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


@pytest.mark.parametrize("prec", [hfx.HFX_BF16X6, hfx.HFX_BF16X3])
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
