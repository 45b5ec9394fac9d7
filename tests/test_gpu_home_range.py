"""Home-atom ranges and passes of the evaluation, through the C ABI.

A plan with hfx_options.home_begin / home_end sums the home-cell atom A of
Eq. exx_expand over that range only; its E, F and sigma are the range's
share, which the oracle computes with the same restriction
(OraclePlan.evaluate(homes=...)), and the shares of disjoint ranges add up
to the whole result (the paper's distribution of quartets over processes,
Sec. 3.3).  home_chunk splits a plan's home atoms into passes that run one
after another with per-pass operand stores; it changes no item, so a
chunked plan matches an unchunked one to rounding.
"""
import json
import os

import numpy as np
import pytest

from oracle import OraclePlan
from paper_2412_11081_gb300 import hfx, inputs

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def rel(a, ref):
    a, ref = np.asarray(a, float), np.asarray(ref, float)
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


def errs(got, ref):
    return abs(got[0] - ref[0]) / abs(ref[0]), rel(got[1], ref[1]), rel(got[2], ref[2])


def run(w, **kw):
    with hfx.Plan(w, **kw) as p:
        return p.evaluate(w.lattice, w.positions)


@pytest.mark.parametrize("prec,tol", [(hfx.HFX_FP64, 1e-10), (hfx.HFX_BF16X6, 1e-5)])
@pytest.mark.parametrize("rng_", [(0, 3), (3, 8), (5, 6)])
def test_home_range_share_matches_oracle(prec, tol, rng_):
    w = inputs.diamond8()
    r = OraclePlan(w).evaluate(homes=range(*rng_))
    got = run(w, precision=prec, home=rng_)
    e = errs(got, (r.E, r.F, r.sigma))
    assert max(e) <= tol, e


@pytest.mark.parametrize("prec", [hfx.HFX_FP64, hfx.HFX_BF16X6])
def test_shares_of_disjoint_ranges_add_up(prec):
    w = inputs.diamond8()
    full = run(w, precision=prec)
    parts = [run(w, precision=prec, home=h) for h in ((0, 2), (2, 7), (7, 8))]
    tot = (sum(p[0] for p in parts), sum(p[1] for p in parts), sum(p[2] for p in parts))
    assert max(errs(tot, full)) <= 1e-12


@pytest.mark.parametrize("prec", [hfx.HFX_FP64, hfx.HFX_BF16X3, hfx.HFX_BF16X6])
def test_passes_change_no_result(prec):
    """Eight atoms in one pass and in three passes of 3/3/2 atoms (per-pass
    scans, stores and launches); the items and their arithmetic are the same."""
    w = inputs.diamond8()
    with hfx.Plan(w, precision=prec) as p:
        one = p.evaluate(w.lattice, w.positions, stats=True)
        assert p.stats.passes == 1
    with hfx.Plan(w, precision=prec, home_chunk=3) as p:
        three = p.evaluate(w.lattice, w.positions, stats=True)
        assert p.stats.passes == 3
        again = p.evaluate(w.lattice, w.positions + 0.01)   # stores reused across passes and calls
    assert max(errs(three, one)) <= 1e-12
    assert np.isfinite(again[0])


def test_passes_on_a_range_of_a_two_species_cell():
    """A home range that starts mid-cell, cut into passes of one atom."""
    rng = np.random.default_rng(11)
    pos = np.array([[0.0, 0.0, 0.0], [1.7, 1.7, 0.0], [1.7, 0.0, 1.7], [0.0, 1.7, 1.7]]) + rng.normal(0, 0.05, (4, 3))
    w = inputs.cut_density(inputs.tiny_model([5, 9], [14, 40], [0, 1, 0, 1], np.eye(3) * 3.4, pos, r_c=2.3,
                                             seed=13), 4.5)
    r = OraclePlan(w).evaluate(homes=[1, 2, 3])
    for prec, tol in ((hfx.HFX_FP64, 1e-10), (hfx.HFX_BF16X6, 1e-5)):
        got = run(w, precision=prec, home=(1, 4), home_chunk=1)
        e = errs(got, (r.E, r.F, r.sigma))
        assert max(e) <= tol, (prec, e)


@pytest.mark.parametrize("prec,tol", [(hfx.HFX_FP64, 1e-10), (hfx.HFX_BF16X6, 1e-5)])
def test_si64_in_four_passes_against_stored_oracle(prec, tol):
    ref = json.load(open(os.path.join(HERE, "golden", "si64_oracle.json")))
    w = inputs.si_supercell(2)
    with hfx.Plan(w, precision=prec, home_chunk=16) as p:
        got = p.evaluate(w.lattice, w.positions, stats=True)
        st = p.stats.as_dict()
    assert st["passes"] == 4 and st["triplets"] == ref["counts"]["triplets"]
    e = errs(got, (ref["E"], ref["F"], ref["sigma"]))
    print(f"si64 four passes, precision {prec}: errE {e[0]:.2e} errF {e[1]:.2e} errS {e[2]:.2e}")
    assert max(e) <= tol, e


def test_reference_error_report():
    """hfx_set_reference: a BF16X6 plan reports its error against the FP64
    result of the same geometry in every stats it fills."""
    w = inputs.diamond8()
    ref = run(w)
    with hfx.Plan(w, precision=hfx.HFX_BF16X6) as p:
        p.evaluate(w.lattice, w.positions, stats=True)
        assert p.stats.ref_err_E == -1.0
        p.set_reference(*ref)
        got = p.evaluate(w.lattice, w.positions, stats=True)
        e = errs(got, ref)
        assert p.stats.ref_err_E == pytest.approx(e[0], rel=1e-12, abs=1e-300)
        assert p.stats.ref_err_F == pytest.approx(e[1], rel=1e-12)
        assert p.stats.ref_err_sigma == pytest.approx(e[2], rel=1e-12)
        assert 0 < max(e) <= 1e-5
        p.set_reference()
        p.evaluate(w.lattice, w.positions, stats=True)
        assert p.stats.ref_err_F == -1.0
        with pytest.raises(ValueError):
            p.set_reference(ref[0], ref[1][:3], ref[2])
