"""Split precision on blocks wider than 16 orbitals (hfx_wide.cu): the
CsSnI3-shaped perovskite cells (Cs n_ao 18, n_abf 75; Sn, I n_ao 13, n_abf 60).

Against the FP64 CPU oracle (small cells) and the FP64 GPU path (itself
within 1e-10 of the oracle); the same 1e-5 relative contract as the other
split-precision tests, the same kept items (screening is FP64 on both sides).
"""
import dataclasses

import numpy as np
import pytest

from oracle import Options, evaluate
from paper_2412_11081_gb300 import hfx, inputs

pytestmark = pytest.mark.gpu
BOUND = 1e-5


def rel(a, ref):
    a, ref = np.asarray(a, float), np.asarray(ref, float)
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


def errs(got, ref):
    return abs(got[0] - ref[0]) / abs(ref[0]), rel(got[1], ref[1]), rel(got[2], ref[2])


def run(w, prec, **kw):
    with hfx.Plan(w, precision=prec, **kw) as p:
        E, F, S = p.evaluate(w.lattice, w.positions, stats=True)
        return E, F, S, p.stats.as_dict()


def wide_two_species(seed=5):
    """Two species, n_ao 18 and 7, n_abf 23 and 11 (ragged tiles everywhere)."""
    rng = np.random.default_rng(seed)
    pos = np.array([[0.1, 0.2, 0.0], [1.6, 1.5, 1.7]]) + rng.normal(0, 0.05, (2, 3))
    w = inputs.tiny_model([18, 7], [23, 11], [0, 1], np.eye(3) * 3.3, pos, r_c=1.4, seed=seed)
    return inputs.cut_density(w, 4.0)


@pytest.mark.parametrize("prec", [hfx.HFX_BF16X6, hfx.HFX_BF16X3])
def test_wide_two_species_against_oracle(prec):
    w = wide_two_species()
    r = evaluate(w)
    E, F, S, st = run(w, prec)
    er = errs((E, F, S), (r.E, r.F, r.sigma))
    print(f"two species n_ao 18/7, precision {prec}: errE {er[0]:.2e} errF {er[1]:.2e} errS {er[2]:.2e}")
    assert st["triplets"] == r.counts["triplets"] and st["term2_pairs"] == r.counts["term2_pairs"]
    assert st["y_blocks"] == r.counts["y_blocks"]
    assert max(er) <= BOUND, er


@pytest.mark.parametrize("terms", [1, 2])
def test_wide_each_exchange_product_alone(terms):
    """Each of the two products of Eq. exx_expand on its own (terms mask)."""
    w = wide_two_species(seed=8)
    r = evaluate(w, dataclasses.replace(Options.from_theta(w.theta), terms=terms))
    E, F, S, _ = run(w, hfx.HFX_BF16X6, terms=terms)
    er = errs((E, F, S), (r.E, r.F, r.sigma))
    assert max(er) <= BOUND, er


def test_perovskite_cell_against_oracle():
    """5-atom CsSnI3-shaped cell, full D (thousands of images)."""
    w = inputs.perovskite_supercell(1, seed=11)
    r = evaluate(w)
    E, F, S, st = run(w, hfx.HFX_BF16X6)
    er = errs((E, F, S), (r.E, r.F, r.sigma))
    print(f"perovskite5 BF16X6: errE {er[0]:.2e} errF {er[1]:.2e} errS {er[2]:.2e}")
    assert st["triplets"] == r.counts["triplets"] and st["term2_pairs"] == r.counts["term2_pairs"]
    assert max(er) <= BOUND, er
    assert abs(st["flops_total"] / r.flops - 1.0) < 1e-12


@pytest.mark.parametrize("chunk", [0, 7])
def test_perovskite40_against_fp64_gpu(chunk):
    """2x2x2 perovskite (40 atoms) with jitter, whole and in passes of 7 home
    atoms, against the FP64 GPU path; sum F = 0 to rounding."""
    w = inputs.perovskite_supercell(2, seed=13)
    ref = run(w, hfx.HFX_FP64)
    got = run(w, hfx.HFX_BF16X6, home_chunk=chunk)
    er = errs(got, ref)
    print(f"perovskite40 BF16X6 (home_chunk {chunk}): errE {er[0]:.2e} errF {er[1]:.2e} errS {er[2]:.2e}")
    assert got[3]["triplets"] == ref[3]["triplets"]
    assert max(er) <= BOUND, er
    F = got[1]
    assert np.max(np.abs(F.sum(0))) <= 1e-9 * np.max(np.abs(F))


def test_wide_anisotropic_gradient_blocks():
    """grad C as a general 3-component block on the wide path too."""
    w = wide_two_species(seed=9)
    rng = np.random.default_rng(4)
    Gp = [rng.standard_normal(g.shape) for g in w.G]
    e = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    r = evaluate(w, dataclasses.replace(Options.from_theta(w.theta), aniso=(Gp, e)))
    E, F, S, _ = run(w, hfx.HFX_BF16X6, aniso=(Gp, e))
    er = errs((E, F, S), (r.E, r.F, r.sigma))
    assert max(er) <= BOUND, er
