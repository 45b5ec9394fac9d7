"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerance: the FP64 path must match the oracle to a relative force and
stress error of 1e-10, read as max|x - x_ref| / max|x_ref| per output
(and |dE|/|E| for the energy).  Screening decisions are taken on both
sides in FP64 from the same norms; a decision that flips at the threshold
changes a result by at most ~theta_CS, far inside this tolerance.
"""
import dataclasses
import json
import os

import numpy as np
import pytest

from oracle import Options, OraclePlan, evaluate
from paper_2412_11081_gb300 import hfx, inputs

pytestmark = pytest.mark.gpu
TOL = 1e-10
HERE = os.path.dirname(os.path.abspath(__file__))
ZERO_TH = dict(C=0.0, dC=0.0, V=0.0, dV=0.0, D=0.0, CS=0.0)


def rel(a, ref):
    a, ref = np.asarray(a, float), np.asarray(ref, float)
    return float(np.max(np.abs(a - ref)) / max(float(np.max(np.abs(ref))), 1e-300))


def gpu_eval(w, **kw):
    with hfx.Plan(w, **kw) as p:
        return p.evaluate(w.lattice, w.positions, stats=True) + (p.stats.as_dict(),)


def assert_parity(g, r, tol=TOL):
    E, F, S = g[0], g[1], g[2]
    assert abs(E - r.E) <= tol * abs(r.E), (E, r.E)
    assert rel(F, r.F) <= tol, rel(F, r.F)
    assert rel(S, r.sigma) <= tol, rel(S, r.sigma)


def tiny_periodic(seed=7, dcut=3.5):
    rng = np.random.default_rng(seed)
    L = np.eye(3) * 3.2
    pos = np.array([[0.1, 0.2, 0.0], [1.5, 1.7, 1.4]]) + rng.normal(0, 0.05, (2, 3))
    w = inputs.tiny_model([2, 3], [3, 4], [0, 1], L, pos, r_c=1.3, seed=seed)
    return inputs.cut_density(w, dcut)


@pytest.mark.parametrize("screened", [False, True])
def test_tiny_periodic_two_species(screened):
    w = tiny_periodic()
    th = w.theta if screened else ZERO_TH
    r = evaluate(w, Options.from_theta(th))
    assert_parity(gpu_eval(w, theta=th), r)


@pytest.mark.parametrize("terms", [1, 2])
def test_each_exchange_product_alone(terms):
    w = tiny_periodic(seed=3)
    r = evaluate(w, dataclasses.replace(Options.from_theta(w.theta), terms=terms))
    assert_parity(gpu_eval(w, terms=terms), r)


def test_anisotropic_gradient_blocks():
    """grad C is a general 3-component block (not template x scalar)."""
    w = tiny_periodic(seed=9)
    rng = np.random.default_rng(4)
    Gp = [rng.standard_normal(g.shape) for g in w.G]
    e = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    r = evaluate(w, dataclasses.replace(Options.from_theta(w.theta), aniso=(Gp, e)))
    assert_parity(gpu_eval(w, aniso=(Gp, e)), r)


def test_diamond8_full():
    """8-atom diamond cell, n_ao 4, n_abf 9, full D (thousands of images)."""
    w = inputs.diamond8()
    r = evaluate(w)
    g = gpu_eval(w)
    assert_parity(g, r)
    st = g[3]
    assert st["triplets"] == r.counts["triplets"]
    assert st["term2_pairs"] == r.counts["term2_pairs"]
    assert st["y_blocks"] == r.counts["y_blocks"]


def test_perovskite_cell_three_species():
    """5-atom CsSnI3-shaped cell: n_ao 18/13/13, n_abf 75/60/60 (ragged
    shapes, chunked shared-memory tiles)."""
    w = inputs.perovskite_supercell(1, seed=11)
    r = evaluate(w)
    assert_parity(gpu_eval(w), r)


def test_si64_full_size_against_stored_oracle():
    """The 64-atom Si-like supercell the benchmark times (n_ao 13, n_abf
    50, r_c 3.7 A, thresholds 1e-10), against the oracle's stored result
    (tests/golden/make_golden.py)."""
    ref = json.load(open(os.path.join(HERE, "golden", "si64_oracle.json")))
    w = inputs.si_supercell(2)
    assert w.seed == ref["seed"] and w.n_atoms == ref["n_atoms"]
    E, F, S, st = gpu_eval(w)
    assert abs(E - ref["E"]) <= TOL * abs(ref["E"])
    assert rel(F, ref["F"]) <= TOL
    assert rel(S, ref["sigma"]) <= TOL
    assert st["triplets"] == ref["counts"]["triplets"]
    assert st["term1_pairs"] == ref["counts"]["term1_pairs"]
    assert st["term2_pairs"] == ref["counts"]["term2_pairs"]
    assert abs(st["flops_total"] / ref["flops"] - 1.0) < 1e-12


def test_single_atom_cell_self_images_only():
    L = np.eye(3) * 2.9
    w = inputs.tiny_model([3], [5], [0], L, np.array([[0.2, 0.1, 0.3]]), r_c=1.6, seed=5)
    w = inputs.cut_density(w, 6.0)
    r = evaluate(w)
    g = gpu_eval(w)
    # one atom: every pair is a self-image, so F = 0 exactly in the oracle and
    # to rounding (FP64 atomics) on the GPU, on the scale of |E| per Angstrom
    assert np.all(r.F == 0.0)
    assert np.max(np.abs(g[1])) <= 1e-13 * abs(r.E)
    assert abs(g[0] - r.E) <= TOL * abs(r.E)
    assert rel(g[2], r.sigma) <= TOL


def test_everything_screened_out():
    w = tiny_periodic()
    th = dict(C=1e30, dC=1e30, V=1e30, dV=1e30, D=1e30, CS=1e30)
    E, F, S, st = gpu_eval(w, theta=th)
    assert E == 0.0 and not F.any() and not S.any()
    assert st["triplets"] == 0 and st["term2_pairs"] == 0


def test_frozen_plan_finite_differences():
    """F = -dE/dx and sigma = -(1/Omega) dE/deps on the GPU path itself
    (frozen lists and screening decisions, four-point formula, Sec. 4.1)."""
    w = inputs.cut_density(inputs.diamond8(), 6.0)
    with hfx.Plan(w, freeze_lists=True) as p:
        E0, F0, S0 = p.evaluate(w.lattice, w.positions)
        h = 1e-3
        for (i, c) in [(2, 1), (6, 0)]:
            def E_at(dx):
                q = w.positions.copy()
                q[i, c] += dx
                return p.evaluate(w.lattice, q)[0]
            fd = -(-E_at(2 * h) + 8 * E_at(h) - 8 * E_at(-h) + E_at(-2 * h)) / (12 * h)
            assert abs(fd - F0[i, c]) <= 1e-7 * np.max(np.abs(F0))
        vol = abs(np.linalg.det(w.lattice))
        he = 1e-4
        for (a, b) in [(0, 0), (1, 2)]:
            def E_eps(e):
                eps = np.zeros((3, 3))
                eps[a, b] = e
                Fm = np.eye(3) + eps
                return p.evaluate(w.lattice @ Fm.T, w.positions @ Fm.T)[0]
            fd = -(-E_eps(2 * he) + 8 * E_eps(he) - 8 * E_eps(-he) + E_eps(-2 * he)) / (12 * he) / vol
            assert abs(fd - S0[a, b]) <= 1e-7 * np.max(np.abs(S0))


def test_frozen_plan_rejects_moves_beyond_skin():
    w = tiny_periodic()
    with hfx.Plan(w, freeze_lists=True, skin=0.2) as p:
        p.evaluate(w.lattice, w.positions)
        q = w.positions.copy()
        q[0, 0] += 0.3
        with pytest.raises(hfx.HfxError) as ei:
            p.evaluate(w.lattice, q)
        assert ei.value.status == 5


def test_lists_rebuilt_when_atoms_move_far():
    w = tiny_periodic(seed=13)
    q = w.positions.copy()
    q[1] += np.array([0.4, -0.3, 0.25])
    w2 = w.with_positions(q)
    r = evaluate(w2)
    with hfx.Plan(w, skin=0.3) as p:
        p.evaluate(w.lattice, w.positions)
        g = p.evaluate(w2.lattice, w2.positions)
    assert_parity(g, r)


def test_device_entry_point_matches_host_entry_point():
    torch = pytest.importorskip("torch")
    w = inputs.cut_density(inputs.diamond8(), 8.0)
    with hfx.Plan(w) as p:
        E, F, S = p.evaluate(w.lattice, w.positions)
        dpos = torch.tensor(w.positions, dtype=torch.float64, device="cuda")
        dout = torch.zeros(1 + 3 * w.n_atoms + 9, dtype=torch.float64, device="cuda")
        p.evaluate_device(w.lattice, dpos.data_ptr(), dout.data_ptr())
        torch.cuda.synchronize()
        out = dout.cpu().numpy()
    assert abs(out[0] - E) <= 1e-13 * abs(E)
    assert rel(out[1:1 + 3 * w.n_atoms].reshape(-1, 3), F) <= 1e-13
    assert rel(out[-9:].reshape(3, 3), S) <= 1e-13


def test_nonfinite_positions_rejected():
    w = tiny_periodic()
    with hfx.Plan(w) as p:
        q = w.positions.copy()
        q[0, 0] = np.nan
        with pytest.raises(hfx.HfxError) as ei:
            p.evaluate(w.lattice, q)
        assert ei.value.status == 1
        # the plan stays usable after a rejected call
        E, F, S = p.evaluate(w.lattice, w.positions)
        assert np.isfinite(E)


def _thin_cell(seed):
    """Three atoms of two species in a long, sheared cell: several pair-list
    cells along the long axis, one or two across, and pairs many images away."""
    rng = np.random.default_rng(seed)
    L = np.array([[3.0, 0.0, 0.0], [0.9, 2.8, 0.0], [-0.6, 0.7, 11.0]])
    frac = np.array([[0.02, 0.97, 0.01], [0.51, 0.48, 0.35], [0.96, 0.03, 0.93]])
    pos = frac @ L + rng.normal(0, 0.05, (3, 3))
    w = inputs.tiny_model([2, 3], [3, 4], [0, 1, 1], L, pos, r_c=1.35, seed=seed)
    return inputs.cut_density(w, 3.6)


def _sheared_cell(seed):
    """Three atoms near the faces of a strongly sheared cell."""
    rng = np.random.default_rng(seed)
    L = np.eye(3) * rng.uniform(2.6, 3.6, 3)
    off = ~np.eye(3, dtype=bool)
    L[off] = rng.uniform(-1.2, 1.2, 6)
    frac = np.array([[0.01, 0.02, 0.99], [0.98, 0.97, 0.03], [0.5, 0.01, 0.5]])
    w = inputs.tiny_model([2, 3], [3, 4], [0, 1, 1], L, frac @ L, r_c=1.3, seed=seed)
    return inputs.cut_density(w, 3.4)


@pytest.mark.parametrize("make,seed", [(_thin_cell, 1), (_thin_cell, 2), (_sheared_cell, 3), (_sheared_cell, 4)])
def test_pair_lists_on_thin_and_sheared_cells(make, seed):
    """The pair lists come from a cell list over wrapped fractional
    coordinates; on cells whose axes get different cell counts, with atoms at
    the faces and pairs across many images, the kept counts and the result
    must still be the oracle's."""
    w = make(seed)
    r = evaluate(w, Options.from_theta(w.theta))
    g = gpu_eval(w)
    st = g[3]
    for k in ("c_pairs", "triplets", "term1_pairs", "term2_pairs", "y_blocks"):
        assert st[k] == r.counts[k], (k, st[k], r.counts[k])
    assert_parity(g, r)
