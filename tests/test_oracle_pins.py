"""Pins of the CPU oracle against things other than itself.

* closed forms: the scalar dimer energy and force (sympy), and the radial
  derivatives of the block model (sympy);
* brute force: the literal quartet sum of Eq. exx_expand with the six-term
  Eq. Fexx1 and three-term Eq. stress (no factorisation, no factor 2);
* finite differences: the four-point formula of Sec. 4.1 in atom positions
  (dx = 0.001 A) and in homogeneous strain, on frozen screening decisions;
* invariants: sum of forces, stress symmetry, the virial of an isolated
  cluster, homogeneity in C, V and D, translation and permutation
  covariance, and the two routes to the energy.
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import Options, OraclePlan, evaluate
from oracle.brute import brute_force
from oracle.hfx_oracle import radial_df, radial_dh, radial_f, radial_h
from paper_2412_11081_gb300 import inputs

ZERO = Options(theta_C=0.0, theta_dC=0.0, theta_V=0.0, theta_dV=0.0, theta_D=0.0, theta_CS=0.0)


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ------------------------------------------------------------ closed forms
def test_radial_derivatives_match_sympy():
    sp = pytest.importorskip("sympy")
    r = sp.symbols("r", positive=True)
    RC, om = sp.Rational(74, 10), sp.Rational(1, 5)
    f = (1 - (r / RC) ** 2) ** 3 * sp.exp(-r ** 2 / 2)
    h = sp.erfc(om * r) / (r + 1)
    fp, hp = sp.diff(f, r), sp.diff(h, r)
    for rv in [0.1, 0.7, 1.9, 3.3, 5.0, 7.3]:
        assert abs(float(radial_f(rv, 7.4)) - float(f.subs(r, rv))) < 1e-15
        assert abs(float(radial_df(rv, 7.4)) - float(fp.subs(r, rv))) < 1e-14
        assert abs(float(radial_h(rv, 0.2)) - float(sp.N(h.subs(r, rv), 30))) < 1e-15
        assert abs(float(radial_dh(rv, 0.2)) - float(sp.N(hp.subs(r, rv), 30))) < 1e-15
    assert float(radial_f(7.4, 7.4)) == 0.0 and float(radial_f(8.0, 7.4)) == 0.0


def _scalar_dimer(r, r0, r_c=1.5):
    L = np.eye(3) * 60.0
    pos = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
    e = math.exp(-r0)
    d_index = np.array([[0, 0, 0, 0, 0], [0, 1, 0, 0, 0], [1, 0, 0, 0, 0], [1, 1, 0, 0, 0]], np.int32)
    d_values = np.array([1.0, e, e, 1.0])
    return inputs.Workload(
        name="dimer", species=np.zeros(2, np.int32), lattice=L, positions=pos,
        n_ao=np.array([1], np.int32), n_abf=np.array([1], np.int32), r_c=r_c, omega=0.2,
        G=[np.ones((1, 1, 1))], M=[np.ones((1, 1))], d_index=d_index,
        d_offset=np.arange(5, dtype=np.int64), d_values=d_values,
        theta=dict(C=0.0, dC=0.0, V=0.0, dV=0.0, D=0.0, CS=0.0), seed=0)


def test_scalar_dimer_closed_form():
    """Two atoms, n_ao = n_abf = 1, G = M = 1, D frozen at exp(-r0)."""
    sp = pytest.importorskip("sympy")
    r = sp.symbols("r", positive=True)
    r_c, r0 = 1.5, 1.4
    RC = sp.Rational(3)
    fs = (1 - (r / RC) ** 2) ** 3 * sp.exp(-r ** 2 / 2)
    hs = sp.erfc(sp.Rational(1, 5) * r) / (r + 1)
    e = sp.exp(-sp.Float(r0, 30))

    def c(X, Y):
        return 1 if X == Y else fs

    def v(X, Y):
        return 1 if X == Y else hs

    def d(X, Y):
        return 1 if X == Y else e
    Esym = 0
    for A in (0, 1):
        for Fq in (0, 1):
            for B in (0, 1):
                for G in (0, 1):
                    Esym += -c(A, Fq) * v(A, B) * c(B, G) * (d(A, B) * d(Fq, G) + d(A, G) * d(Fq, B))
    dE = sp.diff(Esym, r)
    for rv in [1.1, 1.4, 2.0, 2.7]:
        w = _scalar_dimer(rv, r0, r_c)
        res = evaluate(w, ZERO)
        E_ref = float(sp.N(Esym.subs(r, rv), 30))
        dE_ref = float(sp.N(dE.subs(r, rv), 30))
        assert abs(res.E - E_ref) <= 1e-13 * abs(E_ref)
        # atom 1 sits at +x: F_1 = -dE/dr, F_0 = +dE/dr; nothing off-axis
        assert abs(res.F[1, 0] + dE_ref) <= 1e-12 * max(1.0, abs(dE_ref))
        assert abs(res.F[0, 0] - dE_ref) <= 1e-12 * max(1.0, abs(dE_ref))
        assert np.max(np.abs(res.F[:, 1:])) < 1e-14


# ------------------------------------------------------------ brute force
def _tiny_periodic(seed=7, species=(0, 1), a=3.2, dcut=3.5):
    rng = np.random.default_rng(seed)
    L = np.eye(3) * a
    pos = np.array([[0.1, 0.2, 0.0], [1.5, 1.7, 1.4]])[:len(species)] + rng.normal(0, 0.05, (len(species), 3))
    w = inputs.tiny_model([2, 3], [3, 4], species, L, pos, r_c=1.3, seed=seed)
    return inputs.cut_density(w, dcut)


def _aniso_for(w, seed=11):
    rng = np.random.default_rng(seed)
    S = w.n_ao.shape[0]
    Gp = [rng.standard_normal(w.G[k].shape) for k in range(S * S)]
    e = np.array([0.3, -0.5, 0.8])
    return Gp, e / np.linalg.norm(e)


@pytest.mark.parametrize("terms", [1, 2, 3])
def test_factorised_matches_brute_force(terms):
    w = _tiny_periodic()
    ref = brute_force(w, terms=terms)
    res = evaluate(w, dataclasses.replace(ZERO, terms=terms))
    assert abs(res.E - ref[0]) <= 1e-12 * abs(ref[0])
    assert _rel(res.F, ref[1]) < 1e-11
    assert _rel(res.sigma, ref[2]) < 1e-11


def test_factorised_matches_brute_force_anisotropic():
    """grad C is a general 3-component block here (not template x scalar)."""
    w = _tiny_periodic(seed=9)
    an = _aniso_for(w)
    ref = brute_force(w, terms=3, aniso=an)
    res = evaluate(w, dataclasses.replace(ZERO, aniso=an))
    assert abs(res.E - ref[0]) <= 1e-12 * abs(ref[0])
    assert _rel(res.F, ref[1]) < 1e-11
    assert _rel(res.sigma, ref[2]) < 1e-11


def test_brute_force_three_atom_cluster_two_species():
    L = np.eye(3) * 40.0
    pos = np.array([[5.0, 5.0, 5.0], [6.3, 5.4, 4.8], [5.2, 6.6, 5.9]])
    w = inputs.tiny_model([2, 3], [3, 2], [0, 1, 1], L, pos, r_c=1.4, seed=3)
    ref = brute_force(w)
    res = evaluate(w, ZERO)
    assert abs(res.E - ref[0]) <= 1e-12 * abs(ref[0])
    assert _rel(res.F, ref[1]) < 1e-11
    assert _rel(res.sigma, ref[2]) < 1e-11


# ------------------------------------------------------------ finite differences
def _fd4(fun, h):
    """Four-point central formula of Sec. 4.1: O(h^4)."""
    return (-fun(2 * h) + 8 * fun(h) - 8 * fun(-h) + fun(-2 * h)) / (12 * h)


def _fd_check_positions(w, opts, coords, tol, h=1e-3):
    plan = OraclePlan(w, opts, freeze=True)
    res = plan.evaluate()
    for (i, c) in coords:
        def E_at(dx):
            p = w.positions.copy()
            p[i, c] += dx
            return plan.evaluate(positions=p).E
        F_fd = -_fd4(E_at, h)
        assert abs(F_fd - res.F[i, c]) <= tol * np.max(np.abs(res.F)), (i, c, F_fd, res.F[i, c])
    return res


def _fd_check_strain(w, opts, comps, tol, h=1e-4):
    plan = OraclePlan(w, opts, freeze=True)
    res = plan.evaluate()
    vol = abs(np.linalg.det(w.lattice))
    for (al, be) in comps:
        def E_at(e):
            eps = np.zeros((3, 3))
            eps[al, be] = e
            Fm = np.eye(3) + eps
            return plan.evaluate(lattice=w.lattice @ Fm.T, positions=w.positions @ Fm.T).E
        s_fd = -_fd4(E_at, h) / vol
        assert abs(s_fd - res.sigma[al, be]) <= tol * np.max(np.abs(res.sigma)), (al, be, s_fd, res.sigma[al, be])
    return res


def test_fd_positions_tiny_periodic_screened():
    w = _tiny_periodic(seed=5)
    opts = Options.from_theta(w.theta)
    _fd_check_positions(w, opts, [(0, 0), (0, 2), (1, 1)], tol=1e-7)


def test_fd_strain_tiny_periodic_screened():
    w = _tiny_periodic(seed=5)
    opts = Options.from_theta(w.theta)
    _fd_check_strain(w, opts, [(0, 0), (1, 2), (2, 1), (2, 0)], tol=1e-7)


@pytest.mark.slow
def test_fd_diamond8_short_density():
    """8-atom diamond cell (n_ao 4, n_abf 9) with D cut at 6 A, thresholds 1e-10."""
    w = inputs.cut_density(inputs.diamond8(), 6.0)
    opts = Options.from_theta(w.theta)
    _fd_check_positions(w, opts, [(3, 0), (5, 2)], tol=1e-7)
    _fd_check_strain(w, opts, [(0, 1), (2, 2)], tol=1e-7)


def test_fd_anisotropic_positions():
    w = _tiny_periodic(seed=12)
    an = _aniso_for(w, 4)
    opts = dataclasses.replace(Options.from_theta(w.theta), aniso=an)
    _fd_check_positions(w, opts, [(0, 1), (1, 2)], tol=1e-7)
    _fd_check_strain(w, opts, [(0, 2), (2, 0)], tol=1e-7)


# ------------------------------------------------------------ invariants
def test_invariants_sum_forces_and_stress_symmetry():
    w = inputs.cut_density(inputs.diamond8(), 6.0)
    res = evaluate(w)
    assert np.max(np.abs(res.F.sum(0))) <= 1e-12 * np.max(np.abs(res.F))
    assert np.max(np.abs(res.sigma - res.sigma.T)) <= 1e-12 * np.max(np.abs(res.sigma))


def test_isolated_cluster_virial():
    """No images in range: Omega sigma_ab = sum_I F_I^a tau_I^b."""
    L = np.eye(3) * 50.0
    pos = np.array([[5.0, 5.0, 5.0], [6.1, 5.3, 4.6], [5.4, 6.5, 5.8], [6.9, 6.4, 6.2]])
    w = inputs.tiny_model([2, 3], [3, 4], [0, 1, 0, 1], L, pos, r_c=1.5, seed=21)
    res = evaluate(w, ZERO)
    vol = abs(np.linalg.det(L))
    assert _rel(vol * res.sigma, np.einsum("ia,ib->ab", res.F, pos)) < 1e-12


def test_homogeneity():
    w = _tiny_periodic(seed=8)
    base = evaluate(w, ZERO)
    lam = 1.7
    for what, power in (("G", 2), ("M", 1), ("D", 2)):
        w2 = dataclasses.replace(w)
        if what == "G":
            w2.G = [g * lam for g in w.G]
        elif what == "M":
            w2.M = [m * lam for m in w.M]
        else:
            w2.d_values = w.d_values * lam
        r2 = evaluate(w2, ZERO)
        s = lam ** power
        assert abs(r2.E - s * base.E) <= 1e-12 * abs(s * base.E)
        assert _rel(r2.F, s * base.F) < 1e-12
        assert _rel(r2.sigma, s * base.sigma) < 1e-12


def test_translation_and_permutation_covariance():
    w = _tiny_periodic(seed=6, species=(0, 1))
    base = evaluate(w, ZERO)
    # rigid translation of every atom
    wt = w.with_positions(w.positions + np.array([0.37, -0.21, 0.05]))
    rt = evaluate(wt, ZERO)
    assert abs(rt.E - base.E) <= 1e-12 * abs(base.E)
    assert _rel(rt.F, base.F) < 1e-10 and _rel(rt.sigma, base.sigma) < 1e-10
    # swap the two atoms' labels (positions, species and D follow)
    perm = np.array([1, 0])
    wp = dataclasses.replace(w)
    wp.species = w.species[perm]
    wp.positions = w.positions[perm]
    inv = np.argsort(perm)
    idx = w.d_index.copy()
    idx[:, 0], idx[:, 1] = inv[w.d_index[:, 0]], inv[w.d_index[:, 1]]
    order = np.lexsort((idx[:, 4], idx[:, 3], idx[:, 2], idx[:, 1], idx[:, 0]))
    blocks = [w.d_values[w.d_offset[k]:w.d_offset[k + 1]] for k in order]
    wp.d_index = idx[order]
    wp.d_offset = np.concatenate([[0], np.cumsum([b.size for b in blocks])]).astype(np.int64)
    wp.d_values = np.concatenate(blocks)
    rp = evaluate(wp, ZERO)
    assert abs(rp.E - base.E) <= 1e-12 * abs(base.E)
    assert _rel(rp.F, base.F[perm]) < 1e-11
    assert _rel(rp.sigma, base.sigma) < 1e-11


def test_two_energy_routes_agree():
    """E = -sum <V, R> (the V side) equals -sum <C_AF, Q_AF> (the C side)."""
    w = inputs.cut_density(inputs.diamond8(), 6.0)
    res = evaluate(w)
    assert abs(res.counts["E_via_Q"] - res.E) <= 1e-12 * abs(res.E)


def test_screening_error_small_and_decisions_counted():
    """Screened vs unscreened (Sec. 4.2 methodology): small, nonzero work saved."""
    w = _tiny_periodic(seed=5)
    scr = evaluate(w)
    full = evaluate(w, ZERO)
    assert _rel(scr.F, full.F) < 1e-6
    assert scr.counts["triplets"] <= full.counts["triplets"]
