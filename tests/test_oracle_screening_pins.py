"""Pins of the oracle's screening and image enumeration against definitions
written out here, independently of the oracle's own code.

Screening, step 2 (Sec. 3.2, Algorithm 1).  The bound of an item is the
Cauchy-Schwarz product of the Frobenius norms of its blocks; an item is
dropped when the bound does not exceed theta_CS:
  first exchange product, item (A, B, F) summed over G:
      c_AF v_AB d_AB sum_G c_BG d_FG
  second exchange product, item (A, B) summed over F and G:
      v_AB (sum_F c_AF d_FB) (sum_G c_BG d_AG)
with c = max(||C||, ||grad C||), v = max(||V||, ||grad V||) for pairs that
step 1 keeps (0 otherwise) and d = ||D|| for kept D blocks.  These tests
build every block from the block model with brute.py's block routine,
enumerate every candidate item over a fixed box of lattice vectors (not the
oracle's image range), and check
  * that the oracle keeps exactly the items whose bound is above theta_CS,
    with some items kept and some dropped;
  * that every item's exact contribution (its energy and each of its three
    pair-gradient slots, summed by brute force) is no larger than its bound,
    which is the inequality the screening rests on.

Image enumeration.  image_vectors must contain every lattice vector that
brings two atoms of the cell within the range (checked against a large box
on sheared cells with atoms near the cell faces), and the oracle's periodic
sums must equal a lattice sum written out here for a one-atom cell.
"""
import dataclasses
import itertools
import math

import numpy as np
import pytest

from oracle import Options, OraclePlan, evaluate
from oracle.brute import _blocks
from oracle.hfx_oracle import image_vectors, radial_f, radial_h
from paper_2412_11081_gb300 import inputs

BOX = 3   # lattice vectors R with |R_k| <= BOX: far beyond every range used below


def _cell(seed=7):
    """Three atoms of two species in a small periodic cell, D cut at 3.6 A."""
    rng = np.random.default_rng(seed)
    L = np.array([[3.3, 0.0, 0.0], [0.4, 3.1, 0.0], [0.0, 0.3, 3.4]])
    frac = np.array([[0.05, 0.1, 0.0], [0.5, 0.45, 0.55], [0.2, 0.7, 0.35]])
    pos = frac @ L + rng.normal(0, 0.05, (3, 3))
    w = inputs.tiny_model([2, 3], [3, 4], [0, 1, 1], L, pos, r_c=1.35, seed=seed)
    return inputs.cut_density(w, 3.6)


class Model:
    """Blocks, norms and step-1 decisions of one workload over the fixed box."""

    def __init__(self, w, th):
        self.w, self.th = w, th
        self.N = w.n_atoms
        self.L, self.P = np.asarray(w.lattice), np.asarray(w.positions)
        self.RC = 2.0 * w.r_c
        self.box = [tuple(R) for R in itertools.product(range(-BOX, BOX + 1), repeat=3)]
        self.Dm = {}
        for k in range(w.d_index.shape[0]):
            self.Dm[tuple(int(x) for x in w.d_index[k])] = w.d_block(k)
        self._cache = {}
        self._memo = {}

    def _m(self, key, fn):
        if key not in self._memo:
            self._memo[key] = fn()
        return self._memo[key]

    def vec(self, i, j, R):
        return self.P[j] + np.asarray(R, float) @ self.L - self.P[i]

    def blocks(self, i, j, R):
        key = (i, j) + tuple(R)
        if key not in self._cache:
            d = self.vec(i, j, R)
            r = float(np.sqrt(d @ d))
            C, dC, V, dV = _blocks(self.w, i, j, d, r, self.RC)
            if r >= self.RC:   # C pairs are the pairs within R_C
                C, dC = np.zeros_like(C), np.zeros_like(dC)
            self._cache[key] = (C, dC, V, dV)
        return self._cache[key]

    def c(self, i, j, R):
        def f():
            C, dC, _, _ = self.blocks(i, j, R)
            nc, ng = np.linalg.norm(C), np.linalg.norm(dC)
            return max(nc, ng) if (nc > self.th["C"] or ng > self.th["dC"]) else 0.0
        return self._m(("c", i, j) + tuple(R), f)

    def v(self, i, j, R):
        def f():
            _, _, V, dV = self.blocks(i, j, R)
            nv, ng = np.linalg.norm(V), np.linalg.norm(dV)
            return max(nv, ng) if (nv > self.th["V"] or ng > self.th["dV"]) else 0.0
        return self._m(("v", i, j) + tuple(R), f)

    def dn(self, i, j, R):
        D = self.Dm.get((i, j) + tuple(R))
        if D is None:
            return 0.0
        n = np.linalg.norm(D)
        return n if n > self.th["D"] else 0.0

    def D(self, i, j, R):
        return self.Dm[(i, j) + tuple(R)]

    def cpairs(self, i):
        """(j, R) with c > 0: the kept C pairs of atom i."""
        return self._m(("cp", i), lambda: [(j, R) for j in range(self.N) for R in self.box if self.c(i, j, R) > 0.0])

    def yhat(self, x, z, Rz):
        return self._m(("y", x, z) + tuple(Rz), lambda: sum(
            self.c(x, wj, Rw) * self.dn(wj, z, _sub(Rz, Rw)) for (wj, Rw) in self.cpairs(x)))


def _sub(a, b):
    return (a[0] - b[0], a[1] - b[1], a[2] - b[2])


def _bounds(m, terms):
    """Every candidate item with a nonzero bound: {key: bound}."""
    t1, t2 = {}, {}
    for A in range(m.N):
        CA = m.cpairs(A)
        for b in range(m.N):
            for Rb in m.box:
                v = m.v(A, b, Rb)
                if v == 0.0:
                    continue
                if terms & 1:
                    dab = m.dn(A, b, Rb)
                    if dab > 0.0:
                        for (f, Rf) in CA:
                            bd = m.c(A, f, Rf) * v * dab * m.yhat(b, f, _sub(Rf, Rb))
                            if bd > 0.0:
                                t1[(A, b, Rb, f, Rf)] = bd
                if terms & 2:
                    bd = v * m.yhat(A, b, Rb) * m.yhat(b, A, (-Rb[0], -Rb[1], -Rb[2]))
                    if bd > 0.0:
                        t2[(A, b, Rb)] = bd
    return t1, t2


def _kept_by_oracle(plan):
    fr = plan.frozen
    t1, t2 = set(), set()
    for A in range(plan.N):
        Vj, VR, Cj, CR = fr["V_js"][A], fr["V_Rs"][A], fr["C_js"][A], fr["C_Rs"][A]
        for qv, fs in fr["trip"][A].items():
            for qc in fs:
                t1.add((A, int(Vj[qv]), tuple(int(x) for x in VR[qv]), int(Cj[qc]), tuple(int(x) for x in CR[qc])))
        for qv in fr["pair2"][A]:
            t2.add((A, int(Vj[qv]), tuple(int(x) for x in VR[qv])))
    return t1, t2


def _item1(m, A, b, Rb, f, Rf):
    """First-product item (A, B, F) summed over G by brute force: its value
    T = sum_G <C_AF V_AB C_BG, D_AB D_FG> and the three slots with one block
    replaced by its gradient (C_AF, V_AB, and C_BG summed over G)."""
    CAF, dCAF, _, _ = m.blocks(A, f, Rf)
    _, _, VAB, dVAB = m.blocks(A, b, Rb)
    DAB = m.D(A, b, Rb)
    T, gC, gV, gG = 0.0, np.zeros(3), np.zeros(3), np.zeros(3)
    for (g, Rg) in m.cpairs(b):
        Rbg = _add(Rb, Rg)                       # G relative to the home cell
        DFG = m.Dm.get((f, g) + _sub(Rbg, Rf))
        if DFG is None or m.dn(f, g, _sub(Rbg, Rf)) == 0.0:
            continue
        CBG, dCBG, _, _ = m.blocks(b, g, Rg)
        e = "xaf,xy,ybg,ab,fg->"
        T += np.einsum(e, CAF, VAB, CBG, DAB, DFG)
        gC += np.einsum("cxaf,xy,ybg,ab,fg->c", dCAF, VAB, CBG, DAB, DFG)
        gV += np.einsum("xaf,cxy,ybg,ab,fg->c", CAF, dVAB, CBG, DAB, DFG)
        gG += np.einsum("xaf,xy,cybg,ab,fg->c", CAF, VAB, dCBG, DAB, DFG)
    return T, gC, gV, gG


def _item2(m, A, b, Rb):
    """Second-product item (A, B) summed over F and G by brute force."""
    _, _, VAB, dVAB = m.blocks(A, b, Rb)
    T, gC, gV, gG = 0.0, np.zeros(3), np.zeros(3), np.zeros(3)
    for (f, Rf) in m.cpairs(A):
        CAF, dCAF, _, _ = m.blocks(A, f, Rf)
        RFB = _sub(Rb, Rf)
        if m.dn(f, b, RFB) == 0.0:
            continue
        DFB = m.D(f, b, RFB)
        for (g, Rg) in m.cpairs(b):
            Rbg = _add(Rb, Rg)
            if m.dn(A, g, Rbg) == 0.0:
                continue
            DAG = m.D(A, g, Rbg)
            CBG, dCBG, _, _ = m.blocks(b, g, Rg)
            T += np.einsum("xaf,xy,ybg,ag,fb->", CAF, VAB, CBG, DAG, DFB)
            gC += np.einsum("cxaf,xy,ybg,ag,fb->c", dCAF, VAB, CBG, DAG, DFB)
            gV += np.einsum("xaf,cxy,ybg,ag,fb->c", CAF, dVAB, CBG, DAG, DFB)
            gG += np.einsum("xaf,xy,cybg,ag,fb->c", CAF, VAB, dCBG, DAG, DFB)
    return T, gC, gV, gG


def _add(a, b):
    return (a[0] + b[0], a[1] + b[1], a[2] + b[2])


def _split_threshold(bounds, q):
    """A theta_CS near quantile q of the bounds, in a relative gap of at least
    1e-3 between two consecutive bound values (no item sits near it)."""
    v = np.sort(np.array(bounds))
    k0 = int(q * (v.size - 1))
    for k in list(range(k0, v.size - 1)) + list(range(k0 - 1, -1, -1)):
        if v[k + 1] > v[k] * (1 + 1e-3):
            return math.sqrt(v[k] * v[k + 1])
    raise AssertionError("no gap in the bounds")


@pytest.mark.parametrize("step1", [False, True])
def test_cauchy_schwarz_screening_keeps_exactly_the_items_above_theta(step1):
    w = _cell()
    th = dict(C=0.0, dC=0.0, V=0.0, dV=0.0, D=0.0, CS=0.0)
    if step1:
        # step-1 thresholds that drop some C, V and D blocks (C and grad C,
        # V and grad V only jointly)
        th.update(C=0.05, dC=0.08, V=0.3, dV=0.05, D=0.02)
    m = Model(w, th)
    t1, t2 = _bounds(m, 3)
    th["CS"] = _split_threshold(list(t1.values()) + list(t2.values()), 0.4)
    opts = Options.from_theta(th)
    plan = OraclePlan(w, opts, freeze=True)
    k1, k2 = _kept_by_oracle(plan)
    want1 = {k for k, b in t1.items() if b > th["CS"]}
    want2 = {k for k, b in t2.items() if b > th["CS"]}
    assert len(want1) > 0 and len(want1) < len(t1), (len(want1), len(t1))
    assert len(want2) > 0 and len(want2) < len(t2), (len(want2), len(t2))
    assert k1 == want1, (len(k1 - want1), len(want1 - k1))
    assert k2 == want2, (len(k2 - want2), len(want2 - k2))


def test_every_item_is_bounded_by_its_cauchy_schwarz_product():
    """|T| and every component of each gradient slot of every candidate item
    (dropped or kept) stay within the item's bound."""
    w = _cell(seed=3)
    th = dict(C=0.0, dC=0.0, V=0.0, dV=0.0, D=0.0, CS=0.0)
    m = Model(w, th)
    t1, t2 = _bounds(m, 3)
    rng = np.random.default_rng(0)
    keys1 = list(t1)
    pick = [keys1[i] for i in rng.choice(len(keys1), size=min(300, len(keys1)), replace=False)]
    worst = 0.0
    for k in pick:
        T, gC, gV, gG = _item1(m, *k)
        top = max(abs(T), np.abs(gC).max(), np.abs(gV).max(), np.abs(gG).max())
        worst = max(worst, top / t1[k])
        assert top <= t1[k] * (1 + 1e-12), (k, top, t1[k])
    for k, bd in t2.items():
        T, gC, gV, gG = _item2(m, *k)
        top = max(abs(T), np.abs(gC).max(), np.abs(gV).max(), np.abs(gG).max())
        worst = max(worst, top / bd)
        assert top <= bd * (1 + 1e-12), (k, top, bd)
    assert worst > 1e-3   # the bounds are not vacuous


def test_dropped_items_change_the_result_by_no_more_than_their_bounds():
    """Screened minus unscreened energy is the sum of the dropped items'
    energies (every contracted item enters once), so |dE| <= sum of the
    dropped bounds."""
    w = _cell(seed=5)
    th = dict(C=0.0, dC=0.0, V=0.0, dV=0.0, D=0.0, CS=0.0)
    m = Model(w, th)
    t1, t2 = _bounds(m, 3)
    th["CS"] = _split_threshold(list(t1.values()) + list(t2.values()), 0.3)
    full = evaluate(w, Options.from_theta(dict(th, CS=0.0)))
    scr = evaluate(w, Options.from_theta(th))
    dropped = sum(b for b in t1.values() if b <= th["CS"]) + sum(b for b in t2.values() if b <= th["CS"])
    assert 0.0 < abs(scr.E - full.E) <= dropped


# ------------------------------------------------------------ image enumeration
@pytest.mark.parametrize("seed", range(6))
def test_image_vectors_cover_every_pair_within_range(seed):
    rng = np.random.default_rng(seed)
    L = np.eye(3) * rng.uniform(2.0, 4.0, 3)
    off = ~np.eye(3, dtype=bool)
    L[off] = rng.uniform(-2.0, 2.0, 6)   # strongly sheared cell, rows and columns of inv(L) differ
    frac = np.array([[0.01, 0.02, 0.99], [0.98, 0.97, 0.03], [0.5, 0.01, 0.5]])
    pos = frac @ L
    for rmax in (1.0, 2.3, 3.7, 4.9, 6.2):
        have = {tuple(int(x) for x in R) for R in image_vectors(L, rmax)}
        grid = np.array(list(itertools.product(range(-8, 9), repeat=3)), float)
        for i, j in itertools.product(range(3), repeat=2):
            d = pos[j][None, :] + grid @ L - pos[i][None, :]
            for R in grid[(d * d).sum(1) < rmax * rmax].astype(int):
                assert tuple(int(x) for x in R) in have, (rmax, i, j, R)


def _one_atom_cell(a, r_c, dcut):
    """One atom per cubic cell, n_ao = n_abf = 1, G = M = 1, D(R) = exp(-|R L|)
    on the images within dcut (D(0) = 1)."""
    L = np.eye(3) * a
    keys, vals = [], []
    for R in itertools.product(range(-4, 5), repeat=3):
        r = a * math.sqrt(sum(x * x for x in R))
        if r < dcut:
            keys.append((0, 0) + R)
            vals.append(math.exp(-r))
    order = sorted(range(len(keys)), key=lambda k: keys[k])
    return inputs.Workload(
        name="one-atom", species=np.zeros(1, np.int32), lattice=L, positions=np.array([[0.3, -0.2, 0.1]]),
        n_ao=np.array([1], np.int32), n_abf=np.array([1], np.int32), r_c=r_c, omega=0.2,
        G=[np.ones((1, 1, 1))], M=[np.ones((1, 1))], d_index=np.array([keys[k] for k in order], np.int32),
        d_offset=np.arange(len(keys) + 1, dtype=np.int64), d_values=np.array([vals[k] for k in order]),
        theta=dict(C=0.0, dC=0.0, V=0.0, dV=0.0, D=0.0, CS=0.0), seed=0)


def _lattice_sum(w, Fm=np.eye(3)):
    """E = -sum_{F,B,G} c(F) v(B) c(G-B) [d(B) d(G-F) + d(G) d(B-F)] over the
    images of the single atom, with c, v the model's radial functions at the
    strained lattice Fm L and d frozen per image."""
    L = w.lattice @ Fm.T
    RC = 2.0 * w.r_c
    dtab = {tuple(int(x) for x in w.d_index[k, 2:5]): float(w.d_values[k]) for k in range(w.d_index.shape[0])}

    def rr(R):
        return float(np.linalg.norm(np.asarray(R, float) @ L))

    ctab, vtab = {}, {}
    for R in itertools.product(range(-6, 7), repeat=3):
        ctab[R] = 1.0 if R == (0, 0, 0) else float(radial_f(rr(R), RC))
        vtab[R] = 1.0 if R == (0, 0, 0) else float(radial_h(rr(R), w.omega))

    def d(R):
        return dtab.get(R, 0.0)

    near = [R for R in itertools.product(range(-3, 4), repeat=3) if ctab[R] != 0.0]
    E = 0.0
    for B in itertools.product(range(-6, 7), repeat=3):
        vb = vtab[B]
        for Fv in near:
            for Dg in near:
                G = _add(B, Dg)
                E -= ctab[Fv] * vb * ctab[Dg] * (d(B) * d(_sub(G, Fv)) + d(G) * d(_sub(B, Fv)))
    return E


def test_one_atom_cell_matches_the_written_out_lattice_sum():
    w = _one_atom_cell(2.1, 1.2, 4.3)
    res = evaluate(w, Options(theta_C=0, theta_dC=0, theta_V=0, theta_dV=0, theta_D=0, theta_CS=0))
    E = _lattice_sum(w)
    assert abs(res.E - E) <= 1e-12 * abs(E), (res.E, E)
    assert np.max(np.abs(res.F)) <= 1e-12 * abs(E)
    # stress from the four-point formula of Sec. 4.1 applied to the lattice sum in strain
    vol = abs(np.linalg.det(w.lattice))
    h = 1e-4
    for (al, be) in [(0, 0), (1, 2)]:
        def E_at(e):
            eps = np.zeros((3, 3))
            eps[al, be] = e
            return _lattice_sum(w, np.eye(3) + eps)
        s_fd = -(-E_at(2 * h) + 8 * E_at(h) - 8 * E_at(-h) + E_at(-2 * h)) / (12 * h) / vol
        assert abs(s_fd - res.sigma[al, be]) <= 1e-7 * np.max(np.abs(res.sigma)), (al, be, s_fd, res.sigma[al, be])
