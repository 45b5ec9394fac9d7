"""Seeded synthetic workloads for the HFX force/stress hot path.

This module produces INPUTS only: geometry, species, the block-model
templates G and M, and the fixed density matrix D.  It contains none of the
method's arithmetic (no pair lists for C or V, no block values, no
screening, no contraction), so that both the CPU oracle and the CUDA path
can consume the same inputs without sharing any computation.

What the inputs stand in for
----------------------------
The paper (Sec. 2, Eqs. 1-2, Eq. exx_expand) takes the two-centre RI
coefficients C, the ABF Coulomb blocks V, their nuclear gradients and the
density matrix D as given tensors over periodic atom pairs (I, J, R).  Its
own tensors come from NAO/ABF integrals of real crystals (Si supercells and
CsSnI3, Sec. 4), which are not available here.  The synthetic model keeps
the structure those tensors have:

* block shapes n_abf(I) x n_ao(I) x n_ao(J) for C and n_abf(I) x n_abf(J)
  for V, per species pair;
* translational reuse: every block is a species-pair template times a
  radial function of the pair distance (Sec. 3.1);
* the symmetries V_BA = V_AB^T and D_JI(-R) = D_IJ(R)^T (Sec. 3.1);
* a density matrix that decays exponentially with the pair distance and is
  independent of the positions (it is frozen at the initial geometry, as the
  force part F^X1 treats it).

Random numbers come from numpy's Philox counter-based generator seeded per
workload; the draw order is fixed and documented in ``make_workload``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence

import numpy as np

# Diamond-cubic basis (fractional), 8 atoms per conventional cell.
_DIAMOND_FRAC = np.array([
    [0.00, 0.00, 0.00], [0.00, 0.50, 0.50], [0.50, 0.00, 0.50], [0.50, 0.50, 0.00],
    [0.25, 0.25, 0.25], [0.25, 0.75, 0.75], [0.75, 0.25, 0.75], [0.75, 0.75, 0.25],
])

# Cubic ABX3 perovskite basis (fractional): A (Cs) at the corner, B (Sn) at
# the body centre, X (I) at the three face centres.
_PEROVSKITE_FRAC = np.array([
    [0.0, 0.0, 0.0],   # Cs
    [0.5, 0.5, 0.5],   # Sn
    [0.5, 0.5, 0.0],   # I
    [0.5, 0.0, 0.5],   # I
    [0.0, 0.5, 0.5],   # I
])
_PEROVSKITE_SPECIES = np.array([0, 1, 2, 2, 2], dtype=np.int32)

DEFAULT_THETA = 1e-10
D_DECAY_LENGTH = 1.0      # Angstrom, decay length of the synthetic D
OMEGA = 0.2               # 1/Angstrom, screening parameter of the model V
JITTER_SIGMA = 0.05       # Angstrom


@dataclasses.dataclass
class Workload:
    """One synthetic structure plus its block model and density matrix.

    Array conventions (all C-contiguous):
      species    int32  [n_atoms]
      lattice    f64    [3, 3]   rows are the lattice vectors a1, a2, a3 (A)
      positions  f64    [n_atoms, 3]  Cartesian (A)
      n_ao/n_abf int32  [n_species]
      G[s*S+t]   f64    [n_abf(s), n_ao(s), n_ao(t)]   C template
      M[s*S+t]   f64    [n_abf(s), n_abf(t)]           V template
      d_index    int32  [n_d, 5]  rows (I, J, R1, R2, R3), sorted
      d_offset   int64  [n_d + 1] element offsets into d_values
      d_values   f64    [d_offset[-1]]  block (I,J,R) is n_ao(I) x n_ao(J),
                 row-major; both orientations are present and
                 D_JI(-R) = D_IJ(R)^T exactly.
    """
    name: str
    species: np.ndarray
    lattice: np.ndarray
    positions: np.ndarray
    n_ao: np.ndarray
    n_abf: np.ndarray
    r_c: float
    omega: float
    G: List[np.ndarray]
    M: List[np.ndarray]
    d_index: np.ndarray
    d_offset: np.ndarray
    d_values: np.ndarray
    theta: Dict[str, float]
    seed: int
    strain: Optional[np.ndarray] = None
    lattice0: Optional[np.ndarray] = None    # unstrained lattice
    positions0: Optional[np.ndarray] = None  # jittered, unstrained positions

    @property
    def n_atoms(self) -> int:
        return int(self.species.shape[0])

    @property
    def n_species(self) -> int:
        return int(self.n_ao.shape[0])

    def d_block(self, k: int) -> np.ndarray:
        i, j = int(self.d_index[k, 0]), int(self.d_index[k, 1])
        a, b = int(self.n_ao[self.species[i]]), int(self.n_ao[self.species[j]])
        return self.d_values[self.d_offset[k]:self.d_offset[k + 1]].reshape(a, b)

    def with_positions(self, positions: np.ndarray, lattice: Optional[np.ndarray] = None) -> "Workload":
        """Same model and D, new geometry (D stays frozen)."""
        w = dataclasses.replace(self)
        w.positions = np.ascontiguousarray(positions, dtype=np.float64)
        if lattice is not None:
            w.lattice = np.ascontiguousarray(lattice, dtype=np.float64)
        return w

    def thetas(self) -> Dict[str, float]:
        return dict(self.theta)


def image_range(lattice: np.ndarray, rmax: float) -> np.ndarray:
    """Integer lattice vectors R that can bring two atoms of the cell within rmax.

    |R_k| <= ceil(rmax * |b_k|) + 1 with b_k the reciprocal vectors (rows of
    inv(L)^T); the +1 covers fractional differences in (-1, 1).
    """
    recip = np.linalg.inv(lattice).T
    nmax = [int(math.ceil(rmax * np.linalg.norm(recip[k]))) + 1 for k in range(3)]
    rr = [np.arange(-n, n + 1) for n in nmax]
    g = np.stack(np.meshgrid(*rr, indexing="ij"), axis=-1).reshape(-1, 3)
    return g.astype(np.int64)


def _geometry(kind: str, n_rep: int, a: float):
    if kind == "diamond":
        frac, spec = _DIAMOND_FRAC, np.zeros(8, dtype=np.int32)
    elif kind == "perovskite":
        frac, spec = _PEROVSKITE_FRAC, _PEROVSKITE_SPECIES
    else:
        raise ValueError(kind)
    cells = np.stack(np.meshgrid(*([np.arange(n_rep)] * 3), indexing="ij"), -1).reshape(-1, 3)
    fr = (cells[:, None, :] + frac[None, :, :]).reshape(-1, 3) / n_rep
    species = np.tile(spec, cells.shape[0]).astype(np.int32)
    lattice = np.eye(3) * (a * n_rep)
    return species, lattice, fr


def _make_templates(rng, n_ao, n_abf):
    S = len(n_ao)
    G = [None] * (S * S)
    M = [None] * (S * S)
    for s in range(S):
        for t in range(S):
            G[s * S + t] = rng.standard_normal((n_abf[s], n_ao[s], n_ao[t]))
    for s in range(S):
        X = rng.standard_normal((n_abf[s], n_abf[s]))
        M[s * S + s] = X @ X.T / n_abf[s] + np.eye(n_abf[s])       # on-site SPD
        for t in range(s + 1, S):
            Mst = rng.standard_normal((n_abf[s], n_abf[t])) / math.sqrt(n_abf[s])
            M[s * S + t] = Mst
            M[t * S + s] = np.ascontiguousarray(Mst.T)
    return G, M


def _make_density(rng, species, lattice, pos, n_ao, theta_d, ell=D_DECAY_LENGTH):
    """Synthetic fixed D_IJ(R) = S_IJR * exp(-d0/ell) on the pairs where the
    expected block norm sqrt(n_ao(I) n_ao(J)) exp(-d0/ell) exceeds theta_d.

    S ~ N(0,1) is drawn for one orientation of every pair, in the sorted order
    of canonical keys (I < J, or I == J with R lexicographically positive);
    the mirror block D_JI(-R) is its transpose and D_II(0) = (S + S^T)/sqrt(2).
    """
    n = species.shape[0]
    na = n_ao[species]
    nmax = float(n_ao.max())
    rcut = ell * math.log(nmax / theta_d)
    Rs = image_range(lattice, rcut)
    RL = Rs @ lattice
    # drop the images whose translated bounding box of the positions lies
    # rcut or farther from the untranslated one (no pair can reach them)
    span = pos.max(0) - pos.min(0)
    gap = np.maximum(np.abs(RL) - span[None, :], 0.0)
    near = (gap * gap).sum(1) < rcut * rcut
    Rs, RL = Rs[near], RL[near]
    canon = []  # (I, J, R1, R2, R3, d0)
    for i in range(n):
        d = pos[None, :, :] + RL[:, None, :] - pos[i][None, None, :]   # [nR, n, 3]
        r = np.sqrt((d * d).sum(-1))
        thr = ell * np.log(np.sqrt(na[i] * na) / theta_d)               # [n]
        keep = r < thr[None, :]
        kr, kj = np.nonzero(keep)
        Rk = Rs[kr]
        # canonical orientation
        lex = (Rk[:, 0] > 0) | ((Rk[:, 0] == 0) & ((Rk[:, 1] > 0) | ((Rk[:, 1] == 0) & (Rk[:, 2] >= 0))))
        c = (kj > i) | ((kj == i) & lex)
        kr, kj, Rk = kr[c], kj[c], Rk[c]
        rv = r[kr, kj]
        canon.append(np.column_stack([np.full(kj.shape, i), kj, Rk, ]).astype(np.int64))
        canon[-1] = (canon[-1], rv)
    keys = np.concatenate([c[0] for c in canon])
    d0 = np.concatenate([c[1] for c in canon])
    order = np.lexsort((keys[:, 4], keys[:, 3], keys[:, 2], keys[:, 1], keys[:, 0]))
    keys, d0 = keys[order], d0[order]
    sizes = na[keys[:, 0]] * na[keys[:, 1]]
    raw = rng.standard_normal(int(sizes.sum()))
    offs = np.concatenate([[0], np.cumsum(sizes)])
    scale = np.array([math.exp(-x / ell) for x in d0.tolist()])

    # Every stored block: the canonical ones and the mirrors D_JI(-R) = D_IJ(R)^T
    # (not of the on-site blocks), in lexicographic order of (I, J, R1, R2, R3).
    onsite = (keys[:, 0] == keys[:, 1]) & ~keys[:, 2:5].any(axis=1)
    mir = np.nonzero(~onsite)[0]
    mkeys = np.column_stack([keys[mir, 1], keys[mir, 0], -keys[mir, 2:5]])
    all_keys = np.concatenate([keys, mkeys])
    src = np.concatenate([np.arange(keys.shape[0]), mir])                 # canonical block of each entry
    trans = np.concatenate([np.zeros(keys.shape[0], bool), np.ones(mir.size, bool)])
    order = np.lexsort(tuple(all_keys[:, c] for c in (4, 3, 2, 1, 0)))
    all_keys, src, trans = all_keys[order], src[order], trans[order]
    esz = na[all_keys[:, 0]] * na[all_keys[:, 1]]
    d_offset = np.zeros(all_keys.shape[0] + 1, dtype=np.int64)
    d_offset[1:] = np.cumsum(esz)
    d_values = np.zeros(int(d_offset[-1]))
    # fill by canonical shape (a, b) and orientation: S from its draws,
    # symmetrised on site, times exp(-d0/ell), transposed for a mirror
    ca, cb = na[keys[src, 0]], na[keys[src, 1]]
    for a in np.unique(ca):
        for b in np.unique(cb):
            for t in (False, True):
                sel_all = np.nonzero((ca == a) & (cb == b) & (trans == t))[0]
                for s0 in range(0, sel_all.size, 65536):   # bounded index arrays
                    sel = sel_all[s0:s0 + 65536]
                    c = src[sel]
                    S_ = raw[offs[c][:, None] + np.arange(a * b)[None, :]].reshape(-1, a, b)
                    on = onsite[c]
                    if on.any():
                        S_[on] = (S_[on] + S_[on].transpose(0, 2, 1)) / math.sqrt(2.0)
                    blk = S_ * scale[c][:, None, None]
                    if t:
                        blk = blk.transpose(0, 2, 1)
                    d_values[d_offset[sel][:, None] + np.arange(a * b)[None, :]] = blk.reshape(sel.size, a * b)
    return all_keys.astype(np.int32), d_offset, d_values


def make_workload(kind: str, n_rep: int, a: float, n_ao: Sequence[int], n_abf: Sequence[int],
                  r_c: float, seed: int, *, strain_amp: float = 0.0, name: str = "",
                  theta: float = DEFAULT_THETA, jitter: float = JITTER_SIGMA) -> Workload:
    """Build one workload.  Draw order from Philox(seed):
    jitter (n_atoms x 3), strain (6, only if strain_amp > 0), G templates
    (s, t order), M templates (per s: X then M_st for t > s), D blocks.
    """
    rng = np.random.Generator(np.random.Philox(seed))
    species, lattice0, frac = _geometry(kind, n_rep, a)
    n_ao = np.asarray(n_ao, dtype=np.int32)
    n_abf = np.asarray(n_abf, dtype=np.int32)
    pos0 = frac @ lattice0 + rng.normal(0.0, jitter, (species.shape[0], 3))
    strain = None
    lattice, pos = lattice0.copy(), pos0.copy()
    if strain_amp > 0:
        u = rng.uniform(-strain_amp, strain_amp, 6)
        strain = np.array([[u[0], u[3], u[4]], [u[3], u[1], u[5]], [u[4], u[5], u[2]]])
        F = np.eye(3) + strain
        lattice = lattice0 @ F.T
        pos = pos0 @ F.T
    G, M = _make_templates(rng, n_ao, n_abf)
    d_index, d_offset, d_values = _make_density(rng, species, lattice0, pos0, n_ao, theta)
    th = dict(C=theta, dC=theta, V=theta, dV=theta, D=theta, CS=theta)
    return Workload(name=name or f"{kind}{n_rep}", species=species, lattice=lattice,
                    positions=np.ascontiguousarray(pos), n_ao=n_ao, n_abf=n_abf, r_c=r_c,
                    omega=OMEGA, G=G, M=M, d_index=d_index, d_offset=d_offset, d_values=d_values,
                    theta=th, seed=seed, strain=strain, lattice0=lattice0, positions0=pos0)


# The workloads: small diamond cell, Si-like supercells and CsSnI3-shaped
# perovskite supercells (shapes of the paper's Si and CsSnI3 systems, Sec. 4).
def diamond8(seed: int = 1, **kw) -> Workload:
    """8-atom diamond cell, a = 5.43 A, n_ao = 4, n_abf = 9, r_c = 2.6 A."""
    return make_workload("diamond", 1, 5.43, [4], [9], 2.6, seed, name="diamond8", **kw)


def si_supercell(n_rep: int, seed: int = 2, strain_amp: float = 0.0, **kw) -> Workload:
    """n_rep^3 diamond supercell, n_ao = 13 (2s2p1d), n_abf = 50, r_c = 3.7 A."""
    return make_workload("diamond", n_rep, 5.43, [13], [50], 3.7, seed, strain_amp=strain_amp,
                         name=f"si{8 * n_rep ** 3}", **kw)


def perovskite_supercell(n_rep: int, seed: int = 3, strain_amp: float = 0.0, **kw) -> Workload:
    """n_rep^3 CsSnI3-shaped cubic perovskite, a = 6.2 A; n_ao 18/13/13 and
    n_abf 75/60/60 for Cs/Sn/I; r_c = 4.2 A."""
    return make_workload("perovskite", n_rep, 6.2, [18, 13, 13], [75, 60, 60], 4.2, seed,
                         strain_amp=strain_amp, name=f"perovskite{5 * n_rep ** 3}", **kw)


def tiny_model(n_ao: Sequence[int], n_abf: Sequence[int], species: Sequence[int], lattice, positions,
               r_c: float, seed: int, theta: float = DEFAULT_THETA) -> Workload:
    """Arbitrary small structure with random templates (used for brute-force
    and finite-difference checks on a handful of atoms)."""
    rng = np.random.Generator(np.random.Philox(seed))
    species = np.asarray(species, dtype=np.int32)
    lattice = np.asarray(lattice, dtype=np.float64)
    pos = np.asarray(positions, dtype=np.float64)
    n_ao = np.asarray(n_ao, dtype=np.int32)
    n_abf = np.asarray(n_abf, dtype=np.int32)
    G, M = _make_templates(rng, n_ao, n_abf)
    d_index, d_offset, d_values = _make_density(rng, species, lattice, pos, n_ao, theta)
    th = dict(C=theta, dC=theta, V=theta, dV=theta, D=theta, CS=theta)
    return Workload(name="tiny", species=species, lattice=lattice, positions=pos, n_ao=n_ao,
                    n_abf=n_abf, r_c=r_c, omega=OMEGA, G=G, M=M, d_index=d_index,
                    d_offset=d_offset, d_values=d_values, theta=th, seed=seed,
                    lattice0=lattice.copy(), positions0=pos.copy())


def cut_density(w: Workload, rmax: float) -> Workload:
    """Drop D blocks whose initial pair distance is >= rmax (keeps both
    orientations together).  Used to make small brute-force cases cheap."""
    pos0 = w.positions0 if w.positions0 is not None else w.positions
    lat0 = w.lattice0 if w.lattice0 is not None else w.lattice
    i, j = w.d_index[:, 0], w.d_index[:, 1]
    d = pos0[j] + w.d_index[:, 2:5].astype(np.float64) @ lat0 - pos0[i]
    keep = np.sqrt((d * d).sum(1)) < rmax
    idx = np.nonzero(keep)[0]
    sizes = (w.d_offset[1:] - w.d_offset[:-1])[idx]
    off = np.zeros(idx.size + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    vals = np.concatenate([w.d_values[w.d_offset[k]:w.d_offset[k + 1]] for k in idx]) if idx.size else np.zeros(0)
    out = dataclasses.replace(w)
    out.d_index = np.ascontiguousarray(w.d_index[idx])
    out.d_offset = off
    out.d_values = vals
    return out


def geometry_sequence(w: Workload, n: int, seed: int = 17, amp: float = 0.01) -> List[np.ndarray]:
    """n seeded small displacements of w's positions (Gaussian, amp Angstrom
    per coordinate): a relaxation-like sequence that stays within the pair
    lists' skin."""
    rng = np.random.Generator(np.random.Philox(seed))
    return [w.positions + rng.normal(0.0, amp, w.positions.shape) for _ in range(n)]


def lri_pairs(batch: int, m_i: int, m_k: int, n_i: int, n_k: int, seed: int = 5, r_range=(1.8, 4.0)):
    """Synthetic inputs of the LRI fit for `batch` pairs (I, K) of one
    species pair: per pair a random separation vector d (|d| uniform in
    r_range) and the blocks of a smooth model with their exact derivatives
    in d (the position of K):
        A(d)  = [[M_II, s(r) M_IK], [s(r) M_IK^T, M_KK]]
        B(d)  = [[T_I t1(r)], [T_K t2(r)]]
    with M_ss = X X^T / m + 1 (SPD), M_IK ~ N(0,1)/sqrt(m_i), T ~ N(0,1),
    s(r) = 0.3 exp(-r^2/8), t1(r) = exp(-r^2/6), t2(r) = (1 + 0.2 r) exp(-r^2/5).
    Returns (d [batch, 3], A, B, dA [batch, 3, n, n], dB [batch, 3, n, w],
    templates) where templates rebuild A, B at any d via lri_blocks."""
    rng = np.random.Generator(np.random.Philox(seed))
    Xi = rng.standard_normal((m_i, m_i))
    Xk = rng.standard_normal((m_k, m_k))
    tpl = {"M_II": Xi @ Xi.T / m_i + np.eye(m_i), "M_KK": Xk @ Xk.T / m_k + np.eye(m_k),
           "M_IK": rng.standard_normal((m_i, m_k)) / math.sqrt(m_i),
           "T_I": rng.standard_normal((m_i, n_i * n_k)), "T_K": rng.standard_normal((m_k, n_i * n_k))}
    u = rng.standard_normal((batch, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    d = u * rng.uniform(r_range[0], r_range[1], (batch, 1))
    blocks = [lri_blocks(tpl, d[p]) for p in range(batch)]
    A, B, dA, dB = (np.stack([b[k] for b in blocks]) for k in range(4))
    return d, A, B, dA, dB, tpl


def lri_blocks(tpl: dict, d: np.ndarray):
    """A, B, dA, dB of the lri_pairs model at separation d (3,)."""
    d = np.asarray(d, np.float64)
    r = float(np.linalg.norm(d))
    s = 0.3 * math.exp(-r * r / 8.0)
    ds = -r / 4.0 * s
    t1 = math.exp(-r * r / 6.0)
    dt1 = -r / 3.0 * t1
    e2 = math.exp(-r * r / 5.0)
    t2 = (1.0 + 0.2 * r) * e2
    dt2 = 0.2 * e2 - (1.0 + 0.2 * r) * (2.0 * r / 5.0) * e2
    mi, mk = tpl["M_II"].shape[0], tpl["M_KK"].shape[0]
    n = mi + mk
    A = np.zeros((n, n))
    A[:mi, :mi] = tpl["M_II"]
    A[mi:, mi:] = tpl["M_KK"]
    A[:mi, mi:] = s * tpl["M_IK"]
    A[mi:, :mi] = s * tpl["M_IK"].T
    B = np.concatenate([tpl["T_I"] * t1, tpl["T_K"] * t2])
    dA = np.zeros((3, n, n))
    dB = np.zeros((3, n, B.shape[1]))
    for c in range(3):
        g = d[c] / r
        dA[c, :mi, mi:] = ds * g * tpl["M_IK"]
        dA[c, mi:, :mi] = ds * g * tpl["M_IK"].T
        dB[c] = np.concatenate([tpl["T_I"] * dt1 * g, tpl["T_K"] * dt2 * g])
    return A, B, dA, dB


def workload_by_name(name: str) -> Workload:
    table = {
        "diamond8": lambda: diamond8(),
        "si64": lambda: si_supercell(2),
        "perovskite320": lambda: perovskite_supercell(4),
        "si1000": lambda: si_supercell(5, seed=4, strain_amp=0.03),
        "perovskite1080": lambda: perovskite_supercell(6, seed=5, strain_amp=0.03),
    }
    return table[name]()
