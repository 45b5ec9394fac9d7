"""Plain FP64 CPU oracle for the HFX force and stress under LRI.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module; only the tests, the package smoke check and the
benchmark's CPU-baseline leg do.  It shares no code with the CUDA path.

What it computes (paper Sec. 2)
-------------------------------
With real D and one atom A fixed in the home cell (N_k = 1 per cell), the
exchange energy of Eq. exx_expand is

    E = - sum_{A in cell} sum_{F,B,G (all images)} sum_{a f b g alpha beta}
          C^A_{AF}[alpha,a,f] V_{AB}[alpha,beta] C^B_{BG}[beta,b,g]
          ( D_AB[a,b] D_FG[f,g] + D_AG[a,g] D_FB[f,b] )

The force part F^X1 (Eq. Fexx1) and the stress part sigma^X1 (Eq. stress)
are the derivatives of E through the C and V blocks only (D held fixed).
Every block depends on its pair vector d = tau_J + R L - tau_I, so both
follow from the pair gradients g_p = dE/dd_p:

    F_I += g_p,  F_J -= g_p        for every pair p = (I -> J, R)
    sigma = -(1/Omega) sum_p g_p (x) d_p

Screening (Sec. 3.2 and Algorithm 1) is an approximation; the oracle takes
its two steps in the paper's order:
  step 1  per-tensor block filter on Frobenius norms (C with grad C jointly,
          V with grad V jointly, D);
  step 2  Cauchy-Schwarz bound on each item before it is contracted.
An item of the first exchange product is an (A, B, F) triplet summed over G,
an item of the second product is an (A, B) pair summed over F and G.

The sums over G and F are taken in the order of the distributive law, with
library matmuls as steps (each step names the formula it evaluates):
  Y^{XZ}[alpha,x,z] = sum_W sum_w C_XW[alpha,x,w] D_WZ[w,z]
  term 1, per kept (A,B,F):  U = D_AB . Y^{BF} (over b);
      R1_AB += <C_AF, U> (over a,f);   Q_AF += V_AB . U (over beta)
  term 2, per kept (A,B):    R2_AB = <Y^{AB}, Y^{BA}> (over a,b);
      Z = V_AB . Y^{BA};  Q_AF += Z . D_FB^T (over b) for F next to A
  E = -sum <V, R1 + R2>,  g^V = -<grad V, R1 + R2>,  g^C = -2 <grad C, Q>
The factor 2 in g^C is the C_BG slot of Eq. Fexx1 (its last two lines),
which is the mirror image of the C_AF slot (first two lines) under the
relabelling (A,F) <-> (B,G) that leaves Eq. exx_expand unchanged.  Under
triplet screening the mirror slot is screened by the mirrored rule, as
the paper screens each force term with its own loop (Sec. 3.2).

The block model (the stand-in for the NAO/ABF integrals of Sec. 3.1):
  C_{I,(J,R)} = G_{s(I)s(J)} f(r),   f(r) = (1-(r/R_C)^2)^3 exp(-r^2/2), r<R_C
  V_{I,(J,R)} = M_{s(I)s(J)} h(r),   h(r) = erfc(omega r)/(r+1)
  with R_C = 2 r_c; on-site blocks (I = J, R = 0) do not move (grad = 0,
  Sec. 3.1).  An optional anisotropic term C += G'_{st} f(r) (d.e)/R_C makes
  grad C a general 3-component block.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np
from scipy.special import erfc

SQRT_PI = math.sqrt(math.pi)


# --------------------------------------------------------------------------
# Radial functions of the block model and their derivatives (written out by
# hand; pinned against finite differences and sympy in the tests).
# --------------------------------------------------------------------------
def radial_f(r, RC):
    r = np.asarray(r, dtype=np.float64)
    x = 1.0 - (r / RC) ** 2
    return np.where(r < RC, x ** 3 * np.exp(-0.5 * r * r), 0.0)


def radial_df(r, RC):
    r = np.asarray(r, dtype=np.float64)
    x = 1.0 - (r / RC) ** 2
    e = np.exp(-0.5 * r * r)
    val = 3.0 * x * x * (-2.0 * r / (RC * RC)) * e - r * x ** 3 * e
    return np.where(r < RC, val, 0.0)


def radial_h(r, omega):
    r = np.asarray(r, dtype=np.float64)
    return erfc(omega * r) / (r + 1.0)


def radial_dh(r, omega):
    r = np.asarray(r, dtype=np.float64)
    return (-2.0 * omega / SQRT_PI) * np.exp(-(omega * r) ** 2) / (r + 1.0) - erfc(omega * r) / (r + 1.0) ** 2


def image_vectors(lattice, rmax):
    """All integer R such that some pair of atoms in the cell can lie within rmax."""
    recip = np.linalg.inv(lattice).T
    nmax = [int(math.ceil(rmax * np.linalg.norm(recip[k]))) + 1 for k in range(3)]
    rr = [np.arange(-n, n + 1) for n in nmax]
    return np.stack(np.meshgrid(*rr, indexing="ij"), axis=-1).reshape(-1, 3).astype(np.int64)


def neighbours(lattice, positions, i, rmax, Rs=None):
    """Pairs (i -> j, R) with |tau_j + R L - tau_i| < rmax (Eqs. 1-2 labels)."""
    if Rs is None:
        Rs = image_vectors(lattice, rmax)
    RL = Rs @ lattice
    d = positions[None, :, :] + RL[:, None, :] - positions[i][None, None, :]
    r = np.sqrt((d * d).sum(-1))
    kr, kj = np.nonzero(r < rmax)
    order = np.lexsort((Rs[kr, 2], Rs[kr, 1], Rs[kr, 0], kj))
    kr, kj = kr[order], kj[order]
    return kj.astype(np.int64), Rs[kr], d[kr, kj], r[kr, kj]


@dataclass
class Options:
    theta_C: float = 1e-10
    theta_dC: float = 1e-10
    theta_V: float = 1e-10
    theta_dV: float = 1e-10
    theta_D: float = 1e-10
    theta_CS: float = 1e-10
    terms: int = 3                      # bit0: D_AB D_FG product, bit1: D_AG D_FB product
    aniso: Optional[Tuple[list, np.ndarray]] = None   # (G' templates, unit vector e)

    @classmethod
    def from_theta(cls, th: Dict[str, float], **kw):
        return cls(theta_C=th["C"], theta_dC=th["dC"], theta_V=th["V"], theta_dV=th["dV"],
                   theta_D=th["D"], theta_CS=th["CS"], **kw)


@dataclass
class Result:
    E: float
    F: np.ndarray
    sigma: np.ndarray
    counts: Dict[str, int] = field(default_factory=dict)
    flops: float = 0.0


def _key(j, R):
    return (int(j), int(R[0]), int(R[1]), int(R[2]))


class OraclePlan:
    """Pair lists and (optionally frozen) screening decisions for one structure.

    freeze=True records every screening decision at the construction
    geometry and reuses it at later geometries; this makes E a smooth
    function of the positions so that finite differences of E can be
    compared with F and sigma.
    """

    def __init__(self, w, opts: Optional[Options] = None, freeze: bool = False):
        self.w = w
        self.opts = opts or Options.from_theta(w.theta)
        self.freeze = freeze
        self.N = int(w.species.shape[0])
        self.sp = np.asarray(w.species)
        self.n_ao = np.asarray(w.n_ao)
        self.n_abf = np.asarray(w.n_abf)
        self.S = int(self.n_ao.shape[0])
        self.RC = 2.0 * w.r_c
        # D blocks by key (I, J, R1, R2, R3); D_JI(-R) = D_IJ(R)^T is in the input.
        self.D: Dict[tuple, np.ndarray] = {}
        self.Dnorm: Dict[tuple, float] = {}
        for k in range(w.d_index.shape[0]):
            i, j = int(w.d_index[k, 0]), int(w.d_index[k, 1])
            blk = w.d_values[w.d_offset[k]:w.d_offset[k + 1]].reshape(self.n_ao[self.sp[i]], self.n_ao[self.sp[j]])
            key = (i, j, int(w.d_index[k, 2]), int(w.d_index[k, 3]), int(w.d_index[k, 4]))
            self.D[key] = blk
            self.Dnorm[key] = float(np.sqrt((blk * blk).sum()))
        self.Dlist: Dict[int, List[tuple]] = {i: [] for i in range(self.N)}
        for key in self.D:
            self.Dlist[key[0]].append(key)
        self.frozen = None
        if freeze:
            self.frozen = self._evaluate(w.lattice, w.positions, record=True)[1]

    # ---------------------------------------------------------------- blocks
    def _c_blocks(self, i, js, Rs, ds, rs):
        """C and grad_d C for pairs (i -> j, R) (Sec. 3.1 block model)."""
        S, RC = self.S, self.RC
        Cs, dCs = [], []
        for j, R, d, r in zip(js, Rs, ds, rs):
            G = self.w.G[self.sp[i] * S + self.sp[j]]
            onsite = (j == i) and not np.any(R)
            if onsite:
                C = G * 1.0
                dC = np.zeros((3,) + G.shape)
            else:
                f = float(radial_f(r, RC))
                fp = float(radial_df(r, RC))
                C = G * f
                dC = G[None] * (fp * d / r)[:, None, None, None]
            if self.opts.aniso is not None and not onsite:
                Gp_list, e = self.opts.aniso
                Gp = Gp_list[self.sp[i] * S + self.sp[j]]
                f = float(radial_f(r, RC))
                fp = float(radial_df(r, RC))
                de = float(d @ e)
                C = C + Gp * (f * de / RC)
                grad = (fp * (d / r) * de + f * e) / RC
                dC = dC + Gp[None] * grad[:, None, None, None]
            Cs.append(C)
            dCs.append(dC)
        return Cs, dCs

    def _v_block(self, i, j, R, d, r):
        M = self.w.M[self.sp[i] * self.S + self.sp[j]]
        if j == i and not np.any(R):
            return M * 1.0, np.zeros((3,) + M.shape)
        h = float(radial_h(r, self.w.omega))
        hp = float(radial_dh(r, self.w.omega))
        return M * h, M[None] * (hp * d / r)[:, None, None]

    def _v_radius(self):
        """Radius beyond which every V block is below both thresholds.
        h and |h'| decrease monotonically, so bisection on the largest
        template norm gives it."""
        tv, tdv = self.opts.theta_V, self.opts.theta_dV
        mmax = max(float(np.linalg.norm(M)) for M in self.w.M)
        if tv <= 0 and tdv <= 0:
            return math.inf

        def above(r):
            return (mmax * radial_h(r, self.w.omega) > tv) or (mmax * abs(radial_dh(r, self.w.omega)) > tdv)
        lo, hi = 0.0, 1.0
        while above(hi):
            hi *= 2.0
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if above(mid) else (lo, mid)
        return hi + 1.0

    # ------------------------------------------------------------- evaluate
    def evaluate(self, lattice=None, positions=None, homes=None) -> Result:
        """E, F and sigma at the given geometry.  `homes` restricts the sum
        over the home-cell atom A of Eq. exx_expand to a subset (the result is
        then that subset's share; used to time a bounded sample)."""
        lattice = self.w.lattice if lattice is None else np.asarray(lattice, dtype=np.float64)
        positions = self.w.positions if positions is None else np.asarray(positions, dtype=np.float64)
        return self._evaluate(lattice, positions, record=False, homes=homes)[0]

    def _evaluate(self, lattice, positions, record, homes=None):
        o, N, sp, na, nb = self.opts, self.N, self.sp, self.n_ao, self.n_abf
        fr = self.frozen
        Dn = self.Dnorm
        homes = list(range(N)) if homes is None else [int(a) for a in homes]
        flops = [0.0]

        # Atoms with images are labelled relative to a home atom by an integer
        # code of (j, R); lookups in per-atom tables are then sorted searches.
        OFF, K = 64, 129

        def code(j, R):
            R = np.asarray(R, dtype=np.int64).reshape(-1, 3)
            return (((R[:, 0] + OFF) * K + (R[:, 1] + OFF)) * K + (R[:, 2] + OFF)) * N + np.asarray(j, np.int64)

        def lookup(table, q):
            keys, vals = table
            if keys.size == 0:
                return np.zeros(q.shape)
            idx = np.minimum(np.searchsorted(keys, q), keys.size - 1)
            return np.where(keys[idx] == q, vals[idx], 0.0)

        # D kept (step 1): ||D|| > theta_D
        def dnorm(key):
            v = Dn.get(key, 0.0)
            return v if v > o.theta_D else 0.0

        # ---- C pairs: all (A -> F) within R_C (f vanishes beyond it)
        Rs_c = image_vectors(lattice, self.RC)
        Cl = []
        for A in range(N):
            if fr is None:
                js, Rs, ds, rs = neighbours(lattice, positions, A, self.RC, Rs_c)
            else:
                js, Rs = fr["C_js"][A], fr["C_Rs"][A]
                ds = positions[js] + Rs @ lattice - positions[A]
                rs = np.sqrt((ds * ds).sum(1))
            Cs, dCs = self._c_blocks(A, js, Rs, ds, rs)
            nC = np.array([np.sqrt((c * c).sum()) for c in Cs])
            ndC = np.array([np.sqrt((g * g).sum()) for g in dCs])
            keep = (nC > o.theta_C) | (ndC > o.theta_dC) if fr is None else fr["C_keep"][A]
            cn = np.where(keep, np.maximum(nC, ndC), 0.0)
            Cl.append(dict(js=js, Rs=Rs, ds=ds, C=Cs, dC=dCs, keep=keep, c=cn))

        # ---- yhat_{XZ} = sum_{W in C(X)} c_XW d_WZ  (CS factor of Sec. 3.2)
        Dl = []   # per atom W: its D blocks as arrays (z, R, kept norm)
        for i in range(N):
            keys = self.Dlist[i]
            if keys:
                ka = np.array(keys, dtype=np.int64)
                dv = np.array([dnorm(k) for k in keys])
            else:
                ka, dv = np.zeros((0, 5), np.int64), np.zeros(0)
            Dl.append((ka, dv))
        yhat = []
        for X in range(N):
            L = Cl[X]
            cc, ww = [], []
            for q in np.nonzero(L["keep"])[0]:
                ka, dv = Dl[int(L["js"][q])]
                m = dv > 0.0
                cc.append(code(ka[m, 1], ka[m, 2:5] + L["Rs"][q][None, :]))
                ww.append(L["c"][q] * dv[m])
            if cc:
                u, inv = np.unique(np.concatenate(cc), return_inverse=True)
                yhat.append((u, np.bincount(inv, weights=np.concatenate(ww))))
            else:
                yhat.append((np.zeros(0, np.int64), np.zeros(0)))

        # ---- V pairs: candidates within the V radius and within reach of a
        #      nonzero product (D list for term 1, R_C + D reach for term 2)
        rd = 0.0
        for k in self.D:
            dv = positions[k[1]] + np.array(k[2:5], dtype=np.float64) @ lattice - positions[k[0]]
            rd = max(rd, float(np.sqrt(dv @ dv)))
        rv = min(self._v_radius(), self.RC + rd + 1.0)
        Rs_v = image_vectors(lattice, rv)
        Vl = []
        for A in range(N):
            if fr is None:
                js, Rs, ds, rs = neighbours(lattice, positions, A, rv, Rs_v)
            else:
                js, Rs = fr["V_js"][A], fr["V_Rs"][A]
                ds = positions[js] + Rs @ lattice - positions[A]
                rs = np.sqrt((ds * ds).sum(1))
            nV, ndV = self._v_norms(A, js, Rs, ds, rs)
            keep = (nV > o.theta_V) | (ndV > o.theta_dV) if fr is None else fr["V_keep"][A]
            vn = np.where(keep, np.maximum(nV, ndV), 0.0)
            Vl.append(dict(js=js, Rs=Rs, ds=ds, rs=rs, keep=keep, v=vn))

        # ---- step 2: Cauchy-Schwarz screening of items
        trip = [[] for _ in range(N)]   # per A: (qV, array of qC)
        pair2 = [[] for _ in range(N)]  # per A: qV
        for A in homes:
            LV, LC = Vl[A], Cl[A]
            kC = np.nonzero(LC["keep"])[0]
            for qv in np.nonzero(LV["keep"])[0]:
                b, Rb = int(LV["js"][qv]), LV["Rs"][qv]
                v = LV["v"][qv]
                if o.terms & 1:
                    dab = dnorm((A, b, int(Rb[0]), int(Rb[1]), int(Rb[2])))
                    if dab > 0.0:
                        if fr is None:
                            yq = lookup(yhat[b], code(LC["js"][kC], LC["Rs"][kC] - Rb[None, :]))
                            bound = LC["c"][kC] * v * dab * yq      # c_AF v_AB d_AB yhat_BF
                            fs = kC[bound > o.theta_CS]
                        else:
                            fs = np.asarray(fr["trip"][A].get(int(qv), []), dtype=np.int64)
                        if fs.size:
                            trip[A].append((int(qv), fs))
                if o.terms & 2:
                    if fr is None:
                        w1 = lookup(yhat[A], code([b], Rb[None, :]))[0]
                        w2 = lookup(yhat[b], code([A], -Rb[None, :]))[0]
                        ok = v * w1 * w2 > o.theta_CS                # v_AB yhat_AB yhat_BA
                    else:
                        ok = int(qv) in fr["pair2"][A]
                    if ok:
                        pair2[A].append(int(qv))

        # ---- Y^{XZ} = sum_W C_XW D_WZ over kept C and kept D, for every key
        #      the kept items need (one library matmul per home atom X: its
        #      kept C_XW side by side, times the D_WZ blocks stacked by key)
        need = [set() for _ in range(N)]
        for A in homes:
            LV, LC = Vl[A], Cl[A]
            for (qv, fs) in trip[A]:
                b, Rb = int(LV["js"][qv]), LV["Rs"][qv]
                for qc in fs:
                    need[b].add((int(LC["js"][qc]),) + tuple(int(x) for x in LC["Rs"][qc] - Rb))
            for qv in pair2[A]:
                b, Rb = int(LV["js"][qv]), LV["Rs"][qv]
                need[A].add((b,) + tuple(int(x) for x in Rb))
                need[b].add((A,) + tuple(-int(x) for x in Rb))
        Ytab: Dict[tuple, np.ndarray] = {}
        for X in range(N):
            if not need[X]:
                continue
            L = Cl[X]
            kq = np.nonzero(L["keep"])[0]
            nx, mx = na[sp[X]], nb[sp[X]]
            Cx = np.concatenate([L["C"][q].reshape(mx * nx, -1) for q in kq], axis=1)   # [(alpha,x),(W,w)]
            woff = np.concatenate([[0], np.cumsum([na[sp[int(L["js"][q])]] for q in kq])])
            keys = sorted(need[X])
            zoff = np.concatenate([[0], np.cumsum([na[sp[k[0]]] for k in keys])])
            Dg = np.zeros((woff[-1], zoff[-1]))                                      # [(W,w),(Z,z)]
            for kk, zk in enumerate(keys):
                for t, q in enumerate(kq):
                    w_, Rw = int(L["js"][q]), L["Rs"][q]
                    dk = (w_, zk[0], zk[1] - int(Rw[0]), zk[2] - int(Rw[1]), zk[3] - int(Rw[2]))
                    if dnorm(dk) > 0.0:
                        Dg[woff[t]:woff[t + 1], zoff[kk]:zoff[kk + 1]] = self.D[dk]
                        flops[0] += 2.0 * mx * nx * na[sp[w_]] * na[sp[zk[0]]]
            Yx = Cx @ Dg                                                             # contract (W, w)
            for kk, zk in enumerate(keys):
                Ytab[(X,) + zk] = Yx[:, zoff[kk]:zoff[kk + 1]].reshape(mx, nx, -1)

        def Y(x, zk):
            return Ytab[(x,) + tuple(int(v) for v in zk)]

        # ---- contraction
        R_acc = [dict() for _ in range(N)]   # qv -> R_AB (n_abf(A) x n_abf(B))
        Q_acc = [dict() for _ in range(N)]   # qc -> Q_AF (shape of C_AF)

        def addQ(A, qc, Qt):
            if qc in Q_acc[A]:
                Q_acc[A][qc] += Qt
            else:
                Q_acc[A][qc] = Qt.copy()

        for A in homes:
            LC, LV = Cl[A], Vl[A]
            sA = sp[A]
            for (qv, fs) in trip[A]:
                b, Rb = int(LV["js"][qv]), LV["Rs"][qv]
                Vb, _ = self._v_block(A, b, Rb, LV["ds"][qv], LV["rs"][qv])
                Dab = self.D[(A, b, int(Rb[0]), int(Rb[1]), int(Rb[2]))]
                Racc = R_acc[A].setdefault(qv, np.zeros((nb[sA], nb[sp[b]])))
                # the F of one item list, grouped by species so blocks stack
                for s_f in np.unique(sp[LC["js"][fs]]):
                    fsg = fs[sp[LC["js"][fs]] == s_f]
                    Cst = np.stack([LC["C"][qc] for qc in fsg])                          # [F, alpha, a, f]
                    Yst = np.stack([Y(b, (int(LC["js"][qc]),) + tuple(LC["Rs"][qc] - Rb)) for qc in fsg])
                    U = np.matmul(Dab, Yst)                      # U[F,beta,a,f] = sum_b D_AB[a,b] Y^{BF}[beta,b,f]
                    Racc += np.einsum("Fxaf,Fyaf->xy", Cst, U, optimize=True)   # R1_AB += sum_{F,a,f} C_AF U
                    Qt = np.matmul(Vb, U.reshape(U.shape[0], U.shape[1], -1)).reshape(Cst.shape)  # V_AB . U
                    for k, qc in enumerate(fsg):
                        addQ(A, int(qc), Qt[k])
                    flops[0] += fsg.size * (2.0 * nb[sp[b]] * na[sA] * na[sp[b]] * na[s_f]
                                            + 4.0 * nb[sA] * nb[sp[b]] * na[sA] * na[s_f])
            kC = np.nonzero(LC["keep"])[0]
            for qv in pair2[A]:
                b, Rb = int(LV["js"][qv]), LV["Rs"][qv]
                Vb, _ = self._v_block(A, b, Rb, LV["ds"][qv], LV["rs"][qv])
                Yab = Y(A, (b,) + tuple(Rb))
                Yba = Y(b, (A,) + tuple(-Rb))
                R2 = np.einsum("xab,yba->xy", Yab, Yba, optimize=True)        # R2 = <Y^{AB}, Y^{BA}>
                Z = np.einsum("xy,yba->xab", Vb, Yba, optimize=True)          # Z[alpha,a,b] = (V_AB . Y^{BA})
                if qv in R_acc[A]:
                    R_acc[A][qv] += R2
                else:
                    R_acc[A][qv] = R2
                flops[0] += 4.0 * R2.size * Yab.shape[1] * Yab.shape[2]
                for qc in kC:
                    f, Rf = int(LC["js"][qc]), LC["Rs"][qc]
                    dk = (f, b, int(Rb[0] - Rf[0]), int(Rb[1] - Rf[1]), int(Rb[2] - Rf[2]))
                    if dnorm(dk) == 0.0:
                        continue
                    addQ(A, int(qc), Z @ self.D[dk].T)                       # Q_AF += sum_b Z[.,.,b] D_FB[f,b]
                    flops[0] += 2.0 * Z.size * na[sp[f]]

        # ---- energy, pair gradients, forces and stress
        E = 0.0
        E_via_Q = 0.0     # -sum <C_AF, Q_AF>: the same energy from the C side
        F = np.zeros((N, 3))
        W = np.zeros((3, 3))
        for A in homes:
            LV, LC = Vl[A], Cl[A]
            for qv, Racc in R_acc[A].items():
                b, Rb = int(LV["js"][qv]), LV["Rs"][qv]
                Vb, dVb = self._v_block(A, b, Rb, LV["ds"][qv], LV["rs"][qv])
                E -= float((Vb * Racc).sum())
                g = -np.einsum("cxy,xy->c", dVb, Racc)
                F[A] += g
                F[b] -= g
                W += np.outer(g, LV["ds"][qv])
            for qc, Q in Q_acc[A].items():
                f = int(LC["js"][qc])
                E_via_Q -= float((LC["C"][qc] * Q).sum())
                g = -2.0 * np.einsum("cxaf,xaf->c", LC["dC"][qc], Q)
                F[A] += g
                F[f] -= g
                W += np.outer(g, LC["ds"][qc])
        omega_cell = abs(float(np.linalg.det(lattice)))
        sigma = -W / omega_cell
        counts = dict(
            c_pairs=int(sum(int(Cl[A]["keep"].sum()) for A in homes)),
            v_pairs=int(sum(int(Vl[A]["keep"].sum()) for A in homes)),
            triplets=int(sum(fs.size for A in homes for (_, fs) in trip[A])),
            term1_pairs=int(sum(len(trip[A]) for A in homes)),
            term2_pairs=int(sum(len(pair2[A]) for A in homes)),
            y_blocks=len(Ytab),
            E_via_Q=E_via_Q,
        )
        res = Result(E=E, F=F, sigma=sigma, counts=counts, flops=flops[0])
        rec = None
        if record:
            rec = dict(C_js=[L["js"] for L in Cl], C_Rs=[L["Rs"] for L in Cl],
                       C_keep=[L["keep"] for L in Cl],
                       V_js=[L["js"] for L in Vl], V_Rs=[L["Rs"] for L in Vl],
                       V_keep=[L["keep"] for L in Vl],
                       trip=[{qv: fs for (qv, fs) in t} for t in trip],
                       pair2=[set(p) for p in pair2])
        return res, rec

    def _v_norms(self, A, js, Rs, ds, rs):
        """Frobenius norms of V and grad V for the candidate pairs of A,
        taken over the blocks themselves (built in chunks)."""
        nV = np.zeros(js.shape[0])
        ndV = np.zeros(js.shape[0])
        for q0 in range(0, js.shape[0], 256):
            for q in range(q0, min(q0 + 256, js.shape[0])):
                V, dV = self._v_block(A, int(js[q]), Rs[q], ds[q], rs[q])
                nV[q] = np.sqrt((V * V).sum())
                ndV[q] = np.sqrt((dV * dV).sum())
        return nV, ndV


def evaluate(w, opts: Optional[Options] = None) -> Result:
    """E, F, sigma of workload `w` with the screening of `opts` (defaults to
    the workload's thresholds)."""
    return OraclePlan(w, opts).evaluate()
