"""Brute-force quartet sum for tiny structures (TEST INFRASTRUCTURE ONLY).

A literal loop over the atom quartets (A, F, B, G) of Eq. exx_expand, with
every index sum written as one einsum per item and no screening (every
nonzero block enters).  The force is the literal six-term Eq. Fexx1 and the
stress the literal three-term Eq. stress: for each item, the derivative of
the item through each of its three position-dependent blocks (C_AF, V_AB,
C_BG) is taken separately and assigned to the two atoms of that block.  No
intermediate (Y, U, R, Q) and no symmetry factor is used, so this pins the
factorised oracle's contraction order, its factor 2 and the wiring of the
second exchange product.

It builds its own neighbour lists and blocks from the block model; only the
radial functions are shared with the factorised oracle, and those are
pinned separately against finite differences and a symbolic derivative.
"""
from __future__ import annotations

import numpy as np

from .hfx_oracle import image_vectors, radial_df, radial_dh, radial_f, radial_h


def _blocks(w, i, j, d, r, RC, aniso=None):
    S = w.n_ao.shape[0]
    si, sj = int(w.species[i]), int(w.species[j])
    G = w.G[si * S + sj]
    M = w.M[si * S + sj]
    onsite = r == 0.0
    if onsite:
        C, dC = G * 1.0, np.zeros((3,) + G.shape)
        V, dV = M * 1.0, np.zeros((3,) + M.shape)
        return C, dC, V, dV
    f, fp = float(radial_f(r, RC)), float(radial_df(r, RC))
    h, hp = float(radial_h(r, w.omega)), float(radial_dh(r, w.omega))
    C = G * f
    dC = np.einsum("c,xab->cxab", fp * d / r, G)
    if aniso is not None:
        Gp, e = aniso[0][si * S + sj], aniso[1]
        C = C + Gp * (f * float(d @ e) / RC)
        dC = dC + np.einsum("c,xab->cxab", (fp * (d / r) * float(d @ e) + f * e) / RC, Gp)
    V = M * h
    dV = np.einsum("c,xy->cxy", hp * d / r, M)
    return C, dC, V, dV


def brute_force(w, terms: int = 3, aniso=None):
    """Return (E, F, sigma) by the literal quartet sum (no screening)."""
    N = int(w.species.shape[0])
    L, P = np.asarray(w.lattice), np.asarray(w.positions)
    RC = 2.0 * w.r_c
    Dm = {}
    for k in range(w.d_index.shape[0]):
        i, j = int(w.d_index[k, 0]), int(w.d_index[k, 1])
        Dm[(i, j) + tuple(int(x) for x in w.d_index[k, 2:5])] = \
            w.d_values[w.d_offset[k]:w.d_offset[k + 1]].reshape(int(w.n_ao[w.species[i]]), int(w.n_ao[w.species[j]]))
    rd = 0.0
    for key in Dm:
        dv = P[key[1]] + np.array(key[2:5], float) @ L - P[key[0]]
        rd = max(rd, float(np.linalg.norm(dv)))
    rB = RC + rd + 1e-9
    RsC = image_vectors(L, RC)
    RsB = image_vectors(L, rB)

    def pos(j, R):
        return P[j] + np.asarray(R, float) @ L

    def around(x, Rx, rmax, Rs):
        """Atoms (j, R) within rmax of atom (x, Rx)."""
        out = []
        px = pos(x, Rx)
        for R in Rs:
            for j in range(N):
                RR = (Rx[0] + int(R[0]), Rx[1] + int(R[1]), Rx[2] + int(R[2]))
                d = pos(j, RR) - px
                if float(np.linalg.norm(d)) < rmax:
                    out.append((j, RR))
        return out

    def D(X, Y):
        key = (X[0], Y[0], Y[1][0] - X[1][0], Y[1][1] - X[1][1], Y[1][2] - X[1][2])
        return Dm.get(key)

    def blk(X, Y):
        d = pos(Y[0], Y[1]) - pos(X[0], X[1])
        r = float(np.linalg.norm(d))
        if r == 0.0 and not (X[0] == Y[0]):
            raise ValueError("coincident atoms")
        return d, r, _blocks(w, X[0], Y[0], d, r, RC, aniso)

    E = 0.0
    F = np.zeros((N, 3))
    Wv = np.zeros((3, 3))
    for a in range(N):
        A = (a, (0, 0, 0))
        Fs = [X for X in around(a, A[1], RC, RsC)]
        Bs = around(a, A[1], rB, RsB)
        for Fq in Fs:
            dAF, rAF, (CAF, dCAF, _, _) = blk(A, Fq)
            if rAF >= RC:
                continue
            for Bq in Bs:
                dAB, rAB, (_, _, VAB, dVAB) = blk(A, Bq)
                Gs = around(Bq[0], Bq[1], RC, RsC)
                for Gq in Gs:
                    dBG, rBG, (CBG, dCBG, _, _) = blk(Bq, Gq)
                    if rBG >= RC:
                        continue
                    prods = []
                    if terms & 1:
                        d1, d2 = D(A, Bq), D(Fq, Gq)
                        if d1 is not None and d2 is not None:
                            prods.append(("ab,fg", d1, d2))
                    if terms & 2:
                        d1, d2 = D(A, Gq), D(Fq, Bq)
                        if d1 is not None and d2 is not None:
                            prods.append(("ag,fb", d1, d2))
                    for sub, d1, d2 in prods:
                        spec = "xaf,xy,ybg," + sub
                        T = -np.einsum(spec + "->", CAF, VAB, CBG, d1, d2)
                        gAF = -np.einsum("cxaf,xy,ybg," + sub + "->c", dCAF, VAB, CBG, d1, d2)
                        gAB = -np.einsum("xaf,cxy,ybg," + sub + "->c", CAF, dVAB, CBG, d1, d2)
                        gBG = -np.einsum("xaf,xy,cybg," + sub + "->c", CAF, VAB, dCBG, d1, d2)
                        E += T
                        # Eq. Fexx1, one line per (block, atom) pair:
                        F[a] += gAF            # grad_M C_{MF}, M = A
                        F[Fq[0]] -= gAF        # grad_M C_{AM}, M = F
                        F[a] += gAB            # grad_M V_{MB}, M = A
                        F[Bq[0]] -= gAB        # grad_M V_{AM}, M = B
                        F[Bq[0]] += gBG        # grad_M C_{MG}, M = B
                        F[Gq[0]] -= gBG        # grad_M C_{BM}, M = G
                        # Eq. stress, three terms
                        Wv += np.outer(gAF, dAF) + np.outer(gAB, dAB) + np.outer(gBG, dBG)
    omega_cell = abs(float(np.linalg.det(L)))
    return E, F, -Wv / omega_cell
