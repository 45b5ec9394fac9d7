"""Plain FP64 CPU oracle for the LRI coefficient fit and its gradient.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module; only the tests may.  It shares no code with the CUDA
path.

What it computes (paper Sec. 3.1, Eq. C_VA and the gradient equation that
follows Eq. V_inverse)
--------------------------------------------------------------------------
For one atom pair (I, K), with n = n_abf(I) + n_abf(K) auxiliary functions
(first the ABFs of I, then those of K) and w = n_ao(I) n_ao(K) AO pairs:

    A   [n][n]     the two-centre Coulomb metric over the pair's ABFs,
                   blocks (V_II, V_IK; V_KI, V_KK), symmetric positive definite
    B   [n][w]     the three-centre integrals (P_beta | phi_i phi_k)
    dA  [3][n][n]  the gradient of A with respect to the position of K
    dB  [3][n][w]  the gradient of B with respect to the position of K

The coefficients are the solution of the fit equations, and their gradient
follows from differentiating A X = B (with d(A^-1) = -A^-1 dA A^-1):

    X      = A^-1 B                      (the C^I rows, then the C^K rows)
    dX[c]  = A^-1 ( dB[c] - dA[c] X )    for each Cartesian c

Both are computed here with the library solver numpy.linalg.solve, one pair
at a time, exactly as written: no factorisation is shared between the two
lines and nothing is reordered.
"""
from __future__ import annotations

import numpy as np


def fit(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X = A^-1 B for one pair (Eq. C_VA)."""
    return np.linalg.solve(np.asarray(A, np.float64), np.asarray(B, np.float64))


def fit_gradient(A: np.ndarray, B: np.ndarray, dA: np.ndarray, dB: np.ndarray) -> np.ndarray:
    """dX[c] = A^-1 (dB[c] - dA[c] A^-1 B) for one pair (the gradient
    equation after Eq. V_inverse)."""
    X = fit(A, B)
    return np.stack([np.linalg.solve(np.asarray(A, np.float64), np.asarray(dB[c], np.float64) - dA[c] @ X)
                     for c in range(3)])


def fit_batch(A, B, dA, dB):
    """The two functions above over a batch (leading axis = pair)."""
    X = np.stack([fit(A[p], B[p]) for p in range(A.shape[0])])
    dX = np.stack([fit_gradient(A[p], B[p], dA[p], dB[p]) for p in range(A.shape[0])])
    return X, dX
