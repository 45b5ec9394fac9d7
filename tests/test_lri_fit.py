"""LRI coefficient fit (Eq. C_VA) and its gradient: the oracle against
closed forms and finite differences on the CPU, and hfx_lri_fit (the GPU
block preparation) against the oracle."""
import numpy as np
import pytest

from oracle import lri_fit as oracle
from paper_2412_11081_gb300 import inputs


def test_oracle_gradient_matches_finite_differences():
    """d/dd of A(d)^-1 B(d) by a 4-point stencil against the gradient
    equation with the model's exact dA, dB: pins the sign of the metric
    term and that dA multiplies X (not B)."""
    d, A, B, dA, dB, tpl = inputs.lri_pairs(2, 7, 5, 3, 2, seed=9)
    h = 1e-4
    for p in range(2):
        G = oracle.fit_gradient(A[p], B[p], dA[p], dB[p])
        for c in range(3):
            e = np.zeros(3)
            e[c] = h
            f = [oracle.fit(*inputs.lri_blocks(tpl, d[p] + k * e)[:2]) for k in (-2, -1, 1, 2)]
            fd = (f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * h)
            assert np.max(np.abs(fd - G[c])) <= 1e-8 * max(1.0, np.max(np.abs(G[c])))


def test_oracle_special_cases():
    rng = np.random.default_rng(3)
    # identity metric: X = B, and with dA = 0 the gradient is dB
    B = rng.standard_normal((4, 6))
    dB = rng.standard_normal((3, 4, 6))
    assert np.array_equal(oracle.fit(np.eye(4), B), B)
    assert np.allclose(oracle.fit_gradient(np.eye(4), B, np.zeros((3, 4, 4)), dB), dB, rtol=0, atol=1e-15)
    # 2 x 2 metric by Cramer's rule, and its derivative for dA = [[0, 1], [1, 0]] (the I-K coupling)
    a, b, c = 2.0, 0.3, 1.5
    A = np.array([[a, b], [b, c]])
    rhs = np.array([[1.0], [2.0]])
    det = a * c - b * b
    x = np.array([[(c * 1.0 - b * 2.0) / det], [(a * 2.0 - b * 1.0) / det]])
    assert np.allclose(oracle.fit(A, rhs), x, rtol=1e-15, atol=0)
    dA = np.zeros((3, 2, 2))
    dA[0] = [[0.0, 1.0], [1.0, 0.0]]
    # d/db of Cramer's solution
    ddet = -2 * b
    dx0 = ((-2.0) * det - (c - 2 * b) * ddet) / det ** 2
    dx1 = ((-1.0) * det - (2 * a - b) * ddet) / det ** 2
    g = oracle.fit_gradient(A, rhs, dA, np.zeros((3, 2, 1)))
    assert np.allclose(g[0, :, 0], [dx0, dx1], rtol=1e-14, atol=0)


def test_lri_inputs_are_spd_and_seeded():
    d1, A1, *_ = inputs.lri_pairs(3, 50, 50, 13, 13, seed=4)
    d2, A2, *_ = inputs.lri_pairs(3, 50, 50, 13, 13, seed=4)
    assert np.array_equal(A1, A2) and np.array_equal(d1, d2)
    for p in range(3):
        assert np.allclose(A1[p], A1[p].T)
        assert np.linalg.eigvalsh(A1[p]).min() > 0.1


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b))))


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(50, 50, 13, 13, 24), (9, 14, 5, 9, 7), (3, 2, 1, 2, 320)])
def test_gpu_fit_matches_oracle(shape):
    """Si-like pairs (n 100, w 169), an uneven species pair (n 23, w 45) and
    a batch larger than the kernel's grid (320 pairs, n 5, w 2)."""
    from paper_2412_11081_gb300 import hfx
    mi, mk, ni, nk, batch = shape
    d, A, B, dA, dB, _ = inputs.lri_pairs(batch, mi, mk, ni, nk, seed=11)
    X, dX = hfx.lri_fit(A, B, dA, dB)
    Xr, dXr = oracle.fit_batch(A, B, dA, dB)
    assert rel(X, Xr) <= 1e-10 and rel(dX, dXr) <= 1e-10
    X_only = hfx.lri_fit(A, B)
    assert rel(X_only, Xr) <= 1e-10


@pytest.mark.gpu
def test_gpu_fit_errors():
    from paper_2412_11081_gb300 import hfx
    d, A, B, dA, dB, _ = inputs.lri_pairs(2, 4, 3, 2, 2, seed=2)
    A_bad = A.copy()
    A_bad[1] = -np.eye(A.shape[1])     # not positive definite
    with pytest.raises(hfx.HfxError) as ei:
        hfx.lri_fit(A_bad, B, dA, dB)
    assert ei.value.status == 1
    big = np.tile(np.eye(200), (1, 1, 1))
    with pytest.raises(hfx.HfxError) as ei:
        hfx.lri_fit(big, np.ones((1, 200, 1)))
    assert ei.value.status == 6
    X = hfx.lri_fit(A, B)              # the library is still usable
    assert rel(X, oracle.fit_batch(A, B, dA, dB)[0]) <= 1e-10
