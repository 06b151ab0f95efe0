"""Pins for the oracle's brute-force one-sided Jacobi SVD (CPU only)."""
import numpy as np

from oracle import jacobi


def _check(A, tol_rel=1e-13):
    U, s, W, sweeps = jacobi.jacobi_svd(A)
    ref = np.linalg.svd(A, compute_uv=False)           # LAPACK: library special case
    k = min(A.shape)
    assert np.allclose(s[:k], ref[:k], rtol=0, atol=tol_rel * ref[0] * 10)
    big = ref[:k] > 1e-8 * ref[0]
    assert np.max(np.abs(s[:k][big] - ref[:k][big]) / ref[:k][big]) < 1e-12
    assert np.linalg.norm(W.T @ W - np.eye(W.shape[1])) < 1e-13 * W.shape[1]
    R = (U * s[None, :]) @ W.T
    assert np.linalg.norm(A - R) <= 1e-14 * np.linalg.norm(A) * A.shape[1]
    assert sweeps < 30
    return s


def test_random_rectangular():
    rng = np.random.default_rng(0)
    _check(rng.standard_normal((60, 40)))


def test_random_square():
    rng = np.random.default_rng(1)
    _check(rng.standard_normal((64, 64)))


def test_graded_spectrum_relative_accuracy():
    # one-sided Jacobi resolves small singular values of graded matrices to
    # high relative accuracy (Demmel & Veselic 1992)
    rng = np.random.default_rng(2)
    n = 48
    q1, _ = np.linalg.qr(rng.standard_normal((n, n)))
    q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sig = np.logspace(0, -9, n)
    A = (q1 * sig[None, :]) @ q2.T
    _U, s, _W, _ = jacobi.jacobi_svd(A)
    assert np.max(np.abs(s - sig) / sig) < 1e-6


def test_exact_zero_and_duplicate():
    A = np.diag([3.0, 3.0, 0.0, 1.0])
    _U, s, _W, _ = jacobi.jacobi_svd(A)
    assert np.allclose(s, [3.0, 3.0, 1.0, 0.0])
