"""Pins for the oracle randomized SVD (CPU only).

Each pin is fixed by mathematics independent of the oracle's own code:
planted spectra with Haar singular vectors, exactly-low-rank inputs, a
brute-force Jacobi SVD, the Eckart-Young bound, the residual identity and the
Halko-Martinsson-Tropp expected-error bounds.  Non-symmetric inputs are used
where a transposed operand would otherwise go unnoticed.
"""
import os

import numpy as np
import pytest

from oracle import jacobi, rsvd
from paper_2307_15572_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.txt")


def _facts():
    out = {}
    for line in open(GOLD):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            out[k] = float(v)
    return out


@pytest.fixture(scope="module")
def dense():
    return synth.dense_case()


def _planted_pin(res, sig, l, q):
    """sigma_hat_i within max(2e-14, 10x the power-scheme gap) of sigma_i.

    For subspace iteration with q rounds the captured direction i has
    tan(theta_i) ~ (sigma_{l+1}/sigma_i)^(2q+1) and so a relative deficit
    ~ (sigma_{l+1}/sigma_i)^(2(2q+1)); sigma_hat_i <= sigma_i always
    (interlacing of a projection)."""
    k = len(res.S)
    pred = (sig[l] / sig[:k]) ** (2 * (2 * q + 1))
    rel = np.abs(res.S - sig[:k]) / sig[:k]
    assert np.all(res.S <= sig[:k] * (1 + 1e-13))
    assert np.all(rel <= np.maximum(2e-14, 10 * pred)), np.max(rel / np.maximum(2e-14, 10 * pred))


def test_planted_spectrum_dense2048(dense):
    sig = synth.spectrum_exp(2048)
    res = rsvd.rsvd(dense, k=64, p=10, q=2, seed=synth.SEED_DENSE)
    _planted_pin(res, sig, 74, 2)
    # exact-arithmetic identity for the estimate vs the true residual
    err = rsvd.reconstruct_error(dense, res.U, res.S, res.V)
    assert abs(err - res.err_est) < 1e-10
    ey = rsvd.eckart_young(sig, 64)
    assert ey <= err <= ey * 1.001


def test_planted_paper_mode_q0_p5(dense):
    # the paper's own setting: q = 0, p = 5
    sig = synth.spectrum_exp(2048)
    res = rsvd.rsvd(dense, k=40, p=5, q=0, seed=3)
    _planted_pin(res, sig, 45, 0)


def test_mutation_dropped_power_iteration_is_caught(dense, monkeypatch):
    sig = synth.spectrum_exp(2048)
    real = rsvd.range_finder
    monkeypatch.setattr(rsvd, "range_finder", lambda V, l, q, seed, P=None: real(V, l, 0, seed, P))
    res = rsvd.rsvd(dense, k=64, p=10, q=2, seed=synth.SEED_DENSE)
    with pytest.raises(AssertionError):
        _planted_pin(res, sig, 74, 2)


def test_exact_rank_reconstruction_nonsymmetric():
    rng = np.random.default_rng(5)
    n, r = 512, 50
    U = synth.haar_orthogonal(n, rng)[:, :r]
    W = synth.haar_orthogonal(n, rng)[:, :r]
    sig = np.linspace(3.0, 0.5, r)
    A = (U * sig) @ W.T
    res = rsvd.rsvd(A, k=r, p=10, q=0, seed=11)
    assert rsvd.reconstruct_error(A, res.U, res.S, res.V) <= 1e-13
    assert np.max(np.abs(res.S - sig) / sig) <= 1e-12
    # factors: U^T U = I, and U diag(S) V^T reproduces A column space
    assert np.linalg.norm(res.U.T @ res.U - np.eye(r)) < 1e-13


def test_full_basis_equals_bruteforce_jacobi_nonsymmetric():
    rng = np.random.default_rng(6)
    n = 96
    A = rng.standard_normal((n, n)) * np.logspace(0, -3, n)[None, :]
    res = rsvd.rsvd(A, k=n, p=0, q=0, seed=1)       # l = n: Q spans R^n
    _U, sj, _W, _ = jacobi.jacobi_svd(A)
    assert np.max(np.abs(res.S - sj)) <= 1e-12 * sj[0]
    assert rsvd.reconstruct_error(A, res.U, res.S, res.V) < 1e-13


def test_eckart_young_lower_bound_and_residual_identity():
    rng = np.random.default_rng(7)
    n = 400
    sig = synth.spectrum_pow(n, 1.0)
    A = synth.planted_haar(n, sig, 8)
    for k, p, q in [(10, 5, 0), (30, 10, 1), (60, 4, 2)]:
        res = rsvd.rsvd(A, k=k, p=p, q=q, seed=rng.integers(1 << 30))
        err = rsvd.reconstruct_error(A, res.U, res.S, res.V)
        assert err >= rsvd.eckart_young(sig, k) * (1 - 1e-12)
        Q = res.Q
        B = Q.T @ A
        lhs = np.linalg.norm(A - Q @ B) ** 2
        rhs = np.sum(A * A) - np.sum(B * B)
        assert abs(lhs - rhs) <= 1e-12 * np.sum(A * A)


def test_hmt_expected_frobenius_bound_q0():
    """Halko-Martinsson-Tropp (2011) Thm 10.5: for Gaussian P with l = k + p,
    E ||(I - P_Y) A||_F <= (1 + k/(p-1))^(1/2) (sum_{j>k} sigma_j^2)^(1/2)."""
    n, k = 512, 20
    sig = synth.spectrum_pow(n, 1.0)
    A = synth.planted_haar(n, sig, 21)
    tail = np.sqrt(np.sum(sig[k:] ** 2))
    for p in (2, 5, 10):
        errs = []
        for s in range(200):
            Q = rsvd.range_finder(A, k + p, 0, seed=1000 + s)
            errs.append(np.linalg.norm(A - Q @ (Q.T @ A)))
        errs = np.array(errs)
        bound = np.sqrt(1 + k / (p - 1)) * tail
        assert errs.mean() - 3 * errs.std() / np.sqrt(len(errs)) <= bound
        assert errs.min() >= tail * (1 - 1e-12)          # never beats Eckart-Young


def test_hmt_power_scheme_spectral_bound_q1():
    """HMT (2011) Cor. 10.10 for q power rounds (spectral norm):
    E||(I-P_Y)A|| <= [(1+sqrt(k/(p-1))) s_{k+1}^(2q+1)
                      + e sqrt(k+p)/p (sum_{j>k} s_j^(2(2q+1)))^(1/2)]^(1/(2q+1))."""
    n, k, p, q = 256, 15, 5, 1
    sig = synth.spectrum_pow(n, 0.5)
    A = synth.planted_haar(n, sig, 22)
    e = np.e
    t = 2 * q + 1
    bound = ((1 + np.sqrt(k / (p - 1))) * sig[k] ** t
             + e * np.sqrt(k + p) / p * np.sqrt(np.sum(sig[k:] ** (2 * t)))) ** (1.0 / t)
    errs = []
    for s in range(60):
        Q = rsvd.range_finder(A, k + p, q, seed=2000 + s)
        errs.append(np.linalg.norm(A - Q @ (Q.T @ A), 2))
    errs = np.array(errs)
    assert errs.mean() - 3 * errs.std() / np.sqrt(len(errs)) <= bound
    assert errs.min() >= sig[k] * (1 - 1e-12)


def test_tolerance_mode_meets_tol_and_is_minimal():
    n = 1200
    sig = synth.spectrum_pow(n, 2.5)
    A = synth.planted_mixed(n, sig, 31, noise_std=synth.batch_noise_std(n))
    for tol in (1e-3, 1e-4, 1e-5):
        res = rsvd.rsvd(A, tol=tol, l=400, q=1, seed=5)
        err = rsvd.reconstruct_error(A, res.U, res.S, res.V)
        assert err <= tol * (1 + 1e-9)
        # one fewer triplet misses the tolerance
        err_less = rsvd.reconstruct_error(A, res.U[:, :-1], res.S[:-1], res.V[:, :-1])
        assert err_less > tol


def test_mutation_wrong_sign_in_rank_rule_is_caught(monkeypatch):
    n = 600
    sig = synth.spectrum_pow(n, 2.5)
    A = synth.planted_mixed(n, sig, 32)

    def bad(s, normV2, tol, kmax=None):
        kmax = len(s) if kmax is None else min(kmax, len(s))
        tail = normV2 + np.cumsum(s[:kmax] ** 2)           # planted: + instead of -
        ok = np.nonzero(np.sqrt(np.maximum(tail, 0.0)) <= tol * np.sqrt(normV2) * 2)[0]
        return int(ok[0]) + 1 if len(ok) else 1

    monkeypatch.setattr(rsvd, "pick_rank", bad)
    res = rsvd.rsvd(A, tol=1e-4, l=200, q=1, seed=5)
    assert rsvd.reconstruct_error(A, res.U, res.S, res.V) > 1e-4


def test_adaptive_loop_meets_tol():
    n = 1500
    sig = synth.spectrum_pow(n, 2.5)
    A = synth.planted_mixed(n, sig, 33, noise_std=synth.batch_noise_std(n))
    for tol in (1e-3, 1e-5):
        res, drawn, met = rsvd.rsvd_adaptive(A, tol=tol, b=16, q=1, seed=9)
        assert met
        err = rsvd.reconstruct_error(A, res.U, res.S, res.V)
        assert err <= tol * (1 + 1e-9)
        # rank within a few of the optimal (Eckart-Young) rank
        k_opt = next(k for k in range(1, n) if rsvd.eckart_young(sig, k) <= tol)
        assert k_opt - 2 <= res.k <= k_opt + 4
        assert drawn == res.l and drawn % 16 == 0


def test_rayleigh_ritz_variant():
    n = 800
    sig = synth.spectrum_exp(n, 15.0)
    A = synth.planted_haar(n, sig, 34)
    qb = rsvd.rsvd(A, k=40, p=10, q=1, seed=3)
    rr = rsvd.rsvd(A, k=40, p=10, q=1, seed=3, rayleigh_ritz=True)
    e_qb = rsvd.reconstruct_error(A, qb.U, qb.S, qb.V)
    e_rr = rsvd.reconstruct_error(A, rr.U, rr.S, rr.V)
    # two-sided projection: ||A - PAP||^2 <= 2 ||A - PA||^2 for symmetric A
    assert e_qb <= e_rr * (1 + 1e-9)
    assert e_rr <= np.sqrt(2) * e_qb * (1 + 1e-9)
    # Ritz values obey the same interlacing and power-scheme gap as the QB
    # singular values, and never exceed them for PSD A (Q^T A^2 Q >= (Q^T A Q)^2)
    _planted_pin(rr, sig, 50, 1)
    assert np.all(rr.S <= qb.S * (1 + 1e-12))


def test_compression_ratio_readings():
    f = _facts()
    N = 10000
    for rpct, key in ((1.0, "rpct_1_compression"), (0.1, "rpct_0.1_compression")):
        R = int(rpct * N / 100)
        assert abs(rsvd.relative_rank(N, R) - rpct) < 1e-12
        single = rsvd.compression_ratio(N, R, "single")
        eq2 = rsvd.compression_ratio(N, R, "eq2")
        # the text's "C ~ 100 / 1000" matches the one-factor reading; Eq. (2)
        # as printed gives half of it
        assert abs(single / f[key] - 1) < 0.01
        assert abs(eq2 / (f[key] / 2) - 1) < 0.01
    assert f["channel_n_min"] % (f["mesh_np"] * f["mesh_nq"]) == 0
    assert f["channel_n_max"] % (f["mesh_np"] * f["mesh_nq"]) == 0


def _mixed_sign_symmetric(n, lam, seed):
    rng = np.random.default_rng(seed)
    Q, R = np.linalg.qr(rng.standard_normal((n, len(lam))))
    Q = Q * np.sign(np.diag(R))
    return Q @ np.diag(lam) @ Q.T, Q


def test_transform_factors_exact_low_rank():
    """Closed form: for exactly rank-r input and l >= r the factors are exact,
    and B^T A B equals (B^T U) S (B^T V)^T for any B (not only unitary)."""
    n, r, m = 200, 12, 37
    lam = np.array([5.0, -4.0, 3.0, -2.5, 2.0, 1.5, -1.2, 1.0, 0.8, -0.6, 0.5, 0.3])
    A, _ = _mixed_sign_symmetric(n, lam, 3)
    res = rsvd.rsvd(A, k=r, p=8, q=0, seed=4)
    B = np.random.default_rng(5).standard_normal((n, m))
    Lt, Rt = rsvd.transform_factors(res.U, res.V, B)
    ref = B.T @ A @ B
    got = (Lt * res.S) @ Rt.T
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))
    # a plausible slip -- the left factor used on both sides, which drops the
    # signs of the negative eigenvalues -- is far off
    assert np.max(np.abs((Lt * res.S) @ Lt.T - ref)) > 1e-2 * np.max(np.abs(ref))


def test_symmetric_signs_recover_eigenvalue_signs():
    """Closed form: the signs are those of the eigenvalues, in the order of
    |lambda|, and U diag(sign S) U^T reproduces A (one stored factor)."""
    n = 150
    lam = np.array([-6.0, 5.0, -3.0, 2.0, -1.0, 0.5])
    A, _ = _mixed_sign_symmetric(n, lam, 7)
    res = rsvd.rsvd(A, k=6, p=6, q=0, seed=1)
    sg = rsvd.symmetric_signs(res.U, res.V)
    order = np.argsort(-np.abs(lam))
    assert np.array_equal(sg, np.sign(lam[order]))
    assert np.allclose(res.S, np.abs(lam[order]), rtol=1e-12)
    A1 = (res.U * (sg * res.S)) @ res.U.T
    assert np.max(np.abs(A1 - A)) <= 1e-12 * np.max(np.abs(A))


def test_reconstruct_error_of_zero_matrix_is_absolute():
    # relative error is undefined for V = 0: the absolute residual is reported
    n, k = 30, 3
    rng = np.random.default_rng(21)
    U = rng.standard_normal((n, k))
    W = rng.standard_normal((n, k))
    S = np.array([3.0, 2.0, 0.5])
    Z = np.zeros((n, n))
    direct = np.sqrt(np.sum(((U * S) @ W.T) ** 2))
    assert abs(rsvd.reconstruct_error(Z, U, S, W) - direct) <= 1e-14 * direct
    assert rsvd.reconstruct_error(Z, U[:, :0], S[:0], W[:, :0]) == 0.0
