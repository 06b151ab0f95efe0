"""Pins for the oracle MLP and probe features (CPU only)."""
import numpy as np

from oracle import features, mlp
from paper_2307_15572_gb300 import synth


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    d, h, B = 19, 16, 7
    theta = mlp.init(d, 1, h) + 0.05 * rng.standard_normal(mlp.n_params(d, h))
    X = rng.standard_normal((B, d))
    T = rng.standard_normal((B, 2))
    _, g = mlp.loss_and_grad(theta, X, T, h)
    eps = 1e-6
    num = np.empty_like(theta)
    for i in range(theta.size):
        tp = theta.copy(); tp[i] += eps
        tm = theta.copy(); tm[i] -= eps
        num[i] = (mlp.loss_and_grad(tp, X, T, h)[0] - mlp.loss_and_grad(tm, X, T, h)[0]) / (2 * eps)
    assert np.max(np.abs(num - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))


def test_gradient_full_width_sampled_coordinates():
    rng = np.random.default_rng(1)
    d, B = 19, 5
    theta = mlp.init(d, 2)
    X = rng.standard_normal((B, d))
    T = rng.standard_normal((B, 2))
    _, g = mlp.loss_and_grad(theta, X, T)
    eps = 1e-6
    for i in rng.choice(theta.size, 40, replace=False):
        tp = theta.copy(); tp[i] += eps
        tm = theta.copy(); tm[i] -= eps
        num = (mlp.loss_and_grad(tp, X, T)[0] - mlp.loss_and_grad(tm, X, T)[0]) / (2 * eps)
        assert abs(num - g[i]) <= 1e-7 * max(1.0, abs(g[i]))


def test_adam_overfits_small_batch():
    rng = np.random.default_rng(2)
    d = 19
    X = rng.standard_normal((32, d))
    T = rng.standard_normal((32, 2))
    theta = mlp.init(d, 3)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    for t in range(1, 1501):
        loss, g = mlp.loss_and_grad(theta, X, T)
        theta, m, v = mlp.adam_step(theta, g, m, v, t, lr=3e-3)
    assert loss < 1e-3


def test_probe_norm_estimate_unbiased():
    n = 300
    sig = synth.spectrum_pow(n, 1.0)
    A = synth.planted_haar(n, sig, 3)
    est = [features.probe_singular_values(A, seed=s)[1] / 16 for s in range(200)]
    est = np.array(est)
    fro2 = np.sum(sig ** 2)
    assert abs(est.mean() - fro2) < 4 * est.std() / np.sqrt(len(est))


def test_probe_sees_dominant_singular_value():
    # rank-1 A = s u u^T: Y16 = s u (u^T P) has one nonzero singular value
    n = 200
    rng = np.random.default_rng(4)
    u = rng.standard_normal(n); u /= np.linalg.norm(u)
    A = 5.0 * np.outer(u, u)
    t, fro2 = features.probe_singular_values(A, seed=1)
    assert t[1] <= 1e-12 * t[0]
    assert abs(t[0] - 5.0 * np.linalg.norm(u @ features.philox.gaussian_f64(np.arange(n), np.arange(16), 1, features.philox.TAG_PROBE))) < 1e-12 * t[0]
    f = features.features(t, fro2, n, 1e-4)
    assert f.shape == (features.D,)
    assert abs(f[17] - np.log(n)) < 1e-15 and abs(f[18] - np.log(1e-4)) < 1e-15
