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


def test_adam_first_step_closed_form():
    # From m = v = 0 the bias-corrected moments of step 1 are m_hat = g and
    # v_hat = g^2 exactly (Kingma & Ba, Alg. 1), so every parameter moves by
    # -lr g / (|g| + eps).  Without the correction the move would be
    # -lr 0.1 g / (sqrt(0.001) |g| + eps), about 3.16x larger.
    rng = np.random.default_rng(5)
    g = rng.standard_normal(257) * np.logspace(-3, 3, 257)
    theta = rng.standard_normal(257)
    lr, eps = 2e-3, 1e-8
    t1, m1, v1 = mlp.adam_step(theta, g, np.zeros_like(g), np.zeros_like(g), 1, lr=lr, eps=eps)
    # (compared on theta itself: the subtraction t1 - theta would cancel)
    assert np.allclose(t1, theta - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g, rtol=4e-15, atol=0)      # 1 - 0.9 and 1 - 0.999 round
    assert np.allclose(v1, 0.001 * g * g, rtol=4e-15, atol=0)


def test_adam_two_steps_hand_computed():
    # Scalar gradients g1 = 1, g2 = -2 with the default betas, worked by hand:
    #   m1 = 0.1,  v1 = 0.001
    #   m2 = 0.9 * 0.1 + 0.1 * (-2) = -0.11,   v2 = 0.999 * 0.001 + 0.001 * 4 = 0.004999
    #   m_hat2 = -0.11 / (1 - 0.9^2) = -0.11 / 0.19
    #   v_hat2 = 0.004999 / (1 - 0.999^2) = 0.004999 / 0.001999
    lr, eps = 1e-3, 1e-8
    th = np.array([0.25])
    m = np.zeros(1)
    v = np.zeros(1)
    th1, m, v = mlp.adam_step(th, np.array([1.0]), m, v, 1, lr=lr, eps=eps)
    th2, m, v = mlp.adam_step(th1, np.array([-2.0]), m, v, 2, lr=lr, eps=eps)
    step1 = -lr * 1.0 / (1.0 + eps)
    step2 = -lr * (-0.11 / 0.19) / (np.sqrt(0.004999 / 0.001999) + eps)
    assert abs(m[0] - (-0.11)) < 1e-15 and abs(v[0] - 0.004999) < 1e-17
    assert abs(th1[0] - (0.25 + step1)) < 1e-15
    assert abs(th2[0] - (0.25 + step1 + step2)) < 1e-15
    # the second step moves against the first (a sign error in m would not)
    assert step2 > 0


def test_feature_order_on_known_singular_values():
    # t_j = 2^{1-j}: the 15 log-ratios are log(t_j / t_1) = -(j-1) log 2 for
    # j = 2..16 in that order, then log t_1, the norm estimate, log n, log tol.
    t = 3.0 * 2.0 ** -np.arange(16)
    fro2 = 16.0 * 49.0
    f = features.features(t, fro2, 5000, 1e-5)
    assert np.allclose(f[:15], -np.arange(1, 16) * np.log(2.0), rtol=0, atol=1e-14)
    assert abs(f[15] - np.log(3.0)) < 1e-15
    assert abs(f[16] - np.log(7.0)) < 1e-15          # 0.5 log(16 * 49 / 16)
    assert abs(f[17] - np.log(5000.0)) < 1e-14
    assert abs(f[18] - np.log(1e-5)) < 1e-14


def test_probe_of_rank_one_diagonal_input():
    # V = a e_1 e_1^T: Y16 = a e_1 P[0, :], one nonzero singular value
    # |a| ||P[0, :]|| and ||Y16||_F^2 = a^2 ||P[0, :]||^2; the norm feature is
    # then 0.5 log(a^2 ||P[0, :]||^2 / 16).
    n, a = 64, -4.0
    V = np.zeros((n, n))
    V[0, 0] = a
    t, fro2 = features.probe_singular_values(V, seed=9)
    p0 = features.philox.gaussian_f64(np.array([0]), np.arange(16), 9, features.philox.TAG_PROBE)[0]
    assert abs(t[0] - abs(a) * np.linalg.norm(p0)) < 1e-13 * t[0]
    assert np.all(t[1:] <= 1e-14 * t[0])
    assert abs(fro2 - a * a * np.sum(p0 * p0)) < 1e-12 * fro2
