"""Oracle: the rank-prediction MLP, forward, backward and Adam, in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper picks the rank by hand (R_SVD, oversampling p = 5); the library adds
a small learned model that predicts, per channel and tolerance, the rank k and
oversampling p from a cheap probe sketch.  Network (d -> 128 -> 128 -> 2):

  h1 = tanh(x W1 + b1),  h2 = tanh(h1 W2 + b2),  y = h2 W3 + b3,
  loss = mean over the batch and the 2 outputs of (y - t)^2.

Backward pass by the chain rule (d tanh(z)/dz = 1 - tanh(z)^2); Adam as in
Kingma & Ba, ICLR 2015 (Alg. 1): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
theta <- theta - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Parameter blob layout (shared *format*, not code, with the CUDA kernels):
W1 (d x H), b1 (H), W2 (H x H), b2 (H), W3 (H x 2), b3 (2), row-major,
concatenated in that order.

Parity: the analytic gradient is pinned against central finite differences
(h = 1e-6) and training is pinned by an overfit test
(tests/test_oracle_mlp.py).
"""

import numpy as np

H = 128
OUT = 2


def param_shapes(d, h=H):
    return [(d, h), (h,), (h, h), (h,), (h, OUT), (OUT,)]


def n_params(d, h=H):
    return sum(int(np.prod(s)) for s in param_shapes(d, h))


def unpack(theta, d, h=H):
    out, o = [], 0
    for s in param_shapes(d, h):
        m = int(np.prod(s))
        out.append(theta[o:o + m].reshape(s))
        o += m
    return out


def init(d, seed, h=H):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in param_shapes(d, h):
        if len(s) == 2:
            b = 1.0 / np.sqrt(s[0])
            parts.append(rng.uniform(-b, b, size=s).ravel())
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts)


def forward(theta, X, h=H):
    W1, b1, W2, b2, W3, b3 = unpack(theta, X.shape[1], h)
    h1 = np.tanh(X @ W1 + b1)
    h2 = np.tanh(h1 @ W2 + b2)
    y = h2 @ W3 + b3
    return y, (h1, h2)


def loss_and_grad(theta, X, T, h=H):
    d = X.shape[1]
    W1, b1, W2, b2, W3, b3 = unpack(theta, d, h)
    y, (h1, h2) = forward(theta, X, h)
    B = X.shape[0]
    r = y - T
    loss = float(np.mean(r * r))
    gy = 2.0 * r / (B * OUT)
    gW3 = h2.T @ gy
    gb3 = gy.sum(0)
    gz2 = (gy @ W3.T) * (1.0 - h2 * h2)
    gW2 = h1.T @ gz2
    gb2 = gz2.sum(0)
    gz1 = (gz2 @ W2.T) * (1.0 - h1 * h1)
    gW1 = X.T @ gz1
    gb1 = gz1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam_step(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
