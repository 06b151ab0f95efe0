"""Oracle: the Gaussian-bump tile rule for matrices too large to store.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper's problem statement takes a dense symmetric V; when V is larger than
device memory the library accepts a *rule* for its entries instead.  The rule
(symmetric by construction) is

  x_i  = 8 i / (n - 1),                        i = 0 .. n-1
  g_m(x) = exp(-(x - c_m)^2 / (2 s_m^2)),      m = 1 .. M
  A_ij = sum_m w_m g_m(x_i) g_m(x_j) + eta_ij

with seeded centres c_m, widths s_m and weights w_m (input generator
``synth.rule_params``) and a symmetric hash noise

  eta_ij = eta_scale * sqrt(3) * (2 u - 1),
  u = ((h >> 8) + 1/2) 2^-24,
  h = mix(mix(min(i,j) * 0x9E3779B1 + key) ^ (max(i,j) * 0x85EBCA77)),
  key = mix(seed_lo ^ mix(seed_hi)),

where ``mix`` is the 32-bit "lowbias32" integer hash (x ^= x>>16;
x *= 0x7FEB352D; x ^= x>>15; x *= 0x846CA68B; x ^= x>>16; C. Wellons, "Hash
function prospector", 2018) and all arithmetic is modulo 2^32.  eta is uniform
with standard deviation eta_scale.

Parity: ``closed_form_eigs`` pins the rule: with eta = 0, A = G W G^T (G the
n x M matrix of g_m(x_i)), whose nonzero eigenvalues equal those of the M x M
matrix W^(1/2) G^T G W^(1/2); with eta, Weyl's inequality bounds the shift by
||eta||_2 <= ||eta||_F.  The hash itself is pinned by symmetry, range and
moment tests (tests/test_oracle_tilerule.py).
"""

import numpy as np

MASK = np.uint64(0xFFFFFFFF)


def mix32(x):
    x = np.asarray(x, dtype=np.uint64) & MASK
    x ^= x >> np.uint64(16)
    x = (x * np.uint64(0x7FEB352D)) & MASK
    x ^= x >> np.uint64(15)
    x = (x * np.uint64(0x846CA68B)) & MASK
    x ^= x >> np.uint64(16)
    return x


def noise_key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return int(mix32(np.uint64(seed & 0xFFFFFFFF) ^ mix32(np.uint64(seed >> 32))))


def eta(rows, cols, seed, scale):
    """Noise block eta[rows, cols] (FP64)."""
    i = np.asarray(rows, dtype=np.uint64)[:, None]
    j = np.asarray(cols, dtype=np.uint64)[None, :]
    lo = np.minimum(i, j)
    hi = np.maximum(i, j)
    key = np.uint64(noise_key(seed))
    h = mix32(((lo * np.uint64(0x9E3779B1)) & MASK) + key)
    h = mix32(h ^ ((hi * np.uint64(0x85EBCA77)) & MASK))
    u = ((h >> np.uint64(8)).astype(np.float64) + 0.5) * 2.0 ** -24
    return scale * np.sqrt(3.0) * (2.0 * u - 1.0)


def mesh(n):
    return 8.0 * np.arange(n, dtype=np.float64) / (n - 1)


def bumps(x, c, s):
    """G[i, m] = g_m(x_i)."""
    return np.exp(-((x[:, None] - c[None, :]) ** 2) / (2.0 * s[None, :] ** 2))


def block(rows, cols, n, c, s, w, seed, eta_scale):
    """Entries A[rows, cols] of the rule (FP64), evaluated entry by entry."""
    x = mesh(n)
    Gi = bumps(x[np.asarray(rows)], c, s)
    Gj = bumps(x[np.asarray(cols)], c, s)
    A = (Gi * w[None, :]) @ Gj.T
    if eta_scale != 0.0:
        A = A + eta(rows, cols, seed, eta_scale)
    return A


def dense(n, c, s, w, seed, eta_scale):
    idx = np.arange(n)
    return block(idx, idx, n, c, s, w, seed, eta_scale)


def closed_form_eigs(n, c, s, w):
    """Nonzero eigenvalues (descending) of G W G^T via the M x M form."""
    G = bumps(mesh(n), c, s)
    sw = np.sqrt(w)
    K = (G.T @ G) * sw[:, None] * sw[None, :]
    ev = np.linalg.eigvalsh(0.5 * (K + K.T))
    return np.sort(ev)[::-1]


def closed_form_fro2(n, c, s, w):
    """||G W G^T||_F^2 = tr((W G^T G)^2) without forming the n x n matrix."""
    G = bumps(mesh(n), c, s)
    K = (G.T @ G) * w[None, :]
    return float(np.sum(K * K.T))
