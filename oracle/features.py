"""Oracle: probe-sketch features for the learned rank model.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

A cheap 16-column probe Y16 = V P16 (P16 from the Philox stream with tag
TAG_PROBE) sees the leading part of the spectrum.  Its singular values
t_1 >= ... >= t_16 (LAPACK SVD of Y16; going through the Gram would square
the spread and lose the small ones) and the channel's size and tolerance
form the feature vector (d = 19):

  f = [ log(t_j / t_1) for j = 2..16,        (15 values; t_j floored at 1e-300)
        log t_1,
        log ||V||_F estimate = 0.5 log(||Y16||_F^2 / 16),
        log n,
        log tol ]

E||V P||_F^2 = 16 ||V||_F^2 for Gaussian P, which is where the norm estimate
comes from.  The targets are (log k*, log p*) with k* the smallest rank that
meets the tolerance and p* = l - k* the columns the adaptive loop drew beyond
it (at least 1).

Parity: pinned in tests/test_oracle_mlp.py by the norm-estimate expectation
and exact singular values on a diagonal input.
"""

import numpy as np

from . import philox

NPROBE = 16
D = 19


def probe_singular_values(V, seed):
    n = V.shape[0]
    P = philox.gaussian_f64(np.arange(n), np.arange(NPROBE), seed, philox.TAG_PROBE)
    Y = V @ P
    t = np.linalg.svd(Y, compute_uv=False)
    return t, float(np.sum(Y * Y))


def features(t, fro2_probe, n, tol):
    t = np.maximum(np.asarray(t, dtype=np.float64), 1e-300)
    f = np.empty(D)
    f[:15] = np.log(t[1:16] / t[0])
    f[15] = np.log(t[0])
    f[16] = 0.5 * np.log(max(fro2_probe, 1e-300) / NPROBE)
    f[17] = np.log(n)
    f[18] = np.log(tol)
    return f


def targets(k_star, p_star):
    return np.array([np.log(max(k_star, 1)), np.log(max(p_star, 1))])
