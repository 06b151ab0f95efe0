"""Oracle: brute-force one-sided (Hestenes) Jacobi SVD in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

An independent full SVD used to pin the randomized SVD: when l >= N the
random basis spans the whole space and the rSVD must return the exact
singular values (the paper validates its rSVD "against an exact SVD for
small matrices", "Randomized matrix decompositions" paragraph).

Method (Hestenes 1958; Golub & Van Loan, Matrix Computations, 4th ed.,
Sec. 8.6.3 for the symmetric 2 x 2 Schur rotation): repeatedly sweep over all
column pairs (i, j) of the working matrix M in cyclic-by-row order; for each
pair form alpha = ||m_i||^2, beta = ||m_j||^2, gamma = m_i^T m_j and apply the
plane rotation that makes the two columns orthogonal,
    zeta = (beta - alpha) / (2 gamma),  t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
    c = 1 / sqrt(1 + t^2),  s = c t,
    m_i <- c m_i - s m_j,   m_j <- s m_i + c m_j,
accumulating the same rotation into W (starting from I).  Stop when every
pair satisfies |gamma| <= eps sqrt(alpha beta).  Then sigma_i = ||m_i||,
U_i = m_i / sigma_i and V = W; sort descending.

Pure Python loop over pairs: meant for N <= 256.

Parity: pinned against LAPACK's SVD (a library special case) and by
orthogonality and reconstruction in tests/test_oracle_jacobi.py.
"""

import numpy as np


def jacobi_svd(A, eps=None, max_sweeps=60):
    M = np.array(A, dtype=np.float64, copy=True)
    m, n = M.shape
    if eps is None:
        eps = m * np.finfo(np.float64).eps
    W = np.eye(n)
    for sweep in range(max_sweeps):
        rotated = False
        for i in range(n - 1):
            for j in range(i + 1, n):
                mi, mj = M[:, i], M[:, j]
                alpha = float(mi @ mi)
                beta = float(mj @ mj)
                gamma = float(mi @ mj)
                if gamma == 0.0 or abs(gamma) <= eps * np.sqrt(alpha * beta):
                    continue
                rotated = True
                zeta = (beta - alpha) / (2.0 * gamma)
                t = (1.0 if zeta >= 0 else -1.0) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = c * t
                new_i = c * mi - s * mj
                new_j = s * mi + c * mj
                M[:, i], M[:, j] = new_i, new_j
                wi, wj = W[:, i].copy(), W[:, j].copy()
                W[:, i] = c * wi - s * wj
                W[:, j] = s * wi + c * wj
        if not rotated:
            break
    sig = np.linalg.norm(M, axis=0)
    order = np.argsort(-sig, kind="stable")
    sig = sig[order]
    M = M[:, order]
    W = W[:, order]
    U = np.zeros_like(M)
    nz = sig > 0
    U[:, nz] = M[:, nz] / sig[nz][None, :]
    return U, sig, W, sweep + 1
