"""Oracle: the randomized SVD of the paper, step by step, in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Notation follows the paper's "Randomized matrix decompositions" paragraph and
Fig. 1: the input is V (N x N), the decomposition is V = L Sigma R^T (Eq. 1),
l = R_SVD + p columns are drawn, and

  step 1   Z = V P  with a random P (N x l);  QR:  Z = Q X
  (power)  q rounds of  Q <- qr(V^T Q),  Q <- qr(V Q)   [Halko et al., Alg. 4.4]
  step 1'  Y = Q^T V                                     (l x N)
  step 2   thin SVD  Y = L_Y Sigma R^T
  step 3   L = Q L_Y
  keep the R_SVD leading triplets.

The paper itself uses q = 0 and p = 5; q > 0 is the subspace iteration of
Halko, Martinsson & Tropp (2011), which the paper cites as the basis of its
method.  Re-orthogonalising after every product (rather than forming
(V V^T)^q V P) is their recommended form and keeps the sketch well conditioned.

Library primitives used as single steps: ``@`` (BLAS matmul),
``np.linalg.qr`` (LAPACK Householder QR), ``np.linalg.svd`` / ``eigh``
(LAPACK).  No blocking or reordering beyond the steps above.

Readings where the paper is silent:
  * both factors are returned; each pair (L_i, R_i) is sign-fixed so that the
    largest-magnitude entry of L_i is positive;
  * tolerance mode: R_SVD is the smallest k with
    ||V - L_k Sigma_k R_k^T||_F <= tol ||V||_F, computed exactly from the
    identity ||V - Q Q^T ... ||^2 = ||V||_F^2 - sum_{i<=k} s_i^2 (valid because
    L_k has orthonormal columns and R_k Sigma_k = V^T L_k);
  * Rayleigh-Ritz variant (symmetric V): T = Q^T V Q, eigendecomposition
    T = S Lambda S^T, L = Q S, s = |lambda|, R = L sign(lambda).

Parity: pinned in tests/test_oracle_rsvd.py by planted spectra (Haar U),
exact reconstruction of exactly-low-rank inputs, equality with a brute-force
Jacobi full SVD when l >= N, the Eckart-Young lower bound, the residual
identity, and the Halko-Martinsson-Tropp expected-error bound.
"""

from dataclasses import dataclass, field

import numpy as np

from . import philox


@dataclass
class Result:
    U: np.ndarray          # N x k, left factor L
    S: np.ndarray          # k, singular values, descending
    V: np.ndarray          # N x k, right factor R
    k: int
    l: int
    Q: np.ndarray = field(repr=False, default=None)     # N x l basis
    s_all: np.ndarray = field(repr=False, default=None)  # all l singular values
    err_est: float = float("nan")                        # from the identity above


def qr(z):
    """Thin Householder QR (LAPACK dgeqrf/dorgqr); returns Q only."""
    q, _ = np.linalg.qr(z, mode="reduced")
    return q


def sign_fix(L, R):
    """Flip each (L_i, R_i) so the largest-|.| entry of L_i is positive."""
    if L.shape[1] == 0:
        return L, R
    idx = np.argmax(np.abs(L), axis=0)
    sgn = np.sign(L[idx, np.arange(L.shape[1])])
    sgn[sgn == 0] = 1.0
    return L * sgn[None, :], R * sgn[None, :]


def range_finder(V, l, q, seed, P=None):
    """Fig. 1 step 1 plus q rounds of subspace iteration: orthonormal Q (N x l)."""
    N = V.shape[0]
    if P is None:
        P = philox.omega(N, l, seed)
    Z = V @ P                      # Z = V P
    Q = qr(Z)                      # Z = Q X
    for _ in range(q):
        Q = qr(V.T @ Q)
        Q = qr(V @ Q)
    return Q


def pick_rank(s, normV2, tol, kmax=None):
    """Smallest k with sqrt(||V||^2 - sum_{i<=k} s_i^2) <= tol ||V||; None if none."""
    kmax = len(s) if kmax is None else min(kmax, len(s))
    tail = normV2 - np.cumsum(s[:kmax] ** 2)
    ok = np.nonzero(np.sqrt(np.maximum(tail, 0.0)) <= tol * np.sqrt(normV2))[0]
    return int(ok[0]) + 1 if len(ok) else None


def rsvd(V, k=None, p=5, q=0, seed=0, tol=None, P=None, rayleigh_ritz=False,
         l=None):
    """Randomized SVD of V (N x N) following the paper's three steps.

    Fixed rank: give k (R_SVD) and p (l = k + p, capped at N).
    Tolerance mode: give tol and l (columns drawn); k is picked by ``pick_rank``.
    ``P`` overrides the Philox projection matrix (tests only).
    """
    V = np.asarray(V, dtype=np.float64)
    N = V.shape[0]
    if l is None:
        l = k + p
    l = min(l, N)
    Q = range_finder(V, l, q, seed, P)
    normV2 = float(np.sum(V * V))
    if rayleigh_ritz:
        T = Q.T @ (V @ Q)
        T = 0.5 * (T + T.T)
        lam, S = np.linalg.eigh(T)
        order = np.argsort(-np.abs(lam), kind="stable")
        lam, S = lam[order], S[:, order]
        L = Q @ S
        s = np.abs(lam)
        R = L * np.where(lam < 0, -1.0, 1.0)[None, :]
    else:
        Y = Q.T @ V                                     # Y = Q^T V
        LY, s, RT = np.linalg.svd(Y, full_matrices=False)  # step 2
        L = Q @ LY                                      # step 3
        R = RT.T
    if tol is not None:
        kk = pick_rank(s, normV2, tol, k)
        k = kk if kk is not None else len(s)
    k = min(k, len(s))
    Lk, Rk = sign_fix(L[:, :k], R[:, :k])
    est = float(np.sqrt(max(normV2 - np.sum(s[:k] ** 2), 0.0) / normV2)) if normV2 > 0 else 0.0
    return Result(U=Lk, S=s[:k].copy(), V=Rk, k=k, l=l, Q=Q, s_all=s, err_est=est)


def reconstruct_error(V, U, S, W):
    """Exact ||V - U diag(S) W^T||_F / ||V||_F in FP64.

    The relative error is undefined for V = 0; there the absolute residual
    ||U diag(S) W^T||_F is returned (0 for empty or zero factors)."""
    V = np.asarray(V, dtype=np.float64)
    D = V - (U * S[None, :]) @ W.T
    nv = np.linalg.norm(V)
    return float(np.linalg.norm(D) / nv) if nv > 0 else float(np.linalg.norm(D))


def eckart_young(sigma_sorted, k):
    """Optimal relative Frobenius error of a rank-k approximation."""
    s2 = np.asarray(sigma_sorted, dtype=np.float64) ** 2
    return float(np.sqrt(np.sum(s2[k:]) / np.sum(s2)))


def rsvd_adaptive(V, tol, b=16, q=0, seed=0, l_max=None):
    """Tolerance-driven blocked range finder (randQB_EI of Yu, Gu & Li 2018).

    Grows Q by blocks of b columns.  Each block: draw the next b Philox
    columns, form (V - Q B) P_i, orthonormalise, q deflated power rounds,
    re-orthogonalise against the earlier blocks, B_i = Q_i^T V, and update the
    error indicator E = ||V||^2 - ||B||^2; stop once E <= tol^2 ||V||^2.
    Then the thin SVD of B and rank selection as in ``rsvd``.
    Returns (Result, columns drawn).
    """
    V = np.asarray(V, dtype=np.float64)
    N = V.shape[0]
    l_max = N if l_max is None else min(l_max, N)
    normV2 = float(np.sum(V * V))
    thr = tol * tol * normV2
    Q = np.zeros((N, 0))
    B = np.zeros((0, N))
    E = normV2
    col = 0
    while Q.shape[1] < l_max:
        bb = min(b, l_max - Q.shape[1])
        P = philox.omega(N, bb, seed, col0=col)
        col += bb
        Qi = qr(V @ P - Q @ (B @ P))
        for _ in range(q):
            Qi = qr(V.T @ Qi - B.T @ (Q.T @ Qi))
            Qi = qr(V @ Qi - Q @ (B @ Qi))
        Qi = qr(Qi - Q @ (Q.T @ Qi))
        Bi = Qi.T @ V
        Q = np.hstack([Q, Qi])
        B = np.vstack([B, Bi])
        E -= float(np.sum(Bi * Bi))
        if E <= thr:
            break
    LY, s, RT = np.linalg.svd(B, full_matrices=False)
    L = Q @ LY
    R = RT.T
    k = pick_rank(s, normV2, tol)
    met = k is not None
    k = k if met else len(s)
    Lk, Rk = sign_fix(L[:, :k], R[:, :k])
    est = float(np.sqrt(max(normV2 - np.sum(s[:k] ** 2), 0.0) / normV2))
    res = Result(U=Lk, S=s[:k].copy(), V=Rk, k=k, l=Q.shape[1], Q=Q, s_all=s, err_est=est)
    return res, col, met


def compression_ratio(N, R, reading="eq2"):
    """Compression ratio of a rank-R form of an N x N matrix (Eq. 2).

    ``eq2``: N^2 / (2 N R + R) as printed (both factors stored).
    ``single``: N^2 / (N R + R), one factor stored (symmetric V, L = R up to
    signs), the reading under which R% = 1 gives C ~ 100 as the text states.
    """
    if reading == "eq2":
        return N * N / (2.0 * N * R + R)
    return N * N / (1.0 * N * R + R)


def transform_factors(U, V, B):
    """Basis transformation on the thin factors ("Low-rank interactions"
    paragraph after Eq. (3)): with V ~ U S V^T, B^T V B ~ (B^T U) S (B^T V)^T,
    so only the thin factors are multiplied by B."""
    return B.T @ U, B.T @ V


def symmetric_signs(U, V):
    """sign(u_i . v_i): for symmetric input v_i = sign(lambda_i) u_i, so the
    eigenvalue signs, and V ~ U diag(sign * S) U^T (one factor stored)."""
    return np.where(np.einsum("ij,ij->j", U, V) >= 0.0, 1.0, -1.0)


def relative_rank(N, R):
    """R% = 100 R / N (text after Eq. 2)."""
    return 100.0 * R / N
