"""The tensor-core tall x small product (rsvd_panel_product) against the definition.

C = A B with A an n x K FP32 panel and B a K x N matrix (FP32 or FP64), the
product behind CholeskyQR's Q = Y R^{-1} and the lifts of the mixed path.
The reference is the FP64 product of the same data.

Bound: A and B are represented to 2^-25 of 2^e (e the exponent of the row
(column) maximum, so within 2^-24 of the maximum), their slice products are
summed exactly, the four level sums are added in FP32 and the result is
rounded once, so
    |C - A B| <= 2^-24 (maxrow_r ||b_j||_1 + maxcol_j ||a_r||_1
                        + 4 sum_k |a_rk| |b_kj| + |C|),
which the test checks with a factor 2 to spare.  An error in the slice
layout, the exponents or the level sums is O(1) or at least 2^-8 of the
scale and fails it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(lib, plan, A, B, c64, lda=None, ldc=None):
    import torch
    n, K = A.shape
    K2, N = B.shape
    lda = lda or n
    ldc = ldc or n
    At = torch.zeros((K, lda), dtype=torch.float32, device="cuda")
    At[:, :n] = torch.as_tensor(np.ascontiguousarray(A.T), device="cuda")
    Bt = torch.as_tensor(np.ascontiguousarray(B.T), device="cuda")      # column-major K x N
    Ct = torch.full((N, ldc), float("nan"), dtype=torch.float64 if c64 else torch.float32, device="cuda")
    lib.rsvd_panel_product(plan.h, At.data_ptr(), lda, n, K, Bt.data_ptr(), K, B.dtype == np.float64, N,
                           Ct.data_ptr(), ldc, c64)
    return Ct.cpu().numpy().T[:n].astype(np.float64)


def _bound(A, B, C):
    Ad, Bd = A.astype(np.float64), B.astype(np.float64)
    rmax = np.max(np.abs(Ad), axis=1)[:, None]
    cmax = np.max(np.abs(Bd), axis=0)[None, :]
    absAB = np.abs(Ad) @ np.abs(Bd)
    return 2.0 ** -24 * (rmax * np.sum(np.abs(Bd), axis=0)[None, :] + cmax * np.sum(np.abs(Ad), axis=1)[:, None]
                         + 4 * absAB + np.abs(C))


@pytest.mark.parametrize("n,K,N,b64,c64", [(1, 1, 1, False, False), (77, 16, 5, True, False),
                                           (128, 128, 128, False, False), (129, 77, 100, True, True),
                                           (4097, 128, 128, True, False), (12000, 128, 118, False, True)])
def test_panel_product_matches_definition(lib, n, K, N, b64, c64):
    rng = np.random.default_rng(n + 7 * K + N)
    A = rng.standard_normal((n, K)) * 10.0 ** rng.uniform(-4, 4, size=(n, 1))     # rows over eight decades
    A[:, K // 2:] *= 1e-3                                                          # two scales inside a row
    if n > 5:
        A[3] = 0.0                                                                 # a zero row
    A = A.astype(np.float32)
    B = rng.standard_normal((K, N)) * 10.0 ** rng.uniform(-3, 3, size=(1, N))
    B = B if b64 else B.astype(np.float32)
    plan = lib.Plan(max(n, 2), k=1, p=0, precision="bf16x")
    try:
        C = _run(lib, plan, A, B, c64)
        ref = A.astype(np.float64) @ B.astype(np.float64)
        err = np.abs(C - ref)
        assert np.all(err <= 2 * _bound(A, B, C)), float(np.max(err / (_bound(A, B, C) + 1e-300)))
        if n > 5:
            assert np.all(C[3] == 0.0)
        # padded leading dimensions
        C2 = _run(lib, plan, A, B, c64, lda=n + 5, ldc=n + 3)
        assert np.array_equal(C, C2)
    finally:
        plan.close()


def test_panel_product_inverse_factor(lib):
    """CholeskyQR's use: Y (condition ~1e4) times the inverse of its Cholesky
    factor.  The result is orthonormal to the accuracy an FP32 product of
    these operands allows (kappa u_32), like the CUDA-core product."""
    import torch
    rng = np.random.default_rng(5)
    n, l = 6000, 128
    Q0, _ = np.linalg.qr(rng.standard_normal((n, l)))
    Y = (Q0 * np.logspace(0, -4, l)).astype(np.float32)
    Yd = Y.astype(np.float64)
    R = np.linalg.cholesky(Yd.T @ Yd).T
    Ri = np.linalg.inv(R)
    plan = lib.Plan(n, k=1, p=0, precision="bf16x")
    try:
        Q = _run(lib, plan, Y, Ri, False)
    finally:
        plan.close()
    ortho = np.max(np.abs(Q.T @ Q - np.eye(l)))
    Yt = torch.as_tensor(Y, device="cuda")
    Q32 = (Yt @ torch.as_tensor(Ri.astype(np.float32), device="cuda")).double().cpu().numpy()
    ortho32 = np.max(np.abs(Q32.T @ Q32 - np.eye(l)))
    assert ortho <= max(4 * ortho32, 1e-4), (ortho, ortho32)


def test_panel_product_nonfinite_and_errors(lib):
    import torch
    rng = np.random.default_rng(9)
    A = rng.standard_normal((300, 20)).astype(np.float32)
    A[17, 4] = np.nan
    B = rng.standard_normal((20, 10)).astype(np.float32)
    plan = lib.Plan(300, k=1, p=0, precision="bf16x")
    try:
        C = _run(lib, plan, A, B, False)
        assert np.all(np.isnan(C[17]))
        assert np.all(np.isfinite(np.delete(C, 17, 0)))
        buf = torch.zeros((200, 200), dtype=torch.float32, device="cuda")
        for args, status in (((200, 100, 129, 10), lib.RSVD_ERR_UNSUPPORTED),     # K > 128
                             ((200, 100, 10, 129), lib.RSVD_ERR_UNSUPPORTED),     # N > 128
                             ((50, 100, 10, 10), lib.RSVD_ERR_INVALID_ARG),       # lda < n
                             ((200, 0, 10, 10), lib.RSVD_ERR_INVALID_ARG)):       # n < 1
            lda, n, K, N = args
            with pytest.raises(lib.RsvdError) as e:
                lib.rsvd_panel_product(plan.h, buf.data_ptr(), lda, n, K, buf.data_ptr(), 200, False, N,
                                       buf.data_ptr(), 200, False)
            assert e.value.status == status
    finally:
        plan.close()


def test_decomposition_same_with_either_product(lib, monkeypatch):
    """The mixed path with the tensor-core products against the same path with
    the CUDA-core FP32 products: both FP32-grade, so singular values agree to
    ~1e-6 of sigma_1, ranks to one, residuals to 1 %; U stays orthonormal."""
    import torch
    from paper_2307_15572_gb300 import synth
    A = synth.batch_channel(8, 7000)
    At = torch.as_tensor(A, device="cuda")
    out = {}
    for mode in ("tc", "simt"):
        if mode == "simt":
            monkeypatch.setenv("RSVD_NN", "simt")
        else:
            monkeypatch.delenv("RSVD_NN", raising=False)
        plan = lib.Plan(7000, k=80, p=48, q=0, seed=4, precision="bf16x", policy="tol", tol=1e-4)
        try:
            st, r = plan.decompose(At, 128)
            assert st >= 0, lib.last_error()
            U = r["U"].cpu().numpy()
            out[mode] = (r["S"].cpu().numpy(), r["k"], plan.reconstruct_error(At, r),
                         np.max(np.abs(U.T @ U - np.eye(U.shape[1]))))
        finally:
            plan.close()
    (s1, k1, e1, o1), (s2, k2, e2, o2) = out["tc"], out["simt"]
    assert abs(k1 - k2) <= 1
    k = min(k1, k2)
    assert np.max(np.abs(s1[:k] - s2[:k])) <= 1e-6 * s1[0]
    assert abs(e1 - e2) <= 0.01 * e2
    assert o1 <= max(4 * o2, 1e-6), (o1, o2)
