"""The FP64-grade Grams of CholeskyQR (rsvd_gram_f32) against the definition.

G = Y^T Y of an FP32 panel.  Both methods -- the tensor-core split into exact
BF16 slices and the CUDA-core compensated (Dot2) Gram -- are compared with
the plain definition: on sampled entries with math.fsum over the exact FP64
products of the FP32 data (a correctly rounded reference), and on every
entry with the FP64 matrix product.

Bounds (of ||y_i|| ||y_j||): each entry is represented to 2^-49 of its
tile-column maximum, the dropped slice products are below 2^-47 of a row's
product and the one rounded accumulator (slice levels 5-7) holds terms below
2^-23 of the total, so the tensor-core Gram is good to ~1e-13 typically and
the test allows 2e-12 (the FP32-grade three-slice form: 1e-6); the FP64
matrix product itself carries about
n 2^-53 of sum |y_i||y_j|.  An FP32-grade Gram (error ~1e-7) or a slice
layout error fails both checks by orders of magnitude.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TC, DOT2, TC_F32 = 0, 1, 2


def _panel(rng, n, l, kind):
    Y = rng.standard_normal((n, l))
    Y *= 10.0 ** rng.uniform(-3.0, 3.0, size=l)           # columns over six decades
    if kind == "spiky" and n > 3:
        Y[rng.integers(0, n), :] *= 1e4                   # one row dominates every column maximum
        Y[:, 0] = 0.0                                     # a zero column
        Y[: n // 2, -1] *= 1e-6                           # a column with two scales
    if kind == "positive":
        Y = np.abs(Y)
    return Y.astype(np.float32)


def _gram(lib, plan, Y, method, ldy=None):
    import torch
    n, l = Y.shape
    ldy = ldy or (n + 3) // 4 * 4
    buf = torch.zeros((l, ldy), dtype=torch.float32, device="cuda")   # column-major n x l, leading dim ldy
    buf[:, :n] = torch.as_tensor(np.ascontiguousarray(Y.T), device="cuda")
    G = torch.full((l, l), float("nan"), dtype=torch.float64, device="cuda")
    lib.rsvd_gram_f32(plan.h, buf.data_ptr(), ldy, n, l, G.data_ptr(), method)
    return G.cpu().numpy().T                               # column-major l x l


def _check(Y, G, tol):
    Yd = Y.astype(np.float64)
    n, l = Y.shape
    norms = np.linalg.norm(Yd, axis=0)
    scale = np.outer(norms, norms)
    assert np.array_equal(G, G.T)
    ref = Yd.T @ Yd
    absg = np.abs(Yd).T @ np.abs(Yd)
    assert np.all(np.abs(G - ref) <= tol * scale + 4 * n * 2.0 ** -53 * absg), np.max(np.abs(G - ref) / (scale + 1e-300))
    rng = np.random.default_rng(n * 131 + l)
    pairs = [(0, 0), (l - 1, l - 1), (0, l - 1)] + [tuple(rng.integers(0, l, size=2)) for _ in range(24)]
    for i, j in pairs:
        exact = math.fsum((Yd[:, i] * Yd[:, j]).tolist())   # FP32 x FP32 products are exact in FP64
        assert abs(G[i, j] - exact) <= tol * scale[i, j], (i, j, G[i, j], exact, scale[i, j])


@pytest.mark.parametrize("n,l,kind", [(1, 1, "normal"), (77, 16, "normal"), (128, 128, "spiky"),
                                      (129, 77, "normal"), (1000, 128, "positive"), (4097, 100, "spiky"),
                                      (12000, 128, "normal")])
def test_gram_matches_definition(lib, n, l, kind):
    rng = np.random.default_rng(7 + n + l)
    Y = _panel(rng, n, l, kind)
    plan = lib.Plan(max(n, 2), k=1, p=0, precision="bf16x")
    try:
        for method in (TC, DOT2):
            _check(Y, _gram(lib, plan, Y, method), 2e-12)
        # the FP32-grade form: operands rounded to 24 fractional bits of the
        # tile-column maxima, products exact
        _check(Y, _gram(lib, plan, Y, TC_F32), 1e-6)
        # a leading dimension with padding rows after n
        _check(Y, _gram(lib, plan, Y, TC, ldy=(n + 3) // 4 * 4 + 8), 2e-12)
    finally:
        plan.close()


def test_gram_methods_agree_and_beat_fp32(lib):
    """On a sketch-like panel of condition ~1e5 the two FP64-grade Grams agree
    far below FP32 rounding, and each is closer to the exact Gram than an
    FP32 matrix product is."""
    import torch
    rng = np.random.default_rng(11)
    n, l = 9000, 128
    Q, _ = np.linalg.qr(rng.standard_normal((n, l)))
    Y = (Q * np.logspace(0, -5, l)).astype(np.float32)
    plan = lib.Plan(n, k=1, p=0, precision="bf16x")
    try:
        Gt = _gram(lib, plan, Y, TC)
        Gd = _gram(lib, plan, Y, DOT2)
    finally:
        plan.close()
    Yd = Y.astype(np.float64)
    norms = np.linalg.norm(Yd, axis=0)
    scale = np.outer(norms, norms)
    assert np.max(np.abs(Gt - Gd) / scale) <= 2e-12
    Yt = torch.as_tensor(Y, device="cuda")
    G32 = (Yt.T @ Yt).double().cpu().numpy()
    ref = Yd.T @ Yd
    assert np.max(np.abs(Gt - ref) / scale) * 1e3 < np.max(np.abs(G32 - ref) / scale)
    # the Cholesky factor of the tensor-core Gram reproduces the FP64 one
    Rt = np.linalg.cholesky(Gt)
    Rr = np.linalg.cholesky(ref)
    assert np.max(np.abs(Rt - Rr)) <= 1e-5 * np.max(np.abs(Rr))


def test_gram_nonfinite_propagates(lib):
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((300, 40)).astype(np.float32)
    Y[17, 5] = np.nan
    plan = lib.Plan(300, k=1, p=0, precision="bf16x")
    try:
        G = _gram(lib, plan, Y, TC)
    finally:
        plan.close()
    assert np.isnan(G[5, 5]) and np.isnan(G[5, 0]) and np.isnan(G[39, 5])
    assert np.all(np.isfinite(np.delete(np.delete(G, 5, 0), 5, 1)))


def test_gram_argument_errors(lib):
    import torch
    plan = lib.Plan(256, k=1, p=0, precision="bf16x")
    buf = torch.zeros((200, 256), dtype=torch.float32, device="cuda")
    G = torch.zeros((200, 200), dtype=torch.float64, device="cuda")
    try:
        for args, status in (((256, 256, 129, TC), lib.RSVD_ERR_UNSUPPORTED),        # l > 128 on the tensor cores
                             ((256, 256, 8, 5), lib.RSVD_ERR_INVALID_ARG),           # unknown method
                             ((100, 256, 8, TC), lib.RSVD_ERR_INVALID_ARG),          # ldy < n
                             ((256, 0, 8, TC), lib.RSVD_ERR_INVALID_ARG)):           # n < 1
            ldy, n, l, method = args
            with pytest.raises(lib.RsvdError) as e:
                lib.rsvd_gram_f32(plan.h, buf.data_ptr(), ldy, n, l, G.data_ptr(), method)
            assert e.value.status == status
        with pytest.raises(lib.RsvdError) as e:                                # Y not 16-byte aligned
            lib.rsvd_gram_f32(plan.h, buf.data_ptr() + 4, 256, 250, 8, G.data_ptr(), TC)
        assert e.value.status == lib.RSVD_ERR_UNSUPPORTED
        # the CUDA-core method takes l > 128 and a misaligned panel
        lib.rsvd_gram_f32(plan.h, buf.data_ptr() + 4, 256, 250, 150, G.data_ptr(), DOT2)
    finally:
        plan.close()


def test_decomposition_same_with_either_gram(lib, monkeypatch):
    """The mixed path with the tensor-core Grams against the same path with
    the compensated CUDA-core Grams: the Grams differ by ~1e-13, which the
    FP32 small SVD of the mixed path sees at most as FP32 rounding of its
    input, so singular values agree to ~1e-6 of sigma_1, the ranks chosen for
    the tolerance to one, and the residuals to 1 %."""
    import torch
    from paper_2307_15572_gb300 import synth
    A = synth.batch_channel(5, 6000)
    At = torch.as_tensor(A, device="cuda")
    out = {}
    for mode in ("tc", "dot2"):
        if mode == "dot2":
            monkeypatch.setenv("RSVD_GRAM", "dot2")
        else:
            monkeypatch.delenv("RSVD_GRAM", raising=False)
        plan = lib.Plan(6000, k=80, p=48, q=0, seed=9, precision="bf16x", policy="tol", tol=1e-4)
        try:
            st, r = plan.decompose(At, 128)
            assert st >= 0, lib.last_error()
            out[mode] = (r["S"].cpu().numpy(), r["k"], plan.reconstruct_error(At, r))
        finally:
            plan.close()
    (s1, k1, e1), (s2, k2, e2) = out["tc"], out["dot2"]
    assert abs(k1 - k2) <= 1
    k = min(k1, k2)
    assert np.max(np.abs(s1[:k] - s2[:k])) <= 1e-6 * s1[0]
    assert abs(e1 - e2) <= 0.01 * e2
