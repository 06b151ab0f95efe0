"""Variants of the method's use: the paper's own scheme (q = 0, p = 5) on
the GPU paths against the oracle at the same seed, and a repeated-seed
study of the projection error against the Halko-Martinsson-Tropp expected
bound (their Thm. 10.5) -- the spread of the rSVD over the random sketch."""
import numpy as np
import pytest

from oracle import rsvd as orsvd
from paper_2307_15572_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "bf16x"])
def test_paper_mode_q0_p5_matches_oracle(lib, prec):
    import torch
    n, k = 2048, 64
    A = synth.planted_haar(n, np.exp(-np.arange(1, n + 1) / 20.0), synth.SEED_DENSE)
    o = orsvd.rsvd(A, k=k, p=5, q=0, seed=9)
    e_o = orsvd.reconstruct_error(A, o.U, o.S, o.V)
    At = torch.as_tensor(A, device="cuda")
    plan = lib.Plan(n, k=k, p=5, q=0, seed=9, precision=prec)
    try:
        st, r = plan.decompose(At, k)
        assert st >= 0, lib.last_error()
        e = plan.reconstruct_error(At, r)
        assert e <= 1.05 * e_o, (e, e_o)
    finally:
        plan.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x"])
def test_seed_spread_within_hmt_bound(lib, prec):
    """40 seeds, n = 512, sigma_j = 1/j, k = 20: the untruncated projection
    error ||A - Q Q^T A||_F (rank l = k + p factors) has mean within
    (1 + k/(p-1))^(1/2) (sum_{j>k} sigma_j^2)^(1/2) (3 standard errors) and
    never beats the Eckart-Young tail."""
    import torch
    n, k, p = 512, 20, 5
    sig = synth.spectrum_pow(n, 1.0)
    A = synth.planted_haar(n, sig, 21)
    At = torch.as_tensor(A, device="cuda")
    tail = np.sqrt(np.sum(sig[k:] ** 2))
    nA = np.linalg.norm(A)
    errs = []
    for s in range(40):
        plan = lib.Plan(n, k=k + p, p=0, q=0, seed=1000 + s, precision=prec)
        try:
            st, r = plan.decompose(At, k + p)
            assert st >= 0, lib.last_error()
            errs.append(plan.reconstruct_error(At, r) * nA)
        finally:
            plan.close()
    errs = np.array(errs)
    bound = np.sqrt(1 + k / (p - 1)) * tail
    print(f"{prec}: mean {errs.mean():.4f} sd {errs.std():.4f} bound {bound:.4f} tail {tail:.4f}")
    assert errs.mean() - 3 * errs.std() / np.sqrt(len(errs)) <= bound
    assert errs.min() >= np.sqrt(np.sum(sig[k + p:] ** 2)) * (1 - 1e-6)


def test_mixed_power_of_two_scale_invariance(lib):
    """V and 2^(+-36) V on the mixed path: the steps of the method commute
    with an exact power of two up to FP32 rounding (the word splitting, the
    sliced Grams and products take per-row/column exponents, the
    double-float Cholesky and the FP32 Jacobi rescale their input), so the
    rank and the scaled singular values agree, and the relative errors to
    1e-4 of their value (measured: 2.6e-5 at 2^36).  Without
    the Jacobi's rescaling, the products of squared column norms of 2^36 V
    (about 2^144) overflow FP32 and those of 2^-36 V underflow."""
    import torch
    mats = [synth.batch_channel(c, n) for c, n in enumerate([3000, 2200])]
    out = {}
    for e in (0, 36, -36):
        plan = lib.Plan(3000, k=118, p=10, q=0, seed=4, tol=1e-4, policy="tol", precision="bf16x", slices=2)
        try:
            ts = [torch.as_tensor(np.ldexp(A, e), device="cuda") for A in mats]
            st, res = plan.decompose_batched(ts, 128)
            assert st >= 0, lib.last_error()
            out[e] = [(r["k"], np.ldexp(r["S"].cpu().numpy(), -e), plan.reconstruct_error(t, r))
                      for t, r in zip(ts, res)]
        finally:
            plan.close()
    for e in (36, -36):
        for (k0, s0, e0), (k1, s1, e1) in zip(out[0], out[e]):
            assert k1 == k0, (e, k0, k1)
            assert np.max(np.abs(s1[:k0] - s0[:k0])) <= 1e-6 * s0[0], e
            assert e1 <= 1e-4 and abs(e1 - e0) <= 1e-4 * e0, (e, e0, e1)
