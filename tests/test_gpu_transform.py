"""Factor post-processing against the oracle: the basis transformation on
the thin factors, the signs for symmetric (one-factor) storage, and the
compression ratio of the paper's definition."""
import numpy as np
import pytest

from oracle import rsvd as orsvd

pytestmark = pytest.mark.gpu


def _mixed_sign(n, r, seed):
    rng = np.random.default_rng(seed)
    Q, R = np.linalg.qr(rng.standard_normal((n, r)))
    Q = Q * np.sign(np.diag(R))
    lam = np.exp(-np.arange(r) / 8.0) * np.where(rng.random(r) < 0.5, -1.0, 1.0)
    return Q @ np.diag(lam) @ Q.T, lam


@pytest.mark.parametrize("prec", ["fp64", "bf16x"])
def test_transform_and_signs_match_oracle(lib, prec):
    import torch
    n, r, k, m = 1500, 60, 60, 333
    A, lam = _mixed_sign(n, r, 11)
    At = torch.as_tensor(A, device="cuda")
    plan = lib.Plan(n, k=k, p=10, q=1, seed=3, precision=prec)
    try:
        st, res = plan.decompose(At, k)
        assert st >= 0, lib.last_error()
        U, S, V = res["U"], res["S"], res["V"]
        Bn = np.random.default_rng(2).standard_normal((n, m))
        Bcm = torch.as_tensor(np.ascontiguousarray(Bn.T), device="cuda")      # column-major n x m, ld n
        B = Bcm.T
        Lt = torch.empty((k, m), dtype=torch.float64, device="cuda")         # column-major m x k
        Rt = torch.empty((k, m), dtype=torch.float64, device="cuda")
        for _ in range(2):                                                   # twice: no state kept
            lib.rsvd_transform_factors(plan.h, res["_fac"], n, Bcm.data_ptr(), n, m, Lt.data_ptr(), m,
                                       Rt.data_ptr(), m)
            Lo, Ro = orsvd.transform_factors(U.cpu().numpy(), V.cpu().numpy(), Bn)
            assert np.allclose(Lt.T.cpu().numpy(), Lo, rtol=0, atol=1e-12 * np.abs(Lo).max())
            assert np.allclose(Rt.T.cpu().numpy(), Ro, rtol=0, atol=1e-12 * np.abs(Ro).max())
        # B^T A B from the thin factors, within the decomposition's error
        ref = B.T @ At @ B
        got = (Lt.T * S) @ Rt
        err = plan.reconstruct_error(At, res)
        bound = 2.0 * err * torch.linalg.norm(At) * torch.linalg.norm(B, 2) ** 2
        assert torch.linalg.norm(got - ref) <= bound + 1e-12 * torch.linalg.norm(ref)
        signs = torch.empty(k, dtype=torch.float64, device="cuda")
        lib.rsvd_symmetric_signs(plan.h, res["_fac"], n, signs.data_ptr())
        torch.cuda.synchronize()
        so = orsvd.symmetric_signs(U.cpu().numpy(), V.cpu().numpy())
        assert np.array_equal(signs.cpu().numpy(), so)
        order = np.argsort(-np.abs(lam))
        assert np.array_equal(so, np.sign(lam[order][:k]))
        A1 = (U * (signs * S)) @ U.T                                         # one stored factor
        e1 = (torch.linalg.norm(A1 - At) / torch.linalg.norm(At)).item()
        # the one-factor form uses U twice, so it also carries the basis's own
        # rounding, which the two-sided form's projection V = A U S^-1 does
        # not: on the mixed path that is the sketch's word rounding (2^-17
        # relative per entry with two words), here allowed 8x
        slack = 1e-12 if prec == "fp64" else 8 * 2.0 ** -17
        assert e1 <= 2.0 * err + slack, (e1, err)
    finally:
        plan.close()


def test_compression_ratio_matches_definition(lib):
    for n, k in ((7650, 77), (40050, 40), (1000, 1)):
        for one in (False, True):
            ref = orsvd.compression_ratio(n, k, "single" if one else "eq2")
            assert lib.rsvd_compression_ratio(n, k, one) == pytest.approx(ref, rel=1e-15)
    assert lib.rsvd_compression_ratio(0, 5) == 0.0
