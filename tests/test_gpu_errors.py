"""Error and warning paths of the decomposition, made to happen on purpose.

* RSVD_ERR_TIMEOUT: the cooperative Jacobi (l past one CTA's shared memory)
  separates its rounds by a grid barrier whose spin is bounded.  A test hook
  makes CTA 0 leave before its first arrival -- a participant that never
  arrives -- and a short wait budget makes the other CTAs' waits expire
  quickly.  The call must return RSVD_ERR_TIMEOUT, and the same plan must
  then decompose correctly: the context stays usable.
* RSVD_ERR_NOT_CONVERGED: the Jacobi sweep cap forced to one sweep.
* RSVD_WARN_SHIFTED_CQR: an exactly rank-deficient input, whose sketch Gram
  is singular, so the Cholesky breaks down and takes its shifted form; the
  factors are still valid.
No test here faults or hangs the GPU: every wait is bounded, and nothing is
read or written out of bounds.
"""
import numpy as np
import pytest

from oracle import rsvd as orsvd
from paper_2307_15572_gb300 import synth

pytestmark = pytest.mark.gpu


def _fp64_l130_case():
    n, k, p = 600, 120, 10              # l = 130: the FP64 Jacobi runs on the cooperative grid
    A = synth.planted_haar(n, synth.spectrum_exp(n, 30.0), 77)
    return A, n, k, p


def test_barrier_wait_expiry_returns_timeout(lib, monkeypatch):
    import torch
    A, n, k, p = _fp64_l130_case()
    At = torch.as_tensor(A, device="cuda")
    plan = lib.Plan(n, k=k, p=p, q=0, seed=3, precision="fp64")
    try:
        monkeypatch.setenv("RSVD_WAIT_CLOCKS", str(1 << 21))     # ~1 ms per wait
        monkeypatch.setenv("RSVD_TEST_STALL_BARRIER", "1")
        st, _ = plan.decompose(At, k)
        assert st == lib.RSVD_ERR_TIMEOUT, (st, lib.last_error())
        assert "wait" in lib.last_error()
        monkeypatch.delenv("RSVD_TEST_STALL_BARRIER")
        monkeypatch.delenv("RSVD_WAIT_CLOCKS")
        st, r = plan.decompose(At, k)
        assert st == 0, lib.last_error()
    finally:
        plan.close()
    o = orsvd.rsvd(A, k=k, p=p, q=0, seed=3)
    sg = r["S"].cpu().numpy()
    big = o.S > 1e-12 * o.S[0]
    assert np.all(np.abs(sg[big] - o.S[big]) <= 1e-10 * o.S[big])


@pytest.mark.parametrize("prec,k", [("fp64", 40), ("bf16x", 40), ("fp64", 120)])
def test_jacobi_sweep_cap_gives_not_converged(lib, monkeypatch, prec, k):
    import torch
    n, p = 600, 10
    A = synth.planted_haar(n, synth.spectrum_exp(n, 30.0), 78)
    At = torch.as_tensor(A, device="cuda")
    plan = lib.Plan(n, k=k, p=p, q=0, seed=3, precision=prec)
    try:
        monkeypatch.setenv("RSVD_JACOBI_MAX_SWEEPS", "1")
        st, _ = plan.decompose(At, k)
        assert st == lib.RSVD_ERR_NOT_CONVERGED, (st, lib.last_error())
        monkeypatch.delenv("RSVD_JACOBI_MAX_SWEEPS")
        st, r = plan.decompose(At, k)
        assert st == 0, lib.last_error()
        err = plan.reconstruct_error(At, r)
    finally:
        plan.close()
    o = orsvd.rsvd(A, k=k, p=p, q=0, seed=3)
    assert err <= 1.05 * orsvd.reconstruct_error(A, o.U, o.S, o.V)


@pytest.mark.parametrize("prec", ["fp64", "bf16x"])
def test_rank_deficient_input_warns_shifted_cqr(lib, prec):
    import torch
    n, r, k, p = 400, 10, 10, 30
    sig = np.zeros(n)
    sig[:r] = np.exp(-np.arange(r) / 3.0)
    A = synth.planted_haar(n, sig, 79)                 # rank 10 (up to FP64 rounding)
    At = torch.as_tensor(A, device="cuda")
    plan = lib.Plan(n, k=k, p=p, q=0, seed=5, precision=prec)
    try:
        st, res = plan.decompose(At, k)
        err = plan.reconstruct_error(At, res)
    finally:
        plan.close()
    if prec == "fp64":
        # the 40-column FP64 sketch spans only 10 directions: its Gram is
        # singular to rounding, the Cholesky breaks down and takes its shifted
        # form, and the conditional third round restores the basis
        assert st == lib.RSVD_WARN_SHIFTED_CQR, (st, lib.last_error())
        assert res["status"] == lib.RSVD_WARN_SHIFTED_CQR
        assert err <= 1e-12, err
        s = res["S"].cpu().numpy()
        assert np.max(np.abs(s - sig[:k])) <= 1e-12 * sig[0]
    else:
        # the BF16 words' rounding fills the other 30 directions at ~1e-7,
        # so the mixed path's Gram is merely ill-conditioned
        assert st in (0, lib.RSVD_WARN_SHIFTED_CQR), (st, lib.last_error())
        assert err <= 1e-5, err
