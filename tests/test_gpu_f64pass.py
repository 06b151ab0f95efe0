"""The FP64-input tensor-core passes (mixed path, q = 0; taken on request,
RSVD_F64PASS=1) against the oracle and against the word passes (the default).

With q = 0 the sketch and the projection read the stored FP64 V directly and
split it into the same two BF16 words on chip (the word passes first store
the words, then read them twice).  The words are bit-identical, so the two
forms differ only in FP32 summation order: ranks within one of each other,
singular values within FP32 rounding of the small SVD, residuals within 1 %;
both meet the tolerance and stay within the oracle's rank margin.  The batch
has at least one 128-row tile per SM (the passes' condition), even leading
dimensions (the TMA's), and the profile shows which passes ran.
"""
import numpy as np
import pytest

from oracle import rsvd as orsvd
from paper_2307_15572_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [5120, 4994, 5300, 4608]          # 158 row tiles of 128


def _run(lib, mats, monkeypatch, f64pass, **kw):
    import torch
    if f64pass:
        monkeypatch.setenv("RSVD_F64PASS", "1")
    else:
        monkeypatch.delenv("RSVD_F64PASS", raising=False)
    plan = lib.Plan(max(A.shape[0] for A in mats), precision="bf16x", slices=2, **kw)
    try:
        lib.rsvd_plan_set_profiling(plan.h, True)
        ts = [torch.as_tensor(A, device="cuda") for A in mats]
        st, res = plan.decompose_batched(ts, 128)
        prof = lib.rsvd_plan_profile(plan.h, True)
        errs = [plan.reconstruct_error(t, r) if r["k"] > 0 else 1.0 for t, r in zip(ts, res)]
    finally:
        plan.close()
    return st, res, errs, prof


def test_f64pass_tolerance_batch(lib, monkeypatch):
    mats = [synth.batch_channel(c, n) for c, n in enumerate(SIZES)]
    kw = dict(k=118, p=10, q=0, seed=3, tol=1e-4, policy="tol")
    st1, r1, e1, p1 = _run(lib, mats, monkeypatch, True, **kw)
    st0, r0, e0, p0 = _run(lib, mats, monkeypatch, False, **kw)
    assert st1 == 0 and st0 == 0, lib.last_error()
    assert p1["f64in_launches"] == 2 and p1["cvt_launches"] == 1
    assert p0["f64in_launches"] == 0 and p0["cvt_launches"] == 1
    for A, a, b, ea, eb in zip(mats, r1, r0, e1, e0):
        assert ea <= 1e-4 and eb <= 1e-4
        assert abs(a["k"] - b["k"]) <= 1
        k = min(a["k"], b["k"])
        sa, sb = a["S"].cpu().numpy()[:k], b["S"].cpu().numpy()[:k]
        assert np.max(np.abs(sa - sb)) <= 1e-6 * sa[0]
        assert abs(ea - eb) <= 0.01 * eb
        o = orsvd.rsvd(A, tol=1e-4, l=128, q=0, seed=3)
        assert o.k <= a["k"] <= o.k + 12, (A.shape[0], a["k"], o.k)


def test_f64pass_fixed_rank_error_ratio(lib, monkeypatch):
    mats = [synth.batch_channel(10 + c, n) for c, n in enumerate(SIZES)]
    st, res, errs, prof = _run(lib, mats, monkeypatch, True, k=64, p=10, q=0, seed=7)
    assert st == 0, lib.last_error()
    assert prof["f64in_launches"] == 2
    for A, r, e in zip(mats, res, errs):
        o = orsvd.rsvd(A, k=64, p=10, q=0, seed=7)
        e_o = orsvd.reconstruct_error(A, o.U, o.S, o.V)
        assert r["k"] == 64
        assert e <= 1.05 * e_o, (A.shape[0], e, e_o)


def test_f64pass_nonfinite_reported(lib, monkeypatch):
    mats = [synth.batch_channel(c, n) for c, n in enumerate(SIZES)]
    mats[2] = mats[2].copy()
    mats[2][4000, 17] = np.inf
    st, res, errs, prof = _run(lib, mats, monkeypatch, True, k=30, p=10, q=0, seed=1)
    assert prof["f64in_launches"] >= 1
    assert res[2]["status"] == lib.RSVD_ERR_NONFINITE
    assert all(res[c]["status"] >= 0 for c in (0, 1, 3))


def test_f64pass_mixed_odd_even_batch(lib, monkeypatch):
    """Odd leading dimensions cannot be read by the TMA: those channels keep
    the conversion to words and the word passes, in the same call, while the
    even ones read FP64; both kinds meet the tolerance and the oracle's rank
    margin."""
    sizes = [6400, 5001, 6000, 5300, 3999, 4608]
    mats = [synth.batch_channel(20 + c, n) for c, n in enumerate(sizes)]
    st, res, errs, prof = _run(lib, mats, monkeypatch, True, k=118, p=10, q=0, seed=5, tol=1e-4, policy="tol")
    assert st == 0, lib.last_error()
    assert prof["f64in_launches"] == 2 and prof["cvt_launches"] == 1 and prof["tc_launches"] == 2
    for A, r, e in zip(mats, res, errs):
        assert e <= 1e-4, (A.shape[0], e)
        o = orsvd.rsvd(A, tol=1e-4, l=128, q=0, seed=5)
        assert o.k <= r["k"] <= o.k + 12, (A.shape[0], r["k"], o.k)
