"""GPU parity of the C-ABI library against the FP64 oracle (same seeded inputs).

Bars (from the method's statement of the problem and the accuracy targets):
  * all-FP64 path: singular values within 1e-10 relative of the oracle's for
    sigma_i > 1e-12 sigma_1 (smaller ones within 1e-13 sigma_1 absolute), same
    rank, and relative Frobenius error within 1.05x the oracle's;
  * mixed path: relative Frobenius error within 1.05x the oracle's at the same
    (k, p, q, seed); in tolerance mode error <= tol.
"""
import numpy as np
import pytest

from oracle import rsvd as orsvd
from paper_2307_15572_gb300 import synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def run(lib, A, **kw):
    torch = _torch()
    At = torch.as_tensor(A, device="cuda")
    k_cap = kw.pop("k_cap", None)
    n = A.shape[0]
    plan = lib.Plan(n, **kw)
    try:
        st, res = plan.decompose(At, k_cap or max(1, kw.get("k", 0) or n))
        err = plan.reconstruct_error(At, res) if res["k"] > 0 else 1.0
    finally:
        plan.close()
    return st, res, err


def sigma_parity(s_gpu, s_ora, rel=1e-10):
    s1 = s_ora[0]
    big = s_ora > 1e-12 * s1
    d = np.abs(s_gpu - s_ora)
    assert np.all(d[big] <= rel * s_ora[big]), np.max(d[big] / s_ora[big])
    assert np.all(d[~big] <= 1e-13 * s1)


def test_fp64_dense2048_parity(lib):
    A = synth.dense_case()
    o = orsvd.rsvd(A, k=64, p=10, q=2, seed=synth.SEED_DENSE)
    st, r, err = run(lib, A, k=64, p=10, q=2, seed=synth.SEED_DENSE)
    assert st == 0, lib.last_error()
    assert r["k"] == 64 and r["l"] == 74
    sigma_parity(r["S"].cpu().numpy(), o.S)
    e_o = orsvd.reconstruct_error(A, o.U, o.S, o.V)
    assert err <= 1.05 * e_o
    assert abs(r["err_est"] - o.err_est) <= 1e-10
    # singular vectors: same sign convention, columns agree where well separated
    U = r["U"].cpu().numpy()
    dots = np.abs(np.sum(U[:, :40] * o.U[:, :40], axis=0))
    assert np.all(dots > 1 - 1e-8)
    assert np.allclose(U[:, :40], o.U[:, :40], atol=1e-7)


@pytest.mark.parametrize("n,k,p,q", [(1, 1, 0, 0), (7, 3, 2, 1), (33, 8, 5, 0), (127, 20, 5, 2),
                                     (129, 64, 10, 1), (300, 40, 10, 2), (257, 250, 10, 0)])
def test_fp64_ragged_sizes(lib, n, k, p, q):
    rng = np.random.default_rng(n)
    sig = np.exp(-np.arange(1, n + 1) / max(2.0, n / 12))
    A = synth.planted_haar(n, sig, 100 + n)
    A += 1e-3 * rng.standard_normal((n, n)) * (A != 0)       # mildly non-symmetric, generic
    A = 0.5 * (A + A.T)
    o = orsvd.rsvd(A, k=k, p=p, q=q, seed=77)
    st, r, err = run(lib, A, k=k, p=p, q=q, seed=77)
    assert st in (0, 2), lib.last_error()       # 2 = rank capped (k + p > n)
    kk = min(k, n)
    assert r["k"] == kk
    sigma_parity(r["S"].cpu().numpy(), o.S[:kk])
    assert err <= 1.05 * orsvd.reconstruct_error(A, o.U, o.S, o.V) + 1e-14


def test_fp64_tolerance_mode(lib):
    n = 1500
    A = synth.batch_channel(3, n)
    o = orsvd.rsvd(A, tol=1e-4, l=128, q=1, seed=9)
    st, r, err = run(lib, A, k=118, p=10, q=1, seed=9, tol=1e-4, policy="tol", k_cap=128)
    assert st == 0, lib.last_error()
    assert r["k"] == o.k
    sigma_parity(r["S"].cpu().numpy(), o.S)
    assert err <= 1e-4 and err <= 1.05 * orsvd.reconstruct_error(A, o.U, o.S, o.V)


def test_fp64_rayleigh_ritz(lib):
    n = 600
    A = synth.planted_haar(n, synth.spectrum_exp(n, 12.0), 5)
    o = orsvd.rsvd(A, k=30, p=10, q=1, seed=4, rayleigh_ritz=True)
    st, r, err = run(lib, A, k=30, p=10, q=1, seed=4, rayleigh_ritz=True)
    assert st == 0, lib.last_error()
    sigma_parity(r["S"].cpu().numpy(), o.S)
    assert err <= 1.05 * orsvd.reconstruct_error(A, o.U, o.S, o.V)


def test_mixed_dense2048_error_ratio(lib):
    A = synth.dense_case()
    o = orsvd.rsvd(A, k=64, p=10, q=2, seed=synth.SEED_DENSE)
    e_o = orsvd.reconstruct_error(A, o.U, o.S, o.V)
    for slices in (2, 3):
        st, r, err = run(lib, A, k=64, p=10, q=2, seed=synth.SEED_DENSE, precision="bf16x", slices=slices)
        assert st == 0, lib.last_error()
        assert r["k"] == 64
        assert err <= 1.05 * e_o, (slices, err, e_o)
        # singular values: the small SVD runs in FP32 (absolute error ~ l 2^-24
        # sigma_1) on a projection whose entries carry the words' precision
        # (2^-(8 words + 1) relative); allow a factor 4 over their sum
        s = r["S"].cpu().numpy()
        bound = 4 * (74 * 2.0 ** -24 + 2.0 ** -(8 * slices + 1)) * o.S[0]
        assert np.max(np.abs(s - o.S)) <= bound, (slices, np.max(np.abs(s - o.S)), bound)


@pytest.mark.parametrize("n", [1000, 2500])
def test_mixed_tolerance_1e4(lib, n):
    A = synth.batch_channel(1, n)
    o = orsvd.rsvd(A, tol=1e-4, l=128, q=0, seed=3)
    e_o = orsvd.reconstruct_error(A, o.U, o.S, o.V)
    st, r, err = run(lib, A, k=118, p=10, q=0, seed=3, tol=1e-4, policy="tol", precision="bf16x",
                     slices=2, k_cap=128)
    assert st == 0, lib.last_error()
    assert err <= 1e-4
    # same draw, same algorithm: the rank may differ by the estimate's margin only
    assert o.k <= r["k"] <= o.k + 12
    assert abs(r["err_est"] - err) <= 0.35 * err


def test_batched_uneven_channels_fp64_and_mixed(lib):
    torch = _torch()
    sizes = [300, 1000, 129, 2100, 64]
    mats = [synth.batch_channel(c, n) for c, n in enumerate(sizes)]
    for prec in ("fp64", "bf16x"):
        plan = lib.Plan(max(sizes), k=40, p=10, q=1, seed=21, precision=prec)
        try:
            st, res = plan.decompose_batched([torch.as_tensor(A, device="cuda") for A in mats], 40)
            assert st == 0, lib.last_error()
            for A, r in zip(mats, res):
                o = orsvd.rsvd(A, k=40, p=10, q=1, seed=21)
                e_o = orsvd.reconstruct_error(A, o.U, o.S, o.V)
                err = plan.reconstruct_error(torch.as_tensor(A, device="cuda"), r)
                assert r["k"] == 40
                assert err <= 1.05 * e_o, (prec, A.shape[0], err, e_o)
                if prec == "fp64":
                    sigma_parity(r["S"].cpu().numpy(), o.S)
        finally:
            plan.close()


def test_host_buffers_match_device_buffers(lib):
    A = synth.batch_channel(2, 700)
    rs = lib
    plan = rs.Plan(700, k=20, p=10, q=1, seed=8)
    try:
        torch = _torch()
        st, rd = plan.decompose(torch.as_tensor(A, device="cuda"), 20)
        m = rs.dense(np.ascontiguousarray(A))
        f = rs.Factors()
        U = np.zeros((20, 700)); V = np.zeros((20, 700)); S = np.zeros(20)
        f.mem = rs.MEM_HOST; f.U = U.ctypes.data; f.ldu = 700; f.V = V.ctypes.data; f.ldv = 700
        f.S = S.ctypes.data; f.k_cap = 20
        st2 = rs.rsvd_decompose(plan.h, m, f)
        assert st == 0 and st2 == 0
        assert f.k_out == 20
        # k-split FP64 accumulation uses atomics, so two runs agree to rounding
        assert np.allclose(S, rd["S"].cpu().numpy(), rtol=1e-12, atol=0)
        assert np.allclose(U.T, rd["U"].cpu().numpy(), rtol=0, atol=1e-10)
        err_h = rs.rsvd_reconstruct_error(plan.h, m, f)
        assert abs(err_h - plan.reconstruct_error(torch.as_tensor(A, device="cuda"), rd)) < 1e-12
    finally:
        plan.close()


def test_nonfinite_input_reported(lib):
    A = synth.batch_channel(0, 200)
    A[17, 3] = np.nan
    st, r, _ = run(lib, A, k=10, p=5, q=0, seed=1)
    assert st == lib.RSVD_ERR_NONFINITE


def test_invalid_arguments_rejected(lib):
    torch = _torch()
    A = torch.zeros((50, 50), dtype=torch.float64, device="cuda")
    plan = lib.Plan(40, k=5, p=5)
    try:
        with pytest.raises(lib.RsvdError) as e:
            st, _ = plan.decompose(A, 5)          # n > n_max
            lib._check(st)
        assert e.value.status == lib.RSVD_ERR_INVALID_ARG
    finally:
        plan.close()


def test_mixed_tolerance_large_channel(lib):
    # largest channel size of the batched set: long k loops are where a biased
    # accumulation would show (error above the estimate)
    n = 11500
    A = synth.batch_channel(22, n)
    o = orsvd.rsvd(A, tol=1e-4, l=128, q=0, seed=5)
    st, r, err = run(lib, A, k=118, p=10, q=0, seed=5, tol=1e-4, policy="tol", precision="bf16x",
                     slices=2, k_cap=128)
    assert st == 0, lib.last_error()
    assert err <= 1e-4, err
    assert o.k <= r["k"] <= o.k + 12
    assert abs(r["err_est"] - err) <= 0.2 * err


@pytest.mark.parametrize("n,tol,b,q", [(900, 1e-4, 16, 0), (1500, 1e-5, 32, 1), (300, 1e-3, 8, 0)])
def test_fp64_adaptive_matches_oracle(lib, n, tol, b, q):
    A = synth.batch_channel(n % 7, n)
    o, drawn, met = orsvd.rsvd_adaptive(A, tol=tol, b=b, q=q, seed=13, l_max=600)
    st, r, err = run(lib, A, k=0, p=0, q=q, seed=13, tol=tol, policy="adaptive", block_b=b,
                     l_max=600, k_cap=600)
    assert st == 0, lib.last_error()
    assert met
    assert r["l"] == drawn and r["k"] == o.k
    sigma_parity(r["S"].cpu().numpy(), o.S)
    assert err <= tol and err <= 1.05 * orsvd.reconstruct_error(A, o.U, o.S, o.V)


def test_fp64_adaptive_batched_uneven(lib):
    torch = _torch()
    sizes = [400, 1200, 700]
    mats = [synth.batch_channel(c, n) for c, n in enumerate(sizes)]
    plan = lib.Plan(max(sizes), k=0, p=0, q=0, seed=2, tol=1e-4, policy="adaptive", block_b=16, l_max=400)
    try:
        st, res = plan.decompose_batched([torch.as_tensor(A, device="cuda") for A in mats], 400)
        assert st == 0, lib.last_error()
        for A, r in zip(mats, res):
            o, drawn, met = orsvd.rsvd_adaptive(A, tol=1e-4, b=16, q=0, seed=2, l_max=400)
            assert r["l"] == drawn and r["k"] == o.k
            sigma_parity(r["S"].cpu().numpy(), o.S)
    finally:
        plan.close()


# mixed-precision adaptive loop: the probe indicator (an upper confidence
# bound) replaces the exact one and the sketch columns are the FP32 evaluation
# of the Gaussian stream, so the draw may stop up to one block earlier or three
# later than the oracle's and the rank may sit above the oracle's by the
# bound's margin (more columns drawn can also mean a smaller rank)
@pytest.mark.parametrize("n,tol,b,q,slices", [(900, 1e-4, 16, 0, 2), (2500, 1e-4, 32, 0, 2),
                                              (1500, 1e-5, 32, 1, 3)])
def test_mixed_adaptive_meets_tolerance(lib, n, tol, b, q, slices):
    A = synth.batch_channel(n % 7, n)
    o, drawn, met = orsvd.rsvd_adaptive(A, tol=tol, b=b, q=q, seed=13, l_max=600)
    e_o = orsvd.reconstruct_error(A, o.U, o.S, o.V)
    st, r, err = run(lib, A, k=0, p=0, q=q, seed=13, tol=tol, policy="adaptive", block_b=b, l_max=600,
                     k_cap=600, precision="bf16x", slices=slices)
    assert st == 0, lib.last_error()
    assert met
    assert err <= tol, (err, tol)
    assert drawn - b <= r["l"] <= drawn + 3 * b, (r["l"], drawn)
    assert -max(8, 0.1 * o.k) <= r["k"] - o.k <= max(12, 0.25 * o.k), (r["k"], o.k)
    if r["k"] >= o.k and r["l"] >= drawn:
        assert err <= 1.05 * e_o, (err, e_o)
    assert abs(r["err_est"] - err) <= 0.35 * err


def test_mixed_adaptive_batched_uneven(lib):
    torch = _torch()
    sizes = [400, 1200, 700, 2100]
    mats = [synth.batch_channel(c, n) for c, n in enumerate(sizes)]
    plan = lib.Plan(max(sizes), k=0, p=0, q=0, seed=2, tol=1e-4, policy="adaptive", block_b=16, l_max=400,
                    precision="bf16x")
    try:
        dev = [torch.as_tensor(A, device="cuda") for A in mats]
        st, res = plan.decompose_batched(dev, 400)
        assert st == 0, lib.last_error()
        for A, At, r in zip(mats, dev, res):
            o, drawn, met = orsvd.rsvd_adaptive(A, tol=1e-4, b=16, q=0, seed=2, l_max=400)
            err = plan.reconstruct_error(At, r)
            assert err <= 1e-4, (A.shape[0], err)
            assert drawn - 16 <= r["l"] <= drawn + 48
            assert -max(8, 0.1 * o.k) <= r["k"] - o.k <= max(12, 0.25 * o.k)
    finally:
        plan.close()


def test_fp64_tolerance_1e6_batch_channels(lib):
    # the batched set's parity tolerance (1e-6): the noise floor (spectral
    # 1e-8 sigma_1) puts the rank near 700, so l = 800 and the small SVD runs
    # at l = 800 (one CTA per channel: seconds, see the design notes)
    torch = _torch()
    sizes = [1800, 2600]
    mats = [synth.batch_channel(c, n) for c, n in enumerate(sizes)]
    plan = lib.Plan(max(sizes), k=790, p=10, q=1, seed=9, tol=1e-6, policy="tol")
    try:
        dev = [torch.as_tensor(A, device="cuda") for A in mats]
        st, res = plan.decompose_batched(dev, 800)
        for A, At, r in zip(mats, dev, res):
            o = orsvd.rsvd(A, tol=1e-6, l=800, q=1, seed=9)
            e_o = orsvd.reconstruct_error(A, o.U, o.S, o.V)
            err = plan.reconstruct_error(At, r)
            assert r["status"] >= 0, (r["status"], lib.last_error())
            # the tail error crosses 1e-6 within ~1e-3 of tol here, so the
            # rank may differ by one between FP64 implementations
            assert abs(r["k"] - o.k) <= 1, (r["k"], o.k)
            kk = min(r["k"], o.k)
            sigma_parity(r["S"].cpu().numpy()[:kk], o.S[:kk])
            assert err <= 1e-6 * (1 + 1e-9)
            if r["k"] >= o.k:
                assert err <= 1.05 * e_o
    finally:
        plan.close()


def test_mixed_pinned_and_pageable_host_inputs(lib):
    # mixed path: a page-locked host V is read in place by the conversion
    # kernel, a pageable one is staged; both match the device-resident run
    torch = _torch()
    A = synth.batch_channel(4, 1500)
    pinned = torch.empty(A.shape, dtype=torch.float64, pin_memory=True)
    pinned.copy_(torch.as_tensor(A))
    for policy in ("tol", "adaptive"):
        plan = lib.Plan(1500, k=118, p=10, q=0, seed=4, tol=1e-4, policy=policy, precision="bf16x", block_b=32,
                        l_max=256)
        try:
            st0, r0 = plan.decompose(torch.as_tensor(A, device="cuda"), 128)
            e0 = plan.reconstruct_error(torch.as_tensor(A, device="cuda"), r0)
            for host in (pinned, np.ascontiguousarray(A)):
                st, r = plan.decompose(host, 128)
                assert st == st0 == 0, lib.last_error()
                assert r["k"] == r0["k"] and r["l"] == r0["l"]
                # split-k atomics reorder FP32 sums: agreement to the FP32 small
                # SVD's absolute accuracy (~l 2^-24 sigma_1)
                assert torch.allclose(r["S"], r0["S"], rtol=0, atol=1e-5 * float(r0["S"][0]))
                e = plan.reconstruct_error(torch.as_tensor(A, device="cuda"), r)
                assert abs(e - e0) <= 1e-3 * e0
        finally:
            plan.close()


def test_mixed_pinned_host_input_never_staged(lib):
    """Host-resident channel: on the mixed path a page-locked FP64 V is read
    once, in place, by the conversion kernel and never copied to the device;
    the plan's workspace holds only the BF16 words (4 B per entry with two
    words) and the n x l work, so channels whose FP64 matrix exceeds HBM while
    their words fit are decomposed from host memory."""
    torch = _torch()
    n = 6000
    A = synth.batch_channel(9, n)
    pinned = torch.empty(A.shape, dtype=torch.float64, pin_memory=True)
    pinned.copy_(torch.as_tensor(A))
    pageable = np.ascontiguousarray(A)
    sizes = {}
    for name, host in (("pinned", pinned), ("pageable", pageable)):
        plan = lib.Plan(n, k=118, p=10, q=0, seed=4, tol=1e-4, policy="tol", precision="bf16x")
        try:
            st, r = plan.decompose(host, 128)
            assert st >= 0, lib.last_error()
            e = plan.reconstruct_error(torch.as_tensor(A, device="cuda"), r)
            assert e <= 1e-4
            sizes[name] = lib.load().rsvd_plan_workspace_bytes(plan.h)
        finally:
            plan.close()
    # the staged (pageable) run needs the FP64 copy of V; the pinned run does not
    assert sizes["pageable"] - sizes["pinned"] >= 8 * n * n * 0.99, sizes
    assert sizes["pinned"] < 8 * n * n, sizes


@pytest.mark.parametrize("policy", ["fixed", "adaptive"])
def test_fp64_pinned_host_read_in_place(lib, monkeypatch, policy):
    """Host-resident channel on the FP64 path: when its staged copy would not
    fit the device (forced here with RSVD_HOST_IN_PLACE=1), every FP64 pass
    reads the page-locked V in place over the CPU-GPU link.  The workspace
    then holds no copy of V, and the result equals the device-resident run
    (the same kernels; only the order of the split-k atomic additions can
    differ) and the oracle's singular values."""
    torch = _torch()
    n, k = 3000, 40
    A = synth.planted_haar(n, synth.spectrum_exp(n, 10.0), 31)
    pinned = torch.empty(A.shape, dtype=torch.float64, pin_memory=True)
    pinned.copy_(torch.as_tensor(A))
    dev = torch.as_tensor(A, device="cuda")
    kw = dict(k=k, p=10, q=1, seed=4) if policy == "fixed" else dict(tol=1e-6, policy="adaptive", block_b=16, seed=4)
    out = {}
    for name, src in (("device", dev), ("host", pinned)):
        if name == "host":
            monkeypatch.setenv("RSVD_HOST_IN_PLACE", "1")
        plan = lib.Plan(n, precision="fp64", **kw)
        try:
            st, r = plan.decompose(src, 256)             # tol 1e-6 needs rank ~140 here
            assert st >= 0, lib.last_error()
            out[name] = (r["S"].cpu().numpy(), r["U"].cpu().numpy(), lib.load().rsvd_plan_workspace_bytes(plan.h))
        finally:
            plan.close()
        monkeypatch.delenv("RSVD_HOST_IN_PLACE", raising=False)
    (sd, ud, wd), (sh, uh, wh) = out["device"], out["host"]
    assert len(sd) == len(sh)
    assert np.max(np.abs(sd - sh)) <= 1e-12 * sd[0]
    assert np.max(np.abs(ud - uh)) <= 1e-9
    assert wh == wd, (wh, wd)                     # no staged copy: the device-resident layout
    if policy == "fixed":
        o = orsvd.rsvd(A, k=k, p=10, q=1, seed=4)
        big = o.S > 1e-12 * o.S[0]
        assert np.all(np.abs(sh[big] - o.S[big]) <= 1e-10 * o.S[big])
