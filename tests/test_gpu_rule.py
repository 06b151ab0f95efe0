"""GPU parity of the matrix-free tile rule against the oracle.

* generated rows: the same entries as the oracle's rule (hash noise bit for
  bit up to FP32 rounding of its scale; smooth part within the BF16x3 /
  FP32-accumulation error of the tensor-core generator);
* a decomposition at n = 6000 (k = 50, error ~1e-4), several row panels:
  error within 1.05x the oracle's at the same (k, p, q, seed), singular
  values within the mixed path's bound;
* the full-size rule (n = 200,000, M = 300, k = 320, p = 10, q = 1), checked
  against the closed-form spectrum (the nonzero eigenvalues of G W G^T from
  the M x M matrix W^1/2 G^T G W^1/2) with Weyl's bound for the noise.
"""
import math

import numpy as np
import pytest

from oracle import rsvd as orsvd
from oracle import tilerule
from paper_2307_15572_gb300 import synth

pytestmark = pytest.mark.gpu


def _rows(lib, plan, m, r0, rows):
    import torch
    n = m.n
    out = torch.empty((rows, n), dtype=torch.float32, device="cuda")
    lib.rsvd_rule_rows(plan.h, m, r0, rows, out.data_ptr(), n)
    return out.cpu().numpy().astype(np.float64)


def test_rule_rows_match_oracle(lib):
    n, M = 3000, 300
    c, s, w = synth.rule_params(M=M, seed=synth.SEED_RULE)
    m = lib.rule(n, c, s, w, eta=1e-7, seed=synth.SEED_RULE)
    plan = lib.Plan(n, k=16, p=0, precision="bf16x")
    try:
        for r0, rows in ((0, 130), (1234, 200), (n - 77, 77)):
            g = _rows(lib, plan, m, r0, rows)
            ridx, cidx = np.arange(r0, r0 + rows), np.arange(n)
            a0 = tilerule.block(ridx, cidx, n, c, s, w, synth.SEED_RULE, 0.0)
            e = tilerule.eta(ridx, cidx, synth.SEED_RULE, 1e-7)
            # the factor as two FP16 words of its FP32 value times 2^14 / max H:
            # each factor entry within 2^-23 relative plus 2^-39 absolute (the
            # FP16 subnormal spacing, unscaled), so each of the M products
            # within 2^-22 h_i h_j + 2^-39 (h_i + h_j) <= ... + 2^-38; FP32
            # accumulation over M = 300 (20 tensor-core steps rounding toward
            # zero): 4e-6 relative to the (positive) smooth entry
            floor = 2.0 ** -38 * M
            bad = np.abs(g - (a0 + e)) - (4e-6 * a0 + floor)
            assert np.all(bad <= 0), (np.max(bad), np.max(np.abs(g - a0 - e)))
        # noise alone (all weights zero): the hash must agree exactly
        z = lib.rule(n, c, s, np.zeros(M), eta=1e-7, seed=99)
        g = _rows(lib, plan, z, 500, 64)
        e = tilerule.eta(np.arange(500, 564), np.arange(n), 99, 1e-7)
        assert np.max(np.abs(g - e)) <= 1e-7 * math.sqrt(3) * 2.0 ** -23
    finally:
        plan.close()


def test_rule_decompose_matches_oracle(lib, monkeypatch):
    import torch
    monkeypatch.setenv("RSVD_RULE_PANEL", "1024")          # several row panels
    n, M, k, p, q = 6000, 300, 50, 10, 1        # rank 50: error ~1e-4, the metric's tolerance
    c, s, w = synth.rule_params(M=M, seed=synth.SEED_RULE)
    A = tilerule.dense(n, c, s, w, synth.SEED_RULE, 1e-7)
    o = orsvd.rsvd(A, k=k, p=p, q=q, seed=7)
    e_o = orsvd.reconstruct_error(A, o.U, o.S, o.V)
    m = lib.rule(n, c, s, w, eta=1e-7, seed=synth.SEED_RULE)
    for slices in (2, 3):
        plan = lib.Plan(n, k=k, p=p, q=q, seed=7, precision="bf16x", slices=slices)
        try:
            st, r = plan.decompose(m, k)
            assert st == 0, lib.last_error()
            assert r["k"] == k and r["l"] == k + p
            At = torch.as_tensor(A, device="cuda")
            E = At - (r["U"] * r["S"]) @ r["V"].T
            err = (torch.linalg.norm(E) / torch.linalg.norm(At)).item()
            assert err <= 1.05 * e_o, (slices, err, e_o)
            sg = r["S"].cpu().numpy()
            bound = 4 * ((k + p) * 2.0 ** -24 + 2.0 ** -(8 * slices + 1)) * o.S[0]
            assert np.max(np.abs(sg - o.S)) <= bound, (slices, np.max(np.abs(sg - o.S)), bound)
        finally:
            plan.close()


@pytest.mark.parametrize("slices", [2, 3])
def test_rule_full_size_closed_form(lib, slices):
    """The full-size rule in both word formats (two words is the benchmark's
    configuration).  With two words the exact residual is also taken: every
    entry regenerated in FP64 on the device.  It lies between the noise floor
    no rank-320 form can go below -- the hash noise, ||eta||_F^2 = n^2 1e-14
    (std 1e-7, uniform), less at most 320 ||eta||_2^2 (0.7 % of it) -- and
    the rank rule's estimate, which adds the mixed path's precision floor
    (FP32 factors, 2 sqrt(l) eps_32 ~ 2.2e-6) to what its probes see."""
    n, M, k, p, q = 200000, 300, 320, 10, 1
    c, s, w = synth.rule_params(M=M, seed=synth.SEED_RULE)
    lam = tilerule.closed_form_eigs(n, c, s, w)
    fro0 = math.sqrt(tilerule.closed_form_fro2(n, c, s, w))
    m = lib.rule(n, c, s, w, eta=1e-7, seed=synth.SEED_RULE)
    plan = lib.Plan(n, k=k, p=p, q=q, seed=11, precision="bf16x", slices=slices)
    try:
        st, r = plan.decompose(m, k)
        # rank 320 is far past the rule's numerical rank (~80 above the
        # noise), so the sketch is ill-conditioned and CholeskyQR takes its
        # shifted form (status RSVD_WARN_SHIFTED_CQR)
        assert st in (0, 1), lib.last_error()
        sg = r["S"].cpu().numpy()
        U = r["U"]
        import torch
        orth = torch.linalg.norm(U.T @ U - torch.eye(k, dtype=torch.float64, device="cuda")).item()
        exact = plan.reconstruct_error(m, r) if slices == 2 else None
    finally:
        plan.close()
    if exact is not None:
        noise_rel = 1e-7 * n / fro0
        assert 0.99 * noise_rel <= exact <= r["err_est"], (exact, noise_rel, r["err_est"])
        floor = 2.0 * math.sqrt(k + p) * 2.0 ** -24
        assert exact <= math.hypot(noise_rel, floor), (exact, noise_rel, floor)
    assert orth <= 1e-4, orth
    # Weyl: |sigma_i(A0 + eta) - lambda_i(A0)| <= ||eta||_2 (semicircle edge
    # 2 sqrt(n) std, x1.1); three words and FP32 factors add ~l 2^-24 sigma_1
    # and the generator's 4e-6 relative error of the entries (<= 4e-6 ||A0||_F)
    eta2 = 1.1 * 2 * math.sqrt(n) * 1e-7
    slack = eta2 + 4 * (k + p) * 2.0 ** -24 * lam[0] + 4e-6 * fro0
    # A0 = G W G^T is positive semidefinite of rank <= M: its singular values
    # are the eigenvalues (clipped at the numerical zero), then zeros
    top = np.concatenate([np.maximum(lam, 0.0), np.zeros(max(0, k - M))])[:k]
    assert np.all(np.abs(sg - top) <= slack), (np.max(np.abs(sg - top)), slack)
    # and every value to FP32-level accuracy relative to sigma_1 (the FP32
    # small SVD, the generator's ~2e-7 relative rounding bias)
    dev = np.abs(sg - top)
    assert np.all(dev <= eta2 + 2e-6 * lam[0]), (dev.max() / lam[0], np.argmax(dev))


@pytest.mark.parametrize("q", [0, 1])
def test_rule_fp64_path_matches_oracle(lib, monkeypatch, q):
    """FP64 path on a tile rule (every pass generates its FP64 row panels on
    CUDA cores): the all-FP64 bar against the oracle run on the rule's dense
    matrix -- singular values within 1e-10 relative (above 1e-12 sigma_1),
    error within 1.05x the oracle's -- with several row panels."""
    import torch
    monkeypatch.setenv("RSVD_RULE_PANEL", "1024")
    n, M, k, p = 2500, 300, 40, 10
    c, s, w = synth.rule_params(M=M, seed=synth.SEED_RULE)
    A = tilerule.dense(n, c, s, w, synth.SEED_RULE, 1e-7)
    o = orsvd.rsvd(A, k=k, p=p, q=q, seed=7)
    e_o = orsvd.reconstruct_error(A, o.U, o.S, o.V)
    m = lib.rule(n, c, s, w, eta=1e-7, seed=synth.SEED_RULE)
    plan = lib.Plan(n, k=k, p=p, q=q, seed=7, precision="fp64")
    try:
        st, r = plan.decompose(m, k)
        assert st >= 0, lib.last_error()
        assert r["k"] == k and r["l"] == k + p
        sg = r["S"].cpu().numpy()
        big = o.S > 1e-12 * o.S[0]
        assert np.all(np.abs(sg[big] - o.S[big]) <= 1e-10 * o.S[big]), np.max(np.abs(sg - o.S) / o.S)
        At = torch.as_tensor(A, device="cuda")
        E = At - (r["U"] * r["S"]) @ r["V"].T
        err = (torch.linalg.norm(E) / torch.linalg.norm(At)).item()
        assert err <= 1.05 * e_o, (err, e_o)
        # ||V||_F^2 from the generated panels: the FP64 estimate agrees with the oracle's
        assert abs(r["err_est"] - o.err_est) <= 1e-10, (r["err_est"], o.err_est)
    finally:
        plan.close()


def test_rule_fp64_tolerance_policy(lib):
    """Tolerance mode on the FP64 path over a generated rule: error <= tol."""
    import torch
    n, M = 3000, 300
    c, s, w = synth.rule_params(M=M, seed=synth.SEED_RULE)
    A = tilerule.dense(n, c, s, w, synth.SEED_RULE, 1e-7)
    m = lib.rule(n, c, s, w, eta=1e-7, seed=synth.SEED_RULE)
    plan = lib.Plan(n, k=90, p=10, q=1, tol=1e-4, policy="tol", seed=5, precision="fp64")
    try:
        st, r = plan.decompose(m, 90)
        assert st >= 0, lib.last_error()
        At = torch.as_tensor(A, device="cuda")
        E = At - (r["U"] * r["S"]) @ r["V"].T
        err = (torch.linalg.norm(E) / torch.linalg.norm(At)).item()
        assert err <= 1e-4, (err, r["k"])
        o = orsvd.rsvd(A, tol=1e-4, l=100, q=1, seed=5)
        assert abs(r["k"] - len(o.S)) <= 1, (r["k"], len(o.S))
    finally:
        plan.close()
