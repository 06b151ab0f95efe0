"""The exact residual kernels against the oracle's residual on the same factors.

Every mixed-path tolerance assertion and the benchmark's verification read
the residual of ``rsvd_reconstruct_error``; here it is pinned to
``oracle.rsvd.reconstruct_error(A, U, S, V)`` (a plain FP64 numpy evaluation
of ||A - U diag(S) V^T||_F / ||A||_F) on the same A and the same factors --
factors from GPU decompositions and random ones (an O(1) residual), sizes
from one entry to several tiles with ragged tails, k from 0 up, the A = 0
case, and tile rules (entries regenerated in FP64 on the device, compared
with the oracle's dense rule matrix).

Bound: each entry of U diag(S) V^T is a sum of k FP64 products, so the two
evaluations differ by about k u ||A||_F in the residual, i.e. at most
1e-12 relative plus 1e-13 of ||A||_F.
"""
import numpy as np
import pytest

from oracle import rsvd as orsvd
from oracle import tilerule
from paper_2307_15572_gb300 import synth

pytestmark = pytest.mark.gpu


def _close(got, ref):
    return abs(got - ref) <= 1e-12 * ref + 1e-13


def _factors(lib, U, S, V):
    import torch
    n, k = U.shape
    kc = max(k, 1)
    Ut = torch.zeros((kc, n), dtype=torch.float64, device="cuda")
    Vt = torch.zeros((kc, n), dtype=torch.float64, device="cuda")
    St = torch.zeros((kc,), dtype=torch.float64, device="cuda")
    if k:
        Ut[:k] = torch.as_tensor(U.T, device="cuda")
        Vt[:k] = torch.as_tensor(V.T, device="cuda")
        St[:k] = torch.as_tensor(S, device="cuda")
    f = lib.Factors()
    f.mem = lib.MEM_DEVICE
    f.U, f.ldu = Ut.data_ptr(), n
    f.V, f.ldv = Vt.data_ptr(), n
    f.S = St.data_ptr()
    f.k_cap = kc
    f.k_out = k
    return f, (Ut, St, Vt)


def _noalloc(lib, A_colmajor_t, f, n):
    import torch
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    st = lib.rsvd_reconstruct_error_noalloc(A_colmajor_t.data_ptr(), n, n, f.U, f.ldu, f.S, f.V, f.ldv, f.k_out,
                                            out.data_ptr(), None)
    assert st == 0, lib.last_error()
    torch.cuda.synchronize()
    return float(out.item())


@pytest.mark.parametrize("n,k", [(1, 0), (1, 1), (65, 0), (65, 1), (65, 64), (4097, 1), (4097, 118),
                                 (11500, 118)])
def test_residual_random_factors_match_oracle(lib, n, k):
    import torch
    rng = np.random.default_rng(1000 + n + k)
    B = rng.standard_normal((n, n))
    A = 0.5 * (B + B.T)                                  # symmetric: the plan call's contract
    U = rng.standard_normal((n, k)) / np.sqrt(n)
    V = rng.standard_normal((n, k)) / np.sqrt(n)
    S = np.sort(rng.uniform(0.1, 3.0, size=k))[::-1].copy()
    ref = orsvd.reconstruct_error(A, U, S, V)
    At = torch.as_tensor(A, device="cuda")
    f, keep = _factors(lib, U, S, V)
    plan = lib.Plan(n, k=1, p=0)
    try:
        got = lib.rsvd_reconstruct_error(plan.h, lib.dense(At), f)
    finally:
        plan.close()
    assert _close(got, ref), (n, k, got, ref)
    if n <= lib.RSVD_NOALLOC_MAX_N:
        # a general (non-symmetric) matrix, column-major: the entry point
        # reads A[r + c lda], i.e. the transpose of the row-major tensor
        Bt = torch.as_tensor(np.ascontiguousarray(B.T), device="cuda")
        ref_b = orsvd.reconstruct_error(B, U, S, V)
        assert _close(_noalloc(lib, Bt, f, n), ref_b)


def test_residual_of_gpu_factors_matches_oracle(lib):
    import torch
    for n, k, prec in ((11500, 118, "bf16x"), (4097, 60, "fp64")):
        A = synth.batch_channel(7, n)
        At = torch.as_tensor(A, device="cuda")
        plan = lib.Plan(n, k=k, p=10, q=0, seed=3, precision=prec)
        try:
            st, r = plan.decompose(At, k)
            assert st >= 0, lib.last_error()
            got = plan.reconstruct_error(At, r)
        finally:
            plan.close()
        U, S, V = (x.cpu().numpy() for x in (r["U"], r["S"], r["V"]))
        ref = orsvd.reconstruct_error(A, U, S, V)
        assert _close(got, ref), (n, prec, got, ref)
        assert _close(_noalloc(lib, At, r["_fac"], n), ref)


def test_residual_zero_matrix_is_absolute(lib):
    import torch
    n, k = 130, 3
    rng = np.random.default_rng(5)
    U = rng.standard_normal((n, k))
    V = rng.standard_normal((n, k))
    S = np.array([2.0, 1.0, 0.5])
    Z = np.zeros((n, n))
    ref = orsvd.reconstruct_error(Z, U, S, V)
    assert ref > 0
    f, keep = _factors(lib, U, S, V)
    Zt = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    plan = lib.Plan(n, k=1, p=0)
    try:
        got = lib.rsvd_reconstruct_error(plan.h, lib.dense(Zt), f)
    finally:
        plan.close()
    assert _close(got, ref), (got, ref)
    assert _close(_noalloc(lib, Zt, f, n), ref)


def test_residual_host_inputs_match_device(lib):
    import torch
    n, k = 700, 20
    rng = np.random.default_rng(8)
    B = rng.standard_normal((n, n))
    A = 0.5 * (B + B.T)
    U = rng.standard_normal((n, k)) / np.sqrt(n)
    V = rng.standard_normal((n, k)) / np.sqrt(n)
    S = rng.uniform(0.5, 2.0, size=k)
    ref = orsvd.reconstruct_error(A, U, S, V)
    Uh = np.ascontiguousarray(U.T)
    Vh = np.ascontiguousarray(V.T)
    Sh = np.ascontiguousarray(S)
    f = lib.Factors()
    f.mem = lib.MEM_HOST
    f.U, f.ldu = Uh.ctypes.data, n
    f.V, f.ldv = Vh.ctypes.data, n
    f.S = Sh.ctypes.data
    f.k_cap = k
    f.k_out = k
    plan = lib.Plan(n, k=1, p=0)
    try:
        got = lib.rsvd_reconstruct_error(plan.h, lib.dense(A), f)
    finally:
        plan.close()
    assert _close(got, ref), (got, ref)


@pytest.mark.parametrize("prec", ["bf16x", "fp64"])
def test_rule_residual_matches_oracle_dense(lib, prec):
    """Tile rule: the residual regenerates every entry in FP64 and must equal
    the oracle's residual on its dense rule matrix."""
    import torch
    n, M, k = 3001, 300, 40
    c, s, w = synth.rule_params(M=M, seed=synth.SEED_RULE)
    A = tilerule.dense(n, c, s, w, synth.SEED_RULE, 1e-7)
    m = lib.rule(n, c, s, w, eta=1e-7, seed=synth.SEED_RULE)
    plan = lib.Plan(n, k=k, p=10, q=1, seed=4, precision=prec)
    try:
        st, r = plan.decompose(m, k)
        assert st >= 0, lib.last_error()
        got = plan.reconstruct_error(m, r)
        # random factors too: an O(1) residual
        rng = np.random.default_rng(3)
        U7 = rng.standard_normal((n, 7)) / np.sqrt(n)
        V7 = rng.standard_normal((n, 7)) / np.sqrt(n)
        S7 = rng.uniform(0.5, 2.0, 7)
        f, keep = _factors(lib, U7, S7, V7)
        got_r = lib.rsvd_reconstruct_error(plan.h, m, f)
        ref_r = orsvd.reconstruct_error(A, U7, S7, V7)
    finally:
        plan.close()
    Ug, Sg, Vg = (x.cpu().numpy() for x in (r["U"], r["S"], r["V"]))
    ref = orsvd.reconstruct_error(A, Ug, Sg, Vg)
    assert _close(got, ref), (got, ref)
    assert _close(got_r, ref_r), (got_r, ref_r)
    # and against the dense FP64 copy of the same rule through the stored path
    plan = lib.Plan(n, k=1, p=0)
    try:
        got_d = lib.rsvd_reconstruct_error(plan.h, lib.dense(torch.as_tensor(A, device="cuda")), r["_fac"])
    finally:
        plan.close()
    assert _close(got_d, ref)
