"""The no-allocation residual entry point agrees with the regular one.

rsvd_reconstruct_error_noalloc serves callers that cannot allocate device
memory while checking a decomposition (a fully pre-reserved memory pool, or a
pipeline that must not be synchronised by cudaMalloc/cudaFree).  It keeps its
partial sums in a fixed array shared by all calls, so this test checks two
calls in a row -- the second reuses what the first left behind -- against
rsvd_reconstruct_error on the same factors and against the oracle's plain
FP64 residual of the same A and factors.  The file name makes pytest
collect it last.
"""
import pytest

from oracle import rsvd as orsvd
from paper_2307_15572_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_residual_matches_plan_residual_twice(lib):
    import torch

    results = []
    for n, k, seed in ((1500, 40, 3), (700, 25, 4)):
        A = torch.as_tensor(synth.batch_channel(seed, n), device="cuda")
        plan = lib.Plan(n, k=k, p=10, q=1, seed=seed)
        try:
            st, r = plan.decompose(A, k)
            assert st == 0, lib.last_error()
            ref = plan.reconstruct_error(A, r)
        finally:
            plan.close()
        f = r["_fac"]
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        st2 = lib.rsvd_reconstruct_error_noalloc(A.data_ptr(), n, n, f.U, f.ldu, f.S, f.V, f.ldv,
                                                 f.k_out, out.data_ptr(), None)
        assert st2 == 0
        torch.cuda.synchronize()
        got = float(out.item())
        # same FP64 arithmetic, same partials; only the final summation
        # order differs (device tree vs host loop)
        assert abs(got - ref) <= 1e-12 * max(ref, 1e-300), (n, got, ref)
        # and the oracle on the same A and factors (k FP64 products per entry)
        ora = orsvd.reconstruct_error(A.cpu().numpy(), r["U"].cpu().numpy(), r["S"].cpu().numpy(),
                                      r["V"].cpu().numpy())
        assert abs(got - ora) <= 1e-12 * ora + 1e-13, (n, got, ora)
        results.append(got)
    assert results[0] != results[1]


def test_noalloc_rejects_oversize_without_launching(lib):
    n = lib.RSVD_NOALLOC_MAX_N + 1
    st = lib.rsvd_reconstruct_error_noalloc(1, n, n, 1, n, 1, 1, n, 1, 1, None)
    assert st == lib.RSVD_ERR_INVALID_ARG
