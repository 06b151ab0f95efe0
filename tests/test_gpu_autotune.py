"""The launch-shape autotuner: every candidate shape of the grouped passes
gives the decomposition of the default shape (up to the order of FP32/FP64
summation), a plan tunes each pass signature once, and tuned plans replay
through CUDA graphs."""
import numpy as np
import pytest

from paper_2307_15572_gb300 import synth

pytestmark = pytest.mark.gpu


def _run(lib, plan, mats, kcap):
    import torch
    st, res = plan.decompose_batched(mats, kcap)
    torch.cuda.synchronize()
    assert st >= 0, lib.last_error()
    return res


def _same(lib, plan, mats, ref, res, rt, at=0.0, et=1e-3):
    """Same factors up to summation order: singular values within rt relative
    plus at * sigma_1 absolute (the mixed path's FP32 accumulation moves the
    small ones by a few FP32 ulps of sigma_1), residuals within et relative
    (at k = 150 the mixed residual, ~2.3e-5, sits near the FP32 accumulation
    floor and moves by ~0.15% with the summation order)."""
    import torch
    for A, a, b in zip(mats, ref, res):
        assert a["k"] == b["k"] and a["l"] == b["l"]
        atol = at * float(a["S"][0])
        assert torch.allclose(a["S"], b["S"], rtol=rt, atol=atol), (a["S"] - b["S"]).abs().max()
        e0 = plan.reconstruct_error(A, a)
        e1 = plan.reconstruct_error(A, b)
        assert abs(e0 - e1) <= et * e0, (e0, e1)


# few channels: the k-split candidates differ; the mixed batch needs more than
# one column tile at l + probe columns > 160
CASES = {
    "fp64": dict(sizes=[2048, 1500], kw=dict(k=64, p=10, q=1, precision="fp64"), rt=1e-10, at=0.0, et=1e-3),
    "bf16x": dict(sizes=[3000, 1200, 2222], kw=dict(k=150, p=10, q=1, precision="bf16x"), rt=1e-5, at=1e-6, et=1e-2),
}


@pytest.mark.parametrize("prec", ["fp64", "bf16x"])
def test_every_candidate_matches_default(lib, prec, monkeypatch):
    import torch
    cs = CASES[prec]
    mats = [torch.as_tensor(synth.batch_channel(c, n), device="cuda") for c, n in enumerate(cs["sizes"])]
    kcap = cs["kw"]["k"]
    base = lib.Plan(max(cs["sizes"]), seed=4, **cs["kw"])
    try:
        ref = _run(lib, base, mats, kcap)
        ncand = None
        for force in range(16):
            monkeypatch.setenv("RSVD_TUNE_FORCE", str(force))
            plan = lib.Plan(max(cs["sizes"]), seed=4, autotune=True, **cs["kw"])
            try:
                res = _run(lib, plan, mats, kcap)
                recs = lib.rsvd_plan_tune_records(plan.h)
                assert recs, "nothing was tuned"
                ncand = max(r["candidates"] for r in recs)
                for r in recs:
                    assert r["choice"] == force % r["candidates"]
                    assert r["ms_best"] > 0 and r["ms_default"] > 0
                _same(lib, base, mats, ref, res, cs["rt"], cs["at"], cs["et"])
                # a second call on the tuned plan tunes nothing new and agrees
                res2 = _run(lib, plan, mats, kcap)
                assert len(lib.rsvd_plan_tune_records(plan.h)) == len(recs)
                _same(lib, base, mats, ref, res2, cs["rt"], cs["at"], cs["et"])
            finally:
                plan.close()
            if force + 1 >= ncand:
                break
        assert ncand >= 2, "only one candidate shape"
    finally:
        base.close()


def test_tuned_plan_replays_in_graphs(lib):
    import torch
    sizes = [700, 1500, 333, 2500]
    sets = [[torch.as_tensor(synth.batch_channel(c + 10 * r, n), device="cuda") for c, n in enumerate(sizes)]
            for r in range(3)]
    s = torch.cuda.Stream()
    kw = dict(k=40, p=10, q=1, seed=3, tol=1e-3, policy="tol", precision="bf16x", stream=s.cuda_stream)
    direct = lib.Plan(max(sizes), **kw)
    tuned = lib.Plan(max(sizes), autotune=True, **kw)
    lib.rsvd_plan_set_graphs(tuned.h, True)
    try:
        counts = []
        for mats in sets:              # tunes (direct launches), then captures, then replays
            r0 = _run(lib, direct, mats, 50)
            r1 = _run(lib, tuned, mats, 50)
            _same(lib, direct, mats, r0, r1, 1e-5, 1e-6)
            counts.append(len(lib.rsvd_plan_tune_records(tuned.h)))
        assert counts[0] > 0 and counts[0] == counts[1] == counts[2]
        for r in lib.rsvd_plan_tune_records(tuned.h):
            assert 0 <= r["choice"] < r["candidates"]
            assert r["ms_best"] <= r["ms_default"]
    finally:
        direct.close()
        tuned.close()
