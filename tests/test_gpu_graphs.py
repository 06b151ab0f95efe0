"""CUDA-graph replay of decompositions: the same results as direct launches
(up to the order of split-k atomic additions), with new input and output
buffers on every call."""
import numpy as np
import pytest

from paper_2307_15572_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "bf16x"])
def test_graph_replay_matches_direct(lib, prec):
    import torch
    sizes = [700, 1500, 333]
    sets = [[torch.as_tensor(synth.batch_channel(c + 10 * r, n), device="cuda") for c, n in enumerate(sizes)]
            for r in range(3)]
    s = torch.cuda.Stream()
    kw = dict(k=40, p=10, q=1, seed=3, tol=1e-3, policy="tol", precision=prec, stream=s.cuda_stream)
    direct = lib.Plan(max(sizes), **kw)
    graphed = lib.Plan(max(sizes), **kw)
    lib.rsvd_plan_set_graphs(graphed.h, True)
    try:
        for mats in sets:                           # first call captures, the rest replay
            st0, r0 = direct.decompose_batched(mats, 50)
            st1, r1 = graphed.decompose_batched(mats, 50)
            torch.cuda.synchronize()
            assert st0 == st1 and st0 >= 0, lib.last_error()
            rt = 1e-10 if prec == "fp64" else 1e-5
            for A, a, b in zip(mats, r0, r1):
                assert a["k"] == b["k"] and a["l"] == b["l"] and a["status"] == b["status"]
                assert torch.allclose(a["S"], b["S"], rtol=rt, atol=0)
                e0 = direct.reconstruct_error(A, a)
                e1 = graphed.reconstruct_error(A, b)
                assert abs(e0 - e1) <= 1e-3 * e0
        prof = lib.rsvd_plan_profile(graphed.h)
        assert prof["launches"] > 0
    finally:
        direct.close()
        graphed.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x"])
def test_rule_graph_replay_matches_direct(lib, monkeypatch, prec):
    """Tile-rule channels replayed from a CUDA graph (several row panels):
    the same results as direct launches, with new rule centres, widths and
    weights of the same scale, and new outputs, on every call; a different
    noise seed makes a new graph."""
    import torch
    monkeypatch.setenv("RSVD_RULE_PANEL", "1024")
    s = torch.cuda.Stream()
    kw = dict(k=30, p=10, q=1, seed=3, tol=1e-3, policy="tol", precision=prec, stream=s.cuda_stream)
    direct = lib.Plan(3000, **kw)
    graphed = lib.Plan(3000, **kw)
    lib.rsvd_plan_set_graphs(graphed.h, True)
    try:
        for r, seed in enumerate((5, 5, 6, 6)):
            mats = []
            for c, n in enumerate((2500, 1300)):
                cc, ss, ww = synth.rule_params(M=120, seed=100 + 10 * r + c, decay=10.0)
                mats.append(lib.rule(n, cc, ss, ww, eta=1e-7, seed=seed))
            st0, r0 = direct.decompose_batched(mats, 40)
            st1, r1 = graphed.decompose_batched(mats, 40)
            torch.cuda.synchronize()
            assert st0 == st1 and st0 >= 0, lib.last_error()
            for a, b in zip(r0, r1):
                assert a["k"] == b["k"] and a["l"] == b["l"]
                rt = 1e-10 if prec == "fp64" else 1e-5
                assert torch.allclose(a["S"], b["S"], rtol=rt, atol=0)
    finally:
        direct.close()
        graphed.close()
