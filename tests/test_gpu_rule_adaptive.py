"""The adaptive loop (randQB_EI blocks with the probe bound as the stop test)
on tile-rule channels, whose entries every pass generates: the tolerance is
met against the stored (materialised) matrices, and the loop draws the same
number of columns as on those stored copies, up to one block (the generated
entries and the stored FP32 copy differ by ~1e-6 relative)."""
import numpy as np
import pytest

from paper_2307_15572_gb300 import synth

pytestmark = pytest.mark.gpu

BLOCK, LMAX = 16, 256


def _materialise(lib, plan, m):
    import torch
    out = torch.empty((m.n, m.n), dtype=torch.float32, device="cuda")
    lib.rsvd_rule_rows(plan.h, m, 0, m.n, out.data_ptr(), m.n)
    return out.double()


@pytest.mark.parametrize("q", [0, 1])
def test_adaptive_on_rules_meets_tolerance(lib, q):
    chans = synth.learn_channel_params(5, seed=31, nlo=1500, nhi=4000, tlo=1e-4, thi=1e-2)
    descs = [lib.rule(ch["n"], ch["c"], ch["s"], ch["w"], eta=1e-7, seed=ch["seed"]) for ch in chans]
    nmax = max(ch["n"] for ch in chans)
    kw = dict(k=0, p=0, q=q, tol=1e-3, policy="adaptive", precision="bf16x", block_b=BLOCK, l_max=LMAX, seed=3)
    plan = lib.Plan(nmax, **kw)
    dplan = lib.Plan(nmax, **kw)
    try:
        dense = [_materialise(lib, plan, m) for m in descs]
        out = {}
        for name, pl, mats in (("rule", plan, descs), ("stored", dplan, [lib.dense(A) for A in dense])):
            facs, bufs = [], []
            for ch in chans:
                f, b = lib.Plan.factors_for(ch["n"], LMAX)
                f.tol = ch["tol"]
                facs.append(f)
                bufs.append(b)
            st, per = lib.rsvd_decompose_batched(pl.h, mats, facs)
            out[name] = (facs, per, bufs)
        for i, (ch, A) in enumerate(zip(chans, dense)):
            fr, sr = out["rule"][0][i], out["stored"][0][i]
            pr, ps = out["rule"][1][i], out["stored"][1][i]
            assert ps >= 0, (ps, lib.last_error())
            assert pr >= 0, (pr, lib.last_error())
            err = lib.rsvd_reconstruct_error(plan.h, lib.dense(A), fr)
            assert err <= ch["tol"] * (1 + 1e-3), (i, err, ch["tol"], fr.k_out, fr.l_used)
            assert abs(fr.l_used - sr.l_used) <= BLOCK, (i, fr.l_used, sr.l_used)
            assert abs(fr.k_out - sr.k_out) <= 2, (i, fr.k_out, sr.k_out)
            print(f"chan {i}: n {ch['n']} tol {ch['tol']:.1e} rule l {fr.l_used} k {fr.k_out} err {err:.2e}; "
                  f"stored l {sr.l_used} k {sr.k_out}")
    finally:
        plan.close()
        dplan.close()
