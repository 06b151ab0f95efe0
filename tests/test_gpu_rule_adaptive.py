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


def test_fp64_adaptive_on_rule_matches_oracle(lib):
    """FP64 path, adaptive loop on a generated rule: the same columns drawn,
    the same rank and singular values (1e-10 relative) as the oracle's loop
    on the rule's dense matrix."""
    import torch
    from oracle import rsvd as orsvd
    from oracle import tilerule
    n, M, tol, b = 2000, 300, 1e-4, 16
    c, s, w = synth.rule_params(M=M, seed=synth.SEED_RULE)
    A = tilerule.dense(n, c, s, w, synth.SEED_RULE, 1e-7)
    o, drawn, met = orsvd.rsvd_adaptive(A, tol=tol, b=b, q=0, seed=2, l_max=200)
    m = lib.rule(n, c, s, w, eta=1e-7, seed=synth.SEED_RULE)
    plan = lib.Plan(n, k=0, p=0, q=0, seed=2, tol=tol, policy="adaptive", block_b=b, l_max=200, precision="fp64")
    try:
        st, r = plan.decompose(m, 200)
        assert st >= 0 and met, lib.last_error()
        assert r["l"] == drawn and r["k"] == o.k, (r["l"], drawn, r["k"], o.k)
        sg = r["S"].cpu().numpy()
        big = o.S > 1e-12 * o.S[0]
        assert np.all(np.abs(sg[big] - o.S[big]) <= 1e-10 * o.S[big])
        At = torch.as_tensor(A, device="cuda")
        err = (torch.linalg.norm(At - (r["U"] * r["S"]) @ r["V"].T) / torch.linalg.norm(At)).item()
        assert err <= tol
    finally:
        plan.close()


def test_fp64_probe_features_on_rule_match_dense(lib):
    """The FP64 probe of a generated rule gives the features of its dense matrix."""
    import torch
    from oracle import tilerule
    chans = synth.learn_channel_params(3, seed=41, nlo=1200, nhi=2500, tlo=1e-4, thi=1e-2)
    nmax = max(ch["n"] for ch in chans)
    plan = lib.Plan(nmax, k=16, p=0, precision="fp64", seed=1)
    try:
        descs = [lib.rule(ch["n"], ch["c"], ch["s"], ch["w"], eta=1e-7, seed=ch["seed"]) for ch in chans]
        dense = [torch.as_tensor(tilerule.dense(ch["n"], ch["c"], ch["s"], ch["w"], ch["seed"], 1e-7), device="cuda")
                 for ch in chans]
        tols = [ch["tol"] for ch in chans]
        Fr = torch.empty((len(chans), 19), dtype=torch.float32, device="cuda")
        Fd = torch.empty_like(Fr)
        lib.rsvd_probe_features(plan.h, descs, tols, Fr.data_ptr())
        lib.rsvd_probe_features(plan.h, [lib.dense(A) for A in dense], tols, Fd.data_ptr())
        Fr, Fd = Fr.cpu().numpy(), Fd.cpu().numpy()
        lead = Fd[:, :15] > np.log(1e-6)
        assert np.max(np.abs(Fr - Fd)[:, :15][lead]) <= 1e-4, np.max(np.abs(Fr - Fd)[:, :15][lead])
        assert np.max(np.abs(Fr[:, 15:] - Fd[:, 15:])) <= 1e-5
    finally:
        plan.close()
