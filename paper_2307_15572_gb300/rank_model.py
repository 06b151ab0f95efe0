"""Train the rank model on a seeded channel population and write its blob.

Run on a GPU (every arithmetic step goes through the library's kernels):

    python -m paper_2307_15572_gb300.rank_model --out <dir> [--count 4000 --held 500 ...]

Steps:
  1. population: ``synth.learn_population`` -- dense symmetric channels with
     sizes uniform in [nlo, nhi], spectra a e^{-i/tau} + (1 - a) i^{-beta}
     (a ~ U[0,1], tau ~ logU[5, 200], beta ~ U[1.5, 4]) and tolerances
     log-uniform in [tlo, thi]; the last ``held`` channels are held out;
  2. labels: the plain adaptive loop on the FP64 path (randQB_EI, blocks of
     16, at most l_max columns) gives each channel's rank k* and drawn
     columns l*; channels it cannot finish within l_max are left out of
     training;
  3. features: the 16-column probe of each precision (FP64 and the mixed
     path's one-word probe), ``rsvd_probe_features``;
  4. training: ``learn.train`` (standardisation, minibatches, forward,
     backward, Adam and folding in the library's kernels), one network per
     probe precision;
  5. held-out report: on the held-out channels the plain adaptive loop can
     finish within l_max, the learned policy against that loop in the same
     precision -- channels meeting the tolerance, passes over V, wall time --
     FP64 on all of them, the mixed path on those whose tolerance is above its
     precision floor; and the prediction error of log k and log p.

Writes ``rank_model_fp64.bin`` and ``rank_model_bf16x.bin`` (FP32 parameter
blobs in the layout of include/rsvd_mlp.h, little-endian) and
``rank_model.json`` (the recipe, training losses and the held-out report).
Matrices are made and dropped in chunks, so memory stays bounded.
"""

import argparse
import json
import os
import time

import numpy as np

from . import learn, rsvd, synth


def _chunks(seq, size):
    for i in range(0, len(seq), size):
        yield i, seq[i:i + size]


def label_and_features(pop, lmax, block, chunk, seed, label_precision="fp64", models=("fp64", "bf16x")):
    """(k*, l*, met, features per precision) over the population, in chunks."""
    import torch
    ks, ls, met = [], [], []
    feats = {p: [] for p in models}
    for i, sub in _chunks(pop, chunk):
        mats = learn.matrices(sub)
        k, l_, m = learn.label(sub, mats, block=block, lmax=lmax, seed=seed, chunk=chunk,
                               precision=label_precision)
        ks.append(k)
        ls.append(l_)
        met.append(m)
        for prec in feats:
            feats[prec].append(learn.features(sub, mats, prec, seed=seed, chunk=chunk))
        del mats
        torch.cuda.empty_cache()
    return (np.concatenate(ks), np.concatenate(ls), np.concatenate(met),
            {p: torch.cat(v) for p, v in feats.items()})


def compare(pop, theta, precision, lmax, chunk, seed, slices):
    """Learned against adaptive on the given channels (same precision)."""
    import torch
    out = {}
    for policy in ("adaptive", "learned"):
        tot_t, passes, oks, errs = 0.0, 0, [], []
        for i, sub in _chunks(pop, chunk):
            mats = learn.matrices(sub)
            stats = {}
            dt, facs, per, e = learn.run_policy(sub, mats, policy, precision,
                                                theta=theta if policy == "learned" else None,
                                                block=16 if precision == "fp64" else 32, lmax=lmax, seed=seed,
                                                slices=slices, repeat=1, stats=stats)
            tol = np.array([ch["tol"] for ch in sub])
            tot_t += dt
            passes += stats["passes"]
            oks.append((np.array([s >= 0 for s in per])) & (e <= tol * (1 + 1e-9)))
            errs.append(e / tol)
            del mats
            torch.cuda.empty_cache()
        ok = np.concatenate(oks)
        out[policy] = {"seconds": tot_t, "passes_over_v": int(passes), "met": int(ok.sum()),
                       "channels": len(pop), "max_err_over_tol": float(np.max(np.concatenate(errs)))}
    return out


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--count", type=int, default=4000)
    ap.add_argument("--held", type=int, default=500)
    ap.add_argument("--nlo", type=int, default=500)
    ap.add_argument("--nhi", type=int, default=6000)
    ap.add_argument("--tlo", type=float, default=1e-7)
    ap.add_argument("--thi", type=float, default=1e-3)
    ap.add_argument("--lmax", type=int, default=512)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--chunk", type=int, default=64)
    ap.add_argument("--seed", type=int, default=synth.SEED_LEARN)
    ap.add_argument("--mixed-floor", type=float, default=1e-5,
                    help="held-out tolerances at least this large are also compared on the mixed path")
    ap.add_argument("--label-precision", default="fp64", choices=["fp64", "bf16x"],
                    help="path of the adaptive loop that labels the channels")
    ap.add_argument("--models", default="fp64,bf16x", help="probe precisions to train a network for")
    ap.add_argument("--tag", default="", help="suffix of the written file names")
    a = ap.parse_args()
    models = tuple(a.models.split(","))
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    pop = synth.learn_population(a.count, seed=a.seed, nlo=a.nlo, nhi=a.nhi, tlo=a.tlo, thi=a.thi)
    ks, ls, met, feats = label_and_features(pop, a.lmax, 16 if a.label_precision == "fp64" else 32, a.chunk, seed=1,
                                            label_precision=a.label_precision, models=models)
    t_label = time.perf_counter() - t0
    ntr = a.count - a.held
    T = torch.as_tensor(learn.targets(ks, ls), dtype=torch.float32, device="cuda")
    keep = torch.as_tensor(np.nonzero(met[:ntr])[0], device="cuda")
    report = {"population": dict(count=a.count, held_out=a.held, n=[a.nlo, a.nhi], tol=[a.tlo, a.thi],
                                 seed=a.seed, spectrum="a e^-i/tau + (1-a) i^-beta, a~U[0,1], "
                                                       "tau~logU[5,200], beta~U[1.5,4]",
                                 labels="%s adaptive loop, blocks of %d, l_max %d"
                                        % ("FP64" if a.label_precision == "fp64" else "mixed-path (BF16 x2)",
                                           16 if a.label_precision == "fp64" else 32, a.lmax),
                                 trained_on=int(met[:ntr].sum()), unmet_in_l_max=int((~met[:ntr]).sum()),
                                 held_out_met=int(met[ntr:].sum()),
                                 label_and_feature_seconds=t_label),
              "training": {}, "held_out": {}}
    os.makedirs(a.out, exist_ok=True)
    thetas = {}
    hidx = torch.as_tensor(ntr + np.nonzero(met[ntr:])[0], device="cuda")
    for prec in models:
        X = feats[prec].index_select(0, keep)
        th, hist = learn.train(X, T.index_select(0, keep), steps=a.steps, lr=2e-3, log_every=500)
        thetas[prec] = th
        th.cpu().numpy().astype("<f4").tofile(os.path.join(a.out, "rank_model_%s%s.bin" % (prec, a.tag)))
        # prediction quality on the held-out channels the adaptive loop finishes
        P = learn.predict(th, feats[prec].index_select(0, hidx)).cpu().numpy()
        Th = T.index_select(0, hidx).cpu().numpy()
        report["training"][prec] = {"steps": a.steps, "loss": hist,
                                    "held_out_median_abs_log_err": [float(np.median(np.abs(P[:, j] - Th[:, j])))
                                                                    for j in range(2)]}
    held = [ch for ch, m in zip(pop[ntr:], met[ntr:]) if m]
    if "fp64" in models:
        report["held_out"]["fp64"] = compare(held, thetas["fp64"], "fp64", a.lmax, a.chunk, 1, 0)
    if "bf16x" in models:
        mheld = [ch for ch in held if ch["tol"] >= a.mixed_floor]
        report["held_out"]["bf16x"] = compare(mheld, thetas["bf16x"], "bf16x", a.lmax, a.chunk, 1, 2)
    report["seconds"] = time.perf_counter() - t0
    with open(os.path.join(a.out, "rank_model%s.json" % a.tag), "w") as f:
        json.dump(report, f, indent=1)
    print(json.dumps(report["held_out"]))


if __name__ == "__main__":
    main()
