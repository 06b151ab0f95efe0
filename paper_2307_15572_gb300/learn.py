"""Rank model: labels from the adaptive loop, features from the probe sketch,
training with the library's own MLP kernels -- all on the GPU through the C ABI.

Population (seeded, ``synth.learn_population``): dense symmetric channels
whose spectra mix exponential and algebraic decay, with per-channel
tolerances.  Labels: the plain adaptive loop (randQB_EI, FP64 path) gives the
rank k* meeting the tolerance and the columns it drew, l*; targets are
(log k*, log max(l* - k*, 1)).  Features: ``rsvd_probe_features``.  The
network trains on standardised features and targets; the standardisation is
then folded into the first and last layers, so the stored parameter blob takes
the library's raw features (as RSVD_RANK_LEARNED feeds them).

torch is used only for device buffers and to draw the minibatch row numbers;
the standardisation, gathers, every forward, backward and Adam step and the
folding run in the library's kernels.
"""

import math
import time

import numpy as np

from . import rsvd, synth


def matrices(pop, device="cuda"):
    return [synth.population_matrix(ch, device=device) for ch in pop]


def _factors(pop, kcap):
    import torch
    facs, bufs = [], []
    for ch in pop:
        f, b = rsvd.Plan.factors_for(ch["n"], min(kcap, ch["n"]))
        f.tol = ch["tol"]
        facs.append(f)
        bufs.append(b)
    return facs, bufs


def label(pop, mats, block=16, lmax=1024, seed=1, chunk=64, precision="fp64"):
    """(k*, l*, met) per channel from the adaptive loop (FP64 path by default);
    met is False where the tolerance needs more than lmax columns."""
    ks, ls, met = [], [], []
    nmax = max(ch["n"] for ch in pop)
    plan = rsvd.Plan(nmax, k=0, p=0, q=0, tol=1e-3, policy="adaptive", precision=precision, block_b=block,
                     l_max=lmax, seed=seed)
    try:
        for i in range(0, len(pop), chunk):
            sub = pop[i:i + chunk]
            facs, bufs = _factors(sub, lmax)
            descs = [rsvd.dense(A) for A in mats[i:i + chunk]]
            st, per = rsvd.rsvd_decompose_batched(plan.h, descs, facs)
            for f, s in zip(facs, per):
                ks.append(f.k_out)
                ls.append(f.l_used)
                met.append(s >= 0)
    finally:
        plan.close()
    return np.array(ks), np.array(ls), np.array(met)


def features(pop, mats, precision="fp64", seed=1, chunk=64):
    import torch
    nmax = max(ch["n"] for ch in pop)
    plan = rsvd.Plan(nmax, k=16, p=0, q=0, tol=1e-3, precision=precision, seed=seed)
    out = []
    try:
        for i in range(0, len(pop), chunk):
            sub = pop[i:i + chunk]
            F = torch.empty((len(sub), rsvd.MLP_FEATURES), dtype=torch.float32, device="cuda")
            rsvd.rsvd_probe_features(plan.h, [rsvd.dense(A) for A in mats[i:i + chunk]],
                                     [ch["tol"] for ch in sub], F.data_ptr())
            out.append(F)
    finally:
        plan.close()
    return torch.cat(out)


def targets(ks, ls):
    k = np.maximum(ks, 1).astype(np.float64)
    p = np.maximum(ls - ks, 1).astype(np.float64)
    return np.stack([np.log(k), np.log(p)], axis=1)


def init_params(d, seed):
    """Uniform(+-1/sqrt(fan_in)) weights, zero biases (the oracle's scheme)."""
    rng = np.random.default_rng(seed)
    H = rsvd.MLP_HIDDEN
    parts = []
    for shape in [(d, H), (H,), (H, H), (H,), (H, 2), (2,)]:
        if len(shape) == 2:
            b = 1.0 / math.sqrt(shape[0])
            parts.append(rng.uniform(-b, b, size=shape).ravel())
        else:
            parts.append(np.zeros(shape))
    return np.concatenate(parts).astype(np.float32)


def train(X, T, steps=3000, batch=256, lr=2e-3, seed=0, log_every=0):
    """Train on device tensors X (N x d) and T (N x 2); returns (theta with the
    standardisation folded in, loss history).  The standardisation, the
    minibatch gathers, every forward/backward/Adam step and the final folding
    run in the library's kernels; torch provides the buffers and draws the
    minibatch row numbers."""
    import torch
    N, d = X.shape
    X = X.contiguous()
    T = T.contiguous()
    n = rsvd.rsvd_mlp_param_count(d)
    f32 = dict(dtype=torch.float32, device="cuda")
    mx, sx = torch.empty(d, **f32), torch.empty(d, **f32)
    mt, st = torch.empty(2, **f32), torch.empty(2, **f32)
    Xn, Tn = torch.empty((N, d), **f32), torch.empty((N, 2), **f32)
    rsvd.rsvd_mlp_standardize(X.data_ptr(), N, d, 1e-6, mx.data_ptr(), sx.data_ptr(), Xn.data_ptr())
    rsvd.rsvd_mlp_standardize(T.data_ptr(), N, 2, 1e-6, mt.data_ptr(), st.data_ptr(), Tn.data_ptr())
    theta = torch.as_tensor(init_params(d, seed), device="cuda")
    m = torch.zeros(n, **f32)
    v = torch.zeros(n, **f32)
    g = torch.zeros(n, **f32)
    B = min(batch, N)
    work = torch.empty(rsvd.rsvd_mlp_work_floats(d, B), **f32)
    loss = torch.zeros(1, **f32)
    xb, tb = torch.empty((B, d), **f32), torch.empty((B, 2), **f32)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    hist = []
    for t in range(1, steps + 1):
        idx = torch.randint(0, N, (B,), device="cuda", generator=gen)
        rsvd.rsvd_mlp_gather_rows(Xn.data_ptr(), idx.data_ptr(), B, d, xb.data_ptr())
        rsvd.rsvd_mlp_gather_rows(Tn.data_ptr(), idx.data_ptr(), B, 2, tb.data_ptr())
        rsvd.rsvd_mlp_loss_grad(theta.data_ptr(), d, xb.data_ptr(), tb.data_ptr(), B, g.data_ptr(),
                                loss.data_ptr(), work.data_ptr())
        rsvd.rsvd_mlp_adam(theta.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), n, t, lr)
        if log_every and t % log_every == 0:
            hist.append(float(loss.item()))
    out = torch.empty_like(theta)
    rsvd.rsvd_mlp_fold(theta.data_ptr(), d, mx.data_ptr(), sx.data_ptr(), mt.data_ptr(), st.data_ptr(),
                       out.data_ptr())
    return out, hist


def predict(theta, X):
    import torch
    Y = torch.empty((X.shape[0], 2), dtype=torch.float32, device="cuda")
    rsvd.rsvd_mlp_forward(theta.data_ptr(), X.shape[1], X.contiguous().data_ptr(), X.shape[0], Y.data_ptr())
    return Y


def run_policy(pop, mats, policy, precision, theta=None, block=16, lmax=1024, seed=1, slices=0, repeat=1,
               stats=None):
    """Decompose the channels with one policy; returns (seconds of the fastest
    of ``repeat`` calls after the first, which warms up, or of the one call;
    factors, per-channel status, exact relative errors of the last call).
    With ``stats`` (a dict) it also records the passes over V of that call
    (tensor-core passes on the mixed path, dense FP64 passes otherwise) and
    the plan's kernel launches."""
    import torch
    nmax = max(ch["n"] for ch in pop)
    plan = rsvd.Plan(nmax, k=0, p=0, q=0, tol=1e-3, policy=policy, precision=precision, block_b=block,
                     l_max=lmax, seed=seed, slices=slices,
                     mlp_weights=theta.data_ptr() if theta is not None else None)
    try:
        descs = [rsvd.dense(A) for A in mats]
        if stats is not None:
            rsvd.rsvd_plan_set_profiling(plan.h, True)
        times = []
        for _ in range(repeat):
            facs, bufs = _factors(pop, lmax)
            rsvd.rsvd_plan_profile(plan.h, reset=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, per = rsvd.rsvd_decompose_batched(plan.h, descs, facs)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        dt = min(times[1:]) if len(times) > 1 else times[0]
        if stats is not None:
            prof = rsvd.rsvd_plan_profile(plan.h)
            stats["passes"] = prof["tc_launches"] + prof["f64_launches"]
            stats["launches"] = prof["launches"]
        errs = [rsvd.rsvd_reconstruct_error(plan.h, dsc, f) if f.k_out > 0 else 1.0 for dsc, f in zip(descs, facs)]
    finally:
        plan.close()
    return dt, facs, per, np.array(errs)
