#!/usr/bin/env python
"""Throughput benchmark: matrix entries decomposed per second at relative
Frobenius error <= 1e-4, mixed-precision (tensor-core) path vs all-FP64 path.

Workload (one step = one grouped decomposition of the whole channel set):
forty dense symmetric channel matrices, sizes drawn uniformly from
[1000, 12000] (seeded), A_c = U_c diag(sigma) U_c^T with sigma_i = i^-2.5 and
symmetric noise of spectral size 1e-8 sigma_1, decomposed to tolerance 1e-4
(l = 128 columns, q = 0, rank chosen per channel).  Entries = sum n_c^2.
Inputs are resident in HBM before timing; they are larger than L2, so no
flush is needed between steps.

Prints one JSON line (rank 0).  Under torchrun every rank decomposes its own
forty-channel set (weak scaling, no data-path collective).

--impl reference times the CPU oracle (oracle/, FP64 numpy) on the machine's host
cores on the same workload and metric.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "matrix entries decomposed/s at rel-Frobenius err ≤1e-4, mixed vs FP64 path, 1 GB300"
UNIT = "entries/s"
L_COLS = 128          # columns drawn per channel (k cap 118 + p 10)
P_OVER = 10
TOL = 1e-4
# Peaks the driver's MEASURED_PEAKS.json does not carry, measured the same
# way on this machine's GB300 (torch.matmul 8192^3, CUDA events, best of 5-10):
FP64_PEAK_TFLOPS = 1.10       # FP64 (DGEMM); nominal 1.25
TF32_PEAK_TFLOPS = 1021.5     # TF32 tensor cores
FP32_SIMT_TFLOPS = 69.75      # FP32 on the CUDA cores


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--channels", type=int, default=40)
    ap.add_argument("--split", default="weak", choices=["weak", "fixed"],
                    help="weak: a channel set per GPU; fixed: one set split by LPT over the GPUs")
    ap.add_argument("--nmin", type=int, default=1000)
    ap.add_argument("--nmax", type=int, default=12000)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--rule-steps", type=int, default=2)
    ap.add_argument("--rule-n", type=int, default=200000)
    ap.add_argument("--no-rule", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="fixed default launch shapes")
    ap.add_argument("--no-graphs", action="store_true", help="direct launches instead of CUDA-graph replay")
    ap.add_argument("--prof-steps", type=int, default=5, help="profiled (per-kernel event) steps after timing")
    ap.add_argument("--no-rule-verify", action="store_true", help="skip the exact FP64 residual of the rule")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-rank leg")
    ap.add_argument("--learned-steps", type=int, default=10)
    ap.add_argument("--sweep", action="store_true", help="the full mixed sweep over tile-rule channels instead")
    ap.add_argument("--sweep-channels", type=int, default=400)
    ap.add_argument("--sweep-steps", type=int, default=2)
    ap.add_argument("--sweep-check", type=int, default=16, help="channels given the exact FP64 residual")
    ap.add_argument("--sweep-no-fp64", action="store_true")
    return ap.parse_args()


# --------------------------------------------------------------------- setup
def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if ws > 1:
        import torch
        import torch.distributed as dist_
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist_.init_process_group(backend=backend)
        dist = dist_
    return ws, rank, local, dist


def workload_sizes(args, rank, ws=1):
    """(sizes of this rank's channels, seed, their indices in the set).  Weak
    scaling: every rank its own seeded set.  Fixed set (--split fixed): one
    set, split over the ranks by LPT on n^2 l (2q + 2)."""
    from paper_2307_15572_gb300 import synth
    from paper_2307_15572_gb300 import shard
    if args.split == "fixed":
        seed = synth.SEED_BATCH
        sizes = synth.batch_sizes(args.channels, args.nmin, args.nmax, seed=seed)
        mine = shard.split_channels(sizes, L_COLS, 0, ws)[rank]
        return [sizes[c] for c in mine], seed, mine
    seed = shard.rank_seed(synth.SEED_BATCH, rank)
    sizes = synth.batch_sizes(args.channels, args.nmin, args.nmax, seed=seed)
    return sizes, seed, list(range(len(sizes)))


def make_inputs(sizes, seed, device, index=None):
    from paper_2307_15572_gb300 import synth
    index = index if index is not None else list(range(len(sizes)))
    return [synth.batch_channel(c, n, seed=seed, device=device) for c, n in zip(index, sizes)]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def bf16_peak(sustained=False):
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
    if os.path.exists(p):
        d = json.load(open(p))
        if key in d:
            return float(d[key]), "measured (%s)" % ("sustained" if sustained else "burst")
    return (1700.0 if sustained else 1900.0), "fallback"


def traffic_record(summary, source):
    """ncu DRAM bytes of a kernel per algorithmic byte, from a committed profile
    summary -- only if the kernel's source file is unchanged since the capture
    (the summary records its SHA-256 prefix)."""
    p = os.path.join(ROOT, "profiles", summary)
    src = os.path.join(ROOT, "paper_2307_15572_gb300", "csrc", source)
    if not os.path.exists(p) or not os.path.exists(src):
        return None
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    rec = {}
    for line in open(p):
        if line.startswith("traffic_per_algorithmic_byte:"):
            rec["ratio"] = float(line.split(":")[1])
        if line.startswith("source_sha256_16:"):
            rec["sha"] = line.split(":")[1].strip()
    if rec.get("sha") != h or "ratio" not in rec:
        return None
    return rec["ratio"]


def tc_traffic_record():
    return traffic_record("tc_gemm_batch40.md", "k_tc.cu")


def cvt_traffic_record():
    return traffic_record("convert_omega_batch8.md", "k_mixed.cu")


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                       "-lms", "100", "-i", str(dev)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.15)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().split("\n") if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- gpu arm
def run_gpu(args):
    import numpy as np
    import torch

    from paper_2307_15572_gb300 import rsvd

    ws, rank, local, dist = dist_setup(args)
    dev = local if torch.cuda.is_available() else 0
    torch.cuda.set_device(dev)
    sizes, seed, index = workload_sizes(args, rank, ws)
    entries = float(sum(n * n for n in sizes))
    mats = make_inputs(sizes, seed, "cuda", index)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    kcap = L_COLS - P_OVER
    lib = rsvd

    def make_plan(prec, graphs=False):
        # autotuning happens in the first warm-up step (outside the timed region)
        pl = rsvd.Plan(max(sizes), k=kcap, p=P_OVER, q=0, tol=TOL, policy="tol", precision=prec, slices=2,
                       seed=seed, stream=stream.cuda_stream, autotune=not args.no_autotune)
        if graphs:
            rsvd.rsvd_plan_set_graphs(pl.h, True)
        return pl

    def tune_summary(plan):
        recs = rsvd.rsvd_plan_tune_records(plan.h)
        keep = ("kind", "candidates", "choice", "bn", "split_target", "stages", "order")
        return {"on": not args.no_autotune, "signatures": len(recs),
                "non_default": sum(1 for r in recs if r["choice"] != 0),
                "tuning_ms": sum(r["tune_ms"] for r in recs),
                "choices": [dict({k: r[k] for k in keep}, ms_default=round(r["ms_default"], 4),
                                 ms_best=round(r["ms_best"], 4)) for r in recs]}

    def alloc_factors(device="cuda", pin=False, cap=None):
        facs, bufs = [], []
        for n in sizes:
            kk = min(cap or kcap, n)
            if device == "cuda":
                f, b = rsvd.Plan.factors_for(n, kk)
            else:
                U = torch.empty((kk, n), dtype=torch.float64, pin_memory=pin)
                V = torch.empty((kk, n), dtype=torch.float64, pin_memory=pin)
                S = torch.empty((kk,), dtype=torch.float64, pin_memory=pin)
                f = rsvd.Factors()
                f.mem = rsvd.MEM_HOST
                f.U, f.ldu, f.V, f.ldv, f.S, f.k_cap = U.data_ptr(), n, V.data_ptr(), n, S.data_ptr(), kk
                b = (U, S, V)
            facs.append(f)
            bufs.append(b)
        return facs, bufs

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2307_15572_gb300 import shard

    def reduce_runs(ent, ms_):
        """(entries of all ranks, slowest rank's time): timing only, no data."""
        return shard.reduce_timing(dist, ent, ms_, device="cuda")

    descs = [rsvd.dense(A) for A in mats]

    def timed_steps(plan, facs, K, W, descs_, clocks=False):
        for _ in range(W):
            st, _ = rsvd.rsvd_decompose_batched(plan.h, descs_, facs)
            if st < 0:
                raise RuntimeError("decompose failed: %s" % rsvd.last_error())
        rsvd.rsvd_plan_profile(plan.h, reset=True)
        barrier()
        ck = Clocks(dev) if clocks else None
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(K):
            st, _ = rsvd.rsvd_decompose_batched(plan.h, descs_, facs)
            if st < 0:
                raise RuntimeError("decompose failed: %s" % rsvd.last_error())
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        clk = ck.stop() if ck else None
        barrier()
        ms = e0.elapsed_time(e1)
        prof = rsvd.rsvd_plan_profile(plan.h, reset=True)
        return ms, wall, prof, clk

    def verify(plan, facs):
        errs, ks = [], []
        for A, f in zip(mats, facs):
            errs.append(rsvd.rsvd_reconstruct_error(plan.h, rsvd.dense(A), f))
            ks.append(f.k_out)
        return max(errs), ks

    # ---- mixed path (headline): the whole grouped decomposition replayed from
    # a CUDA graph (captured in the warm-up), no per-kernel events
    plan = make_plan("bf16x", graphs=not args.no_graphs)
    facs, bufs = alloc_factors()
    ms, wall, prof_h, clk = timed_steps(plan, facs, args.steps, args.warmup, descs, clocks=(rank == 0))
    max_err, ks = verify(plan, facs)
    # per-channel records to rank 0 (host metadata only)
    records = shard.gather_records(dist, [{"index": c, "gpu": rank, "k": int(f.k_out), "status": int(f.status)}
                                          for c, f in zip(index, facs)])
    errs_all = shard.gather_records(dist, [{"index": rank, "e": max_err}])
    if errs_all:
        max_err = max(r["e"] for r in errs_all)
    tot, ms_max = reduce_runs(entries * args.steps, ms)
    value = tot / (ms_max / 1e3)
    gpu_launches = int(prof_h["launches"])
    tuning = tune_summary(plan)
    # the same steps again with CUDA events around the passes over V (direct
    # launches: events inside a replayed graph are not per launch), for the
    # per-kernel rooflines
    rsvd.rsvd_plan_set_graphs(plan.h, False)
    rsvd.rsvd_plan_set_profiling(plan.h, True)
    ms_p, _, prof, _ = timed_steps(plan, facs, args.prof_steps, 1, descs)
    plan.close()
    hbm_peak, peak_kind = peaks()
    ratio = tc_traffic_record()
    cvt_ratio = cvt_traffic_record()
    kern = []
    if prof["cvt_launches"]:
        c_ms = prof["cvt_ms"] / prof["cvt_launches"]
        c_bytes = prof["cvt_bytes"] / prof["cvt_launches"]
        c_ach = c_bytes / (c_ms / 1e3) / 1e9
        kern.append({"bound": "hbm", "achieved": c_ach, "peak": hbm_peak, "unit": "GB/s", "frac": c_ach / hbm_peak,
                     "traffic": (cvt_ratio * c_bytes) if cvt_ratio else None,
                     "kernel": "k_convert_omega (FP64 V -> BF16 words, ||V||^2, P)",
                     "peak_source": peak_kind, "launches": prof["cvt_launches"], "avg_launch_ms": c_ms,
                     "algorithmic_bytes_per_launch": c_bytes,
                     "bytes_per_unit": "8 B read + 2 B per word written per V entry, + P words",
                     "share_of_step": prof["cvt_ms"] / ms_p})
    if prof["tc_launches"]:
        tc_ms_per = prof["tc_ms"] / prof["tc_launches"]
        tc_bytes_per = prof["tc_bytes"] / prof["tc_launches"]
        achieved = tc_bytes_per / (tc_ms_per / 1e3) / 1e9
        kern.append({"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": (ratio * tc_bytes_per) if ratio else None,
                     "kernel": "k_tc_gemm (tcgen05 pass over V words)", "peak_source": peak_kind,
                     "launches": prof["tc_launches"], "avg_launch_ms": tc_ms_per,
                     "algorithmic_bytes_per_launch": tc_bytes_per,
                     "bytes_per_unit": "2 B per word per V entry, + X words and Y once",
                     "share_of_step": prof["tc_ms"] / ms_p})
    if prof.get("gram_launches"):
        # the FP64-grade Grams of CholeskyQR: algorithmic flops (2 n l^2 per
        # Gram) against the measured FP64 peak they replace, issued slice
        # products against the sustained BF16 peak
        g_ms = prof["gram_ms"] / prof["gram_launches"]
        g_tf = prof["gram_flops"] / prof["gram_launches"] / (g_ms / 1e3) / 1e12
        g_mma = prof["gram_mma_flops"] / prof["gram_launches"] / (g_ms / 1e3) / 1e12
        bf16_s, bf16_kind = bf16_peak(sustained=True)
        kern.append({"bound": "tensor", "achieved": g_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": g_tf / FP64_PEAK_TFLOPS, "traffic": None,
                     "kernel": "k_gram_tc + k_gram_tc_reduce (FP64-grade Gram of the n x l FP32 panels, exact "
                               "BF16 slices on tcgen05)",
                     "peak_source": "FP64 DGEMM, builder-measured (the precision the Gram delivers)",
                     "launches": prof["gram_launches"], "avg_launch_ms": g_ms,
                     "algorithmic_flops_per_launch": prof["gram_flops"] / prof["gram_launches"],
                     "issued_tflops": g_mma, "issued_frac_of_bf16": g_mma / bf16_s, "bf16_peak_source": bf16_kind,
                     "share_of_step": prof["gram_ms"] / ms_p})
    kern.sort(key=lambda r: -r["share_of_step"])
    roofline = dict(kern[0]) if kern else None
    if roofline is not None:
        roofline["note"] = ("dominant kernel of the step by share (CUDA events over %d profiled steps of the "
                            "same workload, direct launches); 'others' lists the other timed kernels"
                            % args.prof_steps)
        roofline["others"] = kern[1:]
        roofline["profiled_ms_per_step"] = ms_p / args.prof_steps

    # ---- learned rank on the same channels: the committed rank model (trained
    # by paper_2307_15572_gb300/rank_model.py on a seeded population of this
    # workload's size range, labelled by the mixed-path adaptive loop) picks
    # each channel's l from a one-word probe; the rank rule checks every
    # channel, misses retry and then fall back to the adaptive loop
    learned = None
    wpath = os.path.join(ROOT, "paper_2307_15572_gb300", "rank_model_bf16x_batch.bin")
    if not args.no_learned and os.path.exists(wpath):
        theta = torch.from_numpy(np.fromfile(wpath, dtype="<f4")).cuda()
        plan = rsvd.Plan(max(sizes), k=0, p=0, q=0, tol=TOL, policy="learned", precision="bf16x", slices=2,
                         l_max=1024, seed=seed, stream=stream.cuda_stream, mlp_weights=theta.data_ptr())
        if not args.no_graphs:
            rsvd.rsvd_plan_set_graphs(plan.h, True)
        lf, lb = alloc_factors(cap=256)
        ms_l, _, prof_l, _ = timed_steps(plan, lf, args.learned_steps, args.warmup, descs)
        err_l, ks_l = verify(plan, lf)
        ls_l = [f.l_used for f in lf]
        st_l = [int(f.status) for f in lf]
        rsvd.rsvd_plan_set_graphs(plan.h, False)
        rsvd.rsvd_plan_set_profiling(plan.h, True)
        _, _, prof_lp, _ = timed_steps(plan, lf, 1, 0, descs)
        plan.close()
        tot_l, ms_l = reduce_runs(entries * args.learned_steps, ms_l)
        learned = {"value": tot_l / (ms_l / 1e3), "unit": UNIT, "ms_per_step": ms_l / args.learned_steps,
                   "steps": args.learned_steps, "policy": "learned", "max_rel_err": err_l,
                   "verified_tol": bool(err_l <= TOL), "ranks": [min(ks_l), max(ks_l)],
                   "l_used": [min(ls_l), max(ls_l)], "mean_l": float(np.mean(ls_l)),
                   "statuses": sorted(set(st_l)),
                   "passes_over_v_per_step": int(prof_lp["tc_launches"]),
                   "vs_tol_policy": (tot_l / (ms_l / 1e3)) / value,
                   "model": "rank_model_bf16x_batch.bin (see rank_model_batch.json for its population, "
                            "labels and held-out report)"}
        del lb

    # ---- e2e through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        hmats = []
        for A in mats:
            h = torch.empty(A.shape, dtype=torch.float64, pin_memory=True)
            h.copy_(A)
            hmats.append(h)
        hdescs = [rsvd.dense(h) for h in hmats]
        plan = make_plan("bf16x", graphs=not args.no_graphs)
        hf, hb = alloc_factors("cpu", pin=True)
        ms_e, wall_e, prof_e, _ = timed_steps(plan, hf, args.e2e_steps, 1, hdescs)
        h2d = sum(8 * n * n for n in sizes)
        d2h = sum(8 * (2 * f.k_out * n + f.k_out) for f, n in zip(hf, sizes))
        tot_e, ms_e = reduce_runs(entries * args.e2e_steps, ms_e)
        e2e = {"value": tot_e / (ms_e / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
               "ms_per_step": ms_e / args.e2e_steps}
        plan.close()
        del hmats, hdescs, hb

    # ---- all-FP64 path on the same workload
    fp64 = None
    if not args.no_fp64:
        plan = make_plan("fp64")
        rsvd.rsvd_plan_set_profiling(plan.h, True)
        ff, fb = alloc_factors()
        ms_f, wall_f, prof_f, _ = timed_steps(plan, ff, args.fp64_steps, 1, descs)
        err_f, ks_f = verify(plan, ff)
        tot_f, ms_f = reduce_runs(entries * args.fp64_steps, ms_f)
        f64_ms = prof_f["f64_ms"] / max(1, prof_f["f64_launches"])
        f64_tf = prof_f["f64_flops"] / max(1, prof_f["f64_launches"]) / (f64_ms / 1e3) / 1e12 if f64_ms else 0
        fp64 = {"value": tot_f / (ms_f / 1e3), "unit": UNIT,
                "ms_per_step": ms_f / args.fp64_steps, "steps": args.fp64_steps, "max_rel_err": err_f,
                "ranks": [min(ks_f), max(ks_f)],
                "roofline": {"bound": "alu", "kernel": "k_tile_mm<double> (FP64 pass over V)",
                             "achieved": f64_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": f64_tf / FP64_PEAK_TFLOPS,
                             "peak_source": "builder-measured: torch.matmul FP64 8192^3, best of 5, this pool's "
                                            "GB300 (nominal 1.25)"},
                "autotune": tune_summary(plan)}
        plan.close()

    # ---- matrix-free tile rule: n = 200,000, M = 300 bumps, k = 320, p = 10, q = 1
    rule = None
    if not args.no_rule:
        from paper_2307_15572_gb300 import synth
        rn, rM, rk, rp, rq = args.rule_n, 300, 320, 10, 1
        c_, s_, w_ = synth.rule_params(M=rM, seed=synth.SEED_RULE)
        rm = rsvd.rule(rn, c_, s_, w_, eta=1e-7, seed=synth.SEED_RULE)
        plan = rsvd.Plan(rn, k=rk, p=rp, q=rq, seed=seed, precision="bf16x", slices=2, policy="fixed",
                         stream=stream.cuda_stream)
        rsvd.rsvd_plan_set_profiling(plan.h, True)
        rf, rb = rsvd.Plan.factors_for(rn, rk)
        rfl = [rf]
        ms_r, wall_r, prof_r, _ = timed_steps(plan, rfl, args.rule_steps, 1, [rm])
        rf = rfl[0]                       # the call returns its results in the list
        tot_r, ms_r = reduce_runs(float(rn) * rn * args.rule_steps, ms_r)
        g_ms = prof_r["gen_ms"] / max(1, prof_r["gen_launches"])
        g_alg = prof_r["gen_flops"] / max(1, prof_r["gen_launches"])
        g_mma = prof_r["gen_mma_flops"] / max(1, prof_r["gen_launches"])
        t_ms = prof_r["tc_ms"] / max(1, prof_r["tc_launches"])
        t_bytes = prof_r["tc_bytes"] / max(1, prof_r["tc_launches"])
        t_flops = prof_r["tc_flops"] / max(1, prof_r["tc_launches"])
        hbm_peak, peak_kind = peaks()
        bps, bps_src = bf16_peak(sustained=True)
        g_ach = g_alg / (g_ms / 1e3) / 1e12 if g_ms else 0.0
        rule_exact = None
        if not args.no_rule_verify:
            # every entry regenerated in FP64 on the device (outside the timed region)
            t0v = time.perf_counter()
            rule_exact = {"rel_err": rsvd.rsvd_reconstruct_error(plan.h, rm, rf),
                          "seconds": time.perf_counter() - t0v,
                          "how": "rsvd_reconstruct_error on the tile rule: all n^2 entries regenerated in FP64 "
                                 "(FP64 factor panel products + hash noise) against U diag(S) V^T"}
        rule = {"value": tot_r / (ms_r / 1e3), "unit": UNIT,
                "ms_per_step": ms_r / args.rule_steps, "steps": args.rule_steps,
                "workload": "rule: Gaussian-bump tile rule, n = %d, M = 300, w_m = e^-m/25, hash noise 1e-7; "
                            "k = 320, p = 10, q = 1, 2 words; every pass generates its entries" % rn,
                "err_est": rf.err_est, "status": int(rf.status), "k": rf.k_out,
                "exact_residual": rule_exact,
                "verified": (rule_exact["rel_err"] <= rf.err_est) if rule_exact else None,
                "passes_per_step": 2 * rq + 2,
                "roofline": {"bound": "tensor",
                             "kernel": "k_tc_gemm<2, 2, true> (tile-rule generation, FP16 factor words, "
                                       "two epilogue groups)",
                             "achieved": g_ach, "peak": bps, "unit": "TFLOP/s", "frac": g_ach / bps,
                             "peak_source": bps_src + " (the generator runs inside a seconds-long step)",
                             "flops_per_unit": "2 M = 600 flops per generated entry (algorithmic)",
                             "launches": prof_r["gen_launches"], "avg_launch_ms": g_ms,
                             "share_of_step": prof_r["gen_ms"] / ms_r if ms_r else None,
                             "issued_tflops": g_mma / (g_ms / 1e3) / 1e12 if g_ms else 0.0,
                             "note": "issued_tflops counts the FP16 word products the kernel issues (3 per "
                                     "entry term, M padded to 320), 3.2x the algorithmic work; frac is on "
                                     "algorithmic flops"},
                "product_roofline": {"bound": "hbm", "kernel": "k_tc_gemm<2, 2> (panel words x X words)",
                                     "achieved": t_bytes / (t_ms / 1e3) / 1e9 if t_ms else 0.0,
                                     "peak": hbm_peak, "unit": "GB/s",
                                     "frac": (t_bytes / (t_ms / 1e3) / 1e9) / hbm_peak if t_ms else 0.0,
                                     "tflops_issued": t_flops / (t_ms / 1e3) / 1e12 if t_ms else 0.0,
                                     "launches": prof_r["tc_launches"], "avg_launch_ms": t_ms,
                                     "algorithmic_bytes_per_launch": t_bytes,
                                     "share_of_step": prof_r["tc_ms"] / ms_r if ms_r else None}}
        plan.close()
        del rb

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_oracle(mats, sizes, seed, args.cpu_seconds)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "strong" if args.split == "fixed" else "weak", "vs_baseline": None, "dtype": "bf16",
               "data": "synthetic",
               "config": {"workload": "batch40: %d dense symmetric channels, n ~ U[%d, %d], "
                                      "sigma_i = i^-2.5 + noise 1e-8 sigma_1, tol 1e-4"
                                      % (args.channels, args.nmin, args.nmax),
                          "channels": args.channels, "sum_n2_per_gpu": entries, "tol": TOL, "l": L_COLS,
                          "q": 0, "words": 2, "policy": "tol",
                          "precision": "V and X as 2 BF16 words, FP32 accumulate; FP64-grade Grams (exact BF16 "
                                       "slices on the tensor cores), double-float (FP64-grade) Cholesky",
                          "l2": "inputs larger than L2 (no flush)", "max_rel_err": max_err,
                          "verified_tol": bool(max_err <= TOL), "ranks": [min(ks), max(ks)],
                          "parallelism": ("fixed set split by LPT over %d GPUs" % ws if args.split == "fixed"
                                          else "a channel set per GPU") if ws > 1 else "single GPU",
                          "channel_records": (None if records is None else
                                              {"channels": len(records),
                                               "gpus": sorted({r["gpu"] for r in records}),
                                               "statuses": sorted({r["status"] for r in records})}),
                          "autotune": tuning},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
               "clocks": clk, "fp64_path": fp64, "rule_path": rule, "learned_path": learned,
               "mixed_over_fp64": (value / fp64["value"]) if fp64 else None}
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def cpu_model():
    """CPU model of the host running the oracle (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


# ------------------------------------------------------------ oracle timing
def cpu_oracle(mats, sizes, seed, budget_s):
    """The oracle as it stands, on the host cores, over channels until the budget."""
    import numpy as np

    from oracle import rsvd as orsvd
    done_entries, t_total, used = 0.0, 0.0, 0
    host = []
    for A in mats:
        host.append(A.cpu().numpy() if hasattr(A, "cpu") else A)
    for c, A in enumerate(host):
        t0 = time.perf_counter()
        r = orsvd.rsvd(A, tol=TOL, l=L_COLS, q=0, seed=seed)
        t_total += time.perf_counter() - t0
        done_entries += float(A.shape[0]) ** 2
        used += 1
        if t_total > budget_s:
            break
    cores = int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1))
    return {"value": done_entries / t_total, "unit": UNIT, "cores": cores, "cpu_model": cpu_model(), "kind": "oracle",
            "sample": "%d of %d channels (sum n^2 = %.3g), tol 1e-4, l = %d, q = 0, numpy FP64"
                      % (used, len(host), done_entries, L_COLS),
            "seconds": t_total}


# ------------------------------------------------------------ config-5 sweep
def run_sweep(args):
    """Full mixed sweep: 400 tile-rule channels of uneven size (p(n) ~ n^-2.41
    on [2000, 40000], ~150 GB of FP64 entries, never stored), each with its
    own seeded bumps and decay, decomposed to tol 1e-4 in one grouped call per
    configuration -- BF16 words (2 or 3) with q = 0..3, the learned rank, and
    the FP64 path at q = 0 -- replayed from CUDA graphs; one JSON line."""
    import numpy as np
    import torch

    from paper_2307_15572_gb300 import rsvd, synth
    torch.cuda.set_device(0)
    params = synth.sweep_channel_params(args.sweep_channels)
    mats = [rsvd.rule(p["n"], p["c"], p["s"], p["w"], eta=p["eta"], seed=p["seed"]) for p in params]
    sizes = [p["n"] for p in params]
    entries = float(sum(float(n) * n for n in sizes))
    stream = torch.cuda.current_stream()
    wpath = os.path.join(ROOT, "paper_2307_15572_gb300", "rank_model_bf16x.bin")
    theta = torch.from_numpy(np.fromfile(wpath, dtype="<f4")).cuda() if os.path.exists(wpath) else None
    confs = [("bf16x", 2, q, "tol") for q in (0, 1, 2, 3)] + [("bf16x", 3, 1, "tol")]
    if theta is not None:
        confs.append(("bf16x", 2, 1, "learned"))
    if not args.sweep_no_fp64:
        confs.append(("fp64", 0, 0, "tol"))
    results, keep = [], None
    for prec, words, q, policy in confs:
        plan = rsvd.Plan(max(sizes), k=246, p=10, q=q, tol=TOL, policy=policy, precision=prec, slices=words,
                         seed=synth.SEED_SWEEP, stream=stream.cuda_stream, l_max=1024,
                         mlp_weights=theta.data_ptr() if policy == "learned" else None)
        rsvd.rsvd_plan_set_graphs(plan.h, True)
        facs = []
        bufs = []
        for n in sizes:
            f, b = rsvd.Plan.factors_for(n, min(256, n))
            facs.append(f)
            bufs.append(b)
        steps = 1 if prec == "fp64" else args.sweep_steps
        for _ in range(1):                                    # warm-up: captures the graph
            st, per = rsvd.rsvd_decompose_batched(plan.h, mats, facs)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            st, per = rsvd.rsvd_decompose_batched(plan.h, mats, facs)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        ks = [f.k_out for f in facs]
        ests = [f.err_est for f in facs]
        results.append({"precision": prec if prec == "fp64" else "bf16 x%d words" % words, "q": q, "policy": policy,
                        "ms": ms, "entries_per_s": entries / (ms / 1e3), "ranks": [min(ks), max(ks)],
                        "mean_rank": float(np.mean(ks)), "max_err_est": float(max(ests)),
                        "statuses": {str(v): int(sum(1 for x in per if x == v)) for v in sorted(set(per))}})
        if prec == "bf16x" and words == 2 and q == 1 and policy == "tol":
            # exact check on a seeded sample of channels: every entry
            # regenerated in FP64 (outside the timed region)
            rng = np.random.default_rng(7)
            pick = sorted(rng.choice(len(sizes), size=min(args.sweep_check, len(sizes)), replace=False))
            errs = [rsvd.rsvd_reconstruct_error(plan.h, mats[i], facs[i]) for i in pick]
            keep = {"configuration": "bf16 x2 words, q = 1, tol", "channels": [int(i) for i in pick],
                    "n": [sizes[i] for i in pick], "exact_rel_err": errs,
                    "err_est": [facs[i].err_est for i in pick],
                    "all_within_tol": bool(all(e <= TOL for e in errs))}
        plan.close()
        del bufs
        print(json.dumps(results[-1]), file=sys.stderr, flush=True)
    out = {"sweep": "config5: full mixed sweep over tile-rule channels", "channels": len(sizes),
           "n_range": [min(sizes), max(sizes)], "sum_n2": entries, "fp64_equivalent_gb": entries * 8 / 1e9,
           "tol": TOL, "data": "synthetic (seeded tile rules; every pass generates its entries)",
           "results": results, "exact_check": keep,
           "not_built": {"tf32": "the word-format emulation (tests/test_sketch_precision.py) meets 1e-4 only "
                                 "with an extra power iteration, i.e. the bytes of two BF16 words at half "
                                 "their tensor rate",
                         "fp8_per_tile": "the same emulation misses 1e-4 by 26x (q = 0) and 8x (q = 1)"}}
    print(json.dumps(out), flush=True)


def run_reference(args):
    ws, rank, local, dist = dist_setup(args)
    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    import numpy as np

    from oracle import rsvd as orsvd
    sizes, seed, _ = workload_sizes(args, 0)
    try:
        import torch
        dev = "cuda" if torch.cuda.is_available() else None
    except Exception:
        dev = None
    # each step: a bounded sample of channels (rotating through the set)
    order = list(range(len(sizes)))
    per_step_budget = 150.0 / max(1, args.steps + args.warmup)
    cache = {}

    def get(c):
        if c not in cache:
            from paper_2307_15572_gb300 import synth
            A = synth.batch_channel(c, sizes[c], seed=seed, device=dev)
            cache[c] = A.cpu().numpy() if dev else A
        return cache[c]

    pos = 0
    times, ents = [], []
    total_steps = args.warmup + args.steps
    for s in range(total_steps):
        t_step, e_step = 0.0, 0.0
        while t_step < per_step_budget or e_step == 0:
            c = order[pos % len(order)]
            pos += 1
            A = get(c)
            t0 = time.perf_counter()
            orsvd.rsvd(A, tol=TOL, l=L_COLS, q=0, seed=seed)
            t_step += time.perf_counter() - t0
            e_step += float(sizes[c]) ** 2
            if len(cache) > 8:
                cache.pop(next(iter(cache)))
        if s >= args.warmup:
            times.append(t_step)
            ents.append(e_step)
    value = sum(ents) / sum(times)
    cores = int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1))
    sample = "per step: channels of the 40-channel set in rotation for ~%.1f s of oracle time" % per_step_budget
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "batch40 (see gb300 arm)", "tol": TOL, "l": L_COLS, "q": 0},
           "impl": "reference",
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "cpu_model": cpu_model(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.sweep:
        run_sweep(a)
    else:
        run_gpu(a)
