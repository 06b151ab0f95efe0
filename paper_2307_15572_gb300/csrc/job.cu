// Jobs: per-channel dimensions, the workspace layout pass, execution (with
// CUDA-graph capture and replay), result collection, and the fixed-l,
// probe and learned-rank drivers.
#include "api_internal.h"

namespace rsvd_api {

// ------------------------------------------------------------ job plumbing
void init_job(Job& J, rsvd_plan_s* P, int C, const rsvd_matrix* A, rsvd_factors* f) {
  J.P = P;
  J.C = C;
  J.A = A;
  J.f = f;
  J.mixed = P->o.precision == RSVD_PREC_BF16X;
  J.q = P->o.q;
  J.nsl = P->slices;
  J.policy = P->o.rank_policy == RSVD_RANK_LEARNED ? RSVD_RANK_TOL : P->o.rank_policy;
  J.tol = P->o.tol;
  J.rule = C > 0 && A[0].kind == RSVD_TILE_RULE;
  J.host_in_place = !J.mixed && !J.rule && fp64_reads_host_in_place(A, C);
}

// Per-channel dims: l from lvec (else k + p, capped at n), s probe columns.
void make_dims(Job& J, const std::vector<int>* lvec, std::vector<int>& warn, int probe_cols) {
  const int C = J.C;
  J.d.assign(C, ChanDims{});
  warn.assign(C, 0);
  J.max_l = J.max_lw = J.max_kcap = 0;
  int64_t sum_gram_tiles = 0;
  for (int c = 0; c < C; ++c) {
    ChanDims& d = J.d[c];
    d.n = (int)J.A[c].n;
    int64_t l = lvec ? (*lvec)[c] : (int64_t)J.P->o.k + J.P->o.p;
    if (l > d.n) { l = d.n; warn[c] = RSVD_WARN_RANK_CAPPED; }
    d.l = (int)std::max<int64_t>(1, l);
    d.s = probe_cols;
    d.lw = d.l + d.s;
    d.kcap = std::min(J.f[c].k_cap, d.l);
    d.ldt = rup(d.n, 4);
    d.ldb = rup(d.n, 64);
    d.tol = J.f[c].tol > 0.0 ? J.f[c].tol : J.P->o.tol;
    sum_gram_tiles += (int64_t)cdiv(d.l, 64) * cdiv(d.l, 64);
    J.max_l = std::max(J.max_l, d.l);
    J.max_lw = std::max(J.max_lw, d.lw);
    J.max_kcap = std::max(J.max_kcap, d.kcap);
  }
  for (int c = 0; c < C; ++c) {
    // rows per Gram split: ~512, more when the batch is too small to fill the GPU
    ChanDims& d = J.d[c];
    int g = cdiv(d.n, 512);
    const int want = (int)((2 * NSM + sum_gram_tiles - 1) / std::max<int64_t>(1, sum_gram_tiles));
    g = std::max(g, std::min(want, cdiv(d.n, 64)));
    d.gsplit = std::max(1, std::min(g, 64));
  }
}

// One layout pass + step building; base == nullptr only measures.  Returns
// the bytes the job needs.
rsvd_status build_job(Job& J, char* base, JobKind kind, bool skip_convert, size_t* need, ProbeOut* po) {
  Bump b(base);
  J.skip_convert = skip_convert;
  J.probe_job = kind == JOB_PROBE;
  J.measure = base == nullptr;
  layout(J, b);
  float* d_feat = nullptr;
  float* d_pred = nullptr;
  if (kind == JOB_PROBE) {
    d_feat = b.take<float>((size_t)J.C * 19);
    d_pred = b.take<float>((size_t)J.C * 2);
    if (po) { po->feat = d_feat; po->pred = d_pred; }
  }
  const size_t buf_bytes = (b.off + 4095) & ~(size_t)4095;
  J.ar = Arena();
  J.ar.dbase = base ? base + buf_bytes : nullptr;
  J.steps.clear();
  {
    std::vector<Chan> tmp(J.ch);
    J.d_ch = J.ar.put(tmp.data(), tmp.size(), 128);
  }
  if (kind == JOB_PROBE) {
    if (rsvd_status s = build_probe(J, d_feat, J.P->o.mlp_weights, J.P->o.mlp_weights ? d_pred : nullptr)) return s;
  } else if (J.mixed) {
    if (rsvd_status s = build_mixed(J, skip_convert)) return s;
  } else {
    build_fp64(J);
  }
  *need = buf_bytes + J.ar.h.size() + 4096;
  return RSVD_OK;
}

// Upload descriptors, stage host inputs (unless reused), run, read results.
// Everything that shapes a job's launch sequence: sizes, options, buffers.
std::string graph_key(const Job& J, bool stage_inputs) {
  const rsvd_plan_s* P = J.P;
  std::string k;
  auto put = [&](const void* p, size_t n) { k.append((const char*)p, n); };
  auto put64 = [&](int64_t v) { put(&v, sizeof(v)); };
  put64(J.C); put64((int64_t)(uintptr_t)P->ws); put64((int64_t)(uintptr_t)P->hp); put64((int64_t)J.ar.h.size());
  put64(J.mixed); put64(J.skip_convert); put64(J.probe_job); put64(stage_inputs); put64(J.q); put64(J.nsl);
  put64(J.host_in_place);
  put64(J.policy); put(&J.tol, sizeof(J.tol)); put64(P->o.rayleigh_ritz); put64((int64_t)(uintptr_t)P->o.mlp_weights);
  for (int c = 0; c < J.C; ++c) {
    const ChanDims& d = J.d[c];
    const int64_t v[] = {d.n, d.l, d.lw, d.s, d.kcap, d.gsplit, d.ldt, d.ldb};
    put(v, sizeof(v));
    if (stage_inputs && J.staged[c]) { put64((int64_t)(uintptr_t)J.A[c].data); put64(J.A[c].ld); }
    if (J.rule) {
      // what tile-rule launches take by value: the layout (M, panel rows),
      // the noise key and amplitude, the factor words' scale
      const rsvd_matrix& a = J.A[c];
      const double hs = rule_hscale(a.rule_w, a.rule_m);
      put64(a.rule_m); put64((int64_t)a.rule_seed); put(&a.rule_eta, sizeof(double)); put(&hs, sizeof(double));
    }
  }
  if (J.rule) put64(J.panel);
  return k;
}

// Upload descriptors, stage host inputs (unless reused), run, read results.
// With graphs on (and a capturable stream), the whole sequence is captured
// once per key and replayed; the first node re-uploads the descriptors, so a
// replay sees this call's pointers.
rsvd_status execute(Job& J, bool stage_inputs, std::vector<ChanResult>& res) {
  rsvd_plan_s* P = J.P;
  const int C = J.C;
  if (rsvd_status s = grow_pinned(P, std::max(J.ar.h.size(), sizeof(ChanResult) * C) + 64)) return s;
  memcpy(P->hp, J.ar.h.data(), J.ar.h.size());
  ChanResult* hres = (ChanResult*)P->hp;
  int* herr = (int*)(P->hp + ((sizeof(ChanResult) * C + 63) & ~(size_t)63));
  auto enqueue = [&]() -> rsvd_status {
    CK(cudaMemsetAsync(J.d_res, 0, sizeof(ChanResult) * C, P->st));
    CK(cudaMemcpyAsync(J.ar.dbase, P->hp, J.ar.h.size(), cudaMemcpyHostToDevice, P->st));
    if (stage_inputs)
      for (int c = 0; c < C; ++c)
        if (J.staged[c]) {
          const size_t row = (size_t)J.d[c].n * sizeof(double);
          if (J.A[c].ld == J.d[c].n)
            CK(cudaMemcpyAsync((void*)J.ch[c].A, J.A[c].data, row * J.d[c].n, cudaMemcpyHostToDevice, P->st));
          else
            CK(cudaMemcpy2DAsync((void*)J.ch[c].A, row, J.A[c].data, (size_t)J.A[c].ld * sizeof(double), row,
                                 J.d[c].n, cudaMemcpyHostToDevice, P->st));
        }
    CK(cudaMemsetAsync(P->d_err, 0, sizeof(int), P->st));
    for (auto& step : J.steps)
      if (rsvd_status s = step()) return s;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(hres, J.d_res, sizeof(ChanResult) * C, cudaMemcpyDeviceToHost, P->st));
    CK(cudaMemcpyAsync(herr, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, P->st));
    return RSVD_OK;
  };
  const bool use_graph = P->graphs && !P->profiling && !J.tuning && P->st != nullptr;
  if (!use_graph) {
    if (rsvd_status s = enqueue()) return s;
  } else {
    const std::string key = graph_key(J, stage_inputs);
    rsvd_plan_s::GraphEntry* ge = nullptr;
    for (auto& g : P->gcache)
      if (g.key == key) ge = &g;
    if (ge) {
      ge->used = ++P->gclock;
      CK(cudaGraphLaunch(ge->exec, P->st));
      note_launch((int)ge->launches);
    } else {
      const long long l0 = launch_count();
      CK(cudaStreamBeginCapture(P->st, cudaStreamCaptureModeRelaxed));
      const rsvd_status s = enqueue();
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(P->st, &g);
      if (s) { if (g) cudaGraphDestroy(g); return s; }
      if (e != cudaSuccess) return seterr(RSVD_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
      cudaGraphExec_t x = nullptr;
      const cudaError_t ei = cudaGraphInstantiate(&x, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) return seterr(RSVD_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
      if (P->gcache.size() >= 8) {                       // evict the least recently used
        size_t lru = 0;
        for (size_t i = 1; i < P->gcache.size(); ++i)
          if (P->gcache[i].used < P->gcache[lru].used) lru = i;
        cudaGraphExecDestroy(P->gcache[lru].exec);
        P->gcache.erase(P->gcache.begin() + lru);
      }
      P->gcache.push_back({key, x, launch_count() - l0, ++P->gclock});
      CK(cudaGraphLaunch(x, P->st));
    }
  }
  CK(cudaStreamSynchronize(P->st));
  res.assign(hres, hres + C);
  drain_profile(P);
  if (getenv("RSVD_DEBUG"))
    for (int c = 0; c < C; ++c)
      fprintf(stderr, "rsvd: chan %d n %d l %d k %d flags %d sweeps %d err_est %.3e status %d\n", c, J.d[c].n,
              J.d[c].l, res[c].k_out, res[c].flags, res[c].sweeps, res[c].err_est, res[c].status);
  if (*herr) return seterr(RSVD_ERR_TIMEOUT, "a bounded device wait expired (code %d)", *herr);
  return RSVD_OK;
}

// Fill the caller's factor records (and host copies of U, S, V).
rsvd_status collect(Job& J, const std::vector<ChanResult>& res, const std::vector<int>& warn, rsvd_factors* f,
                    rsvd_status* per_item, rsvd_status* worst_out) {
  rsvd_plan_s* P = J.P;
  rsvd_status worst = RSVD_OK;
  for (int c = 0; c < J.C; ++c) {
    rsvd_status s = (rsvd_status)res[c].status;
    if (s == RSVD_OK && warn[c]) s = (rsvd_status)warn[c];
    f[c].k_out = res[c].k_out;
    f[c].l_used = res[c].l_used;
    f[c].err_est = res[c].err_est;
    f[c].status = s;
    if (per_item) per_item[c] = s;
    if (s < 0 && (worst >= 0 || s < worst)) worst = s;
    else if (worst >= 0 && s > worst) worst = s;
    if (f[c].mem == RSVD_MEM_HOST && res[c].k_out > 0) {
      const int k = res[c].k_out, n = J.d[c].n;
      CK(cudaMemcpy2DAsync(f[c].U, f[c].ldu * sizeof(double), J.ch[c].U, (size_t)n * sizeof(double),
                           (size_t)n * sizeof(double), k, cudaMemcpyDeviceToHost, P->st));
      CK(cudaMemcpy2DAsync(f[c].V, f[c].ldv * sizeof(double), J.ch[c].V, (size_t)n * sizeof(double),
                           (size_t)n * sizeof(double), k, cudaMemcpyDeviceToHost, P->st));
      CK(cudaMemcpyAsync(f[c].S, J.ch[c].S, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, P->st));
    }
  }
  CK(cudaStreamSynchronize(P->st));
  *worst_out = worst;
  return RSVD_OK;
}

// Fixed l per channel (lvec, else k + p): FIXED and TOL policies.
rsvd_status run_fixed_l(rsvd_plan_s* P, int C, const rsvd_matrix* A, rsvd_factors* f, rsvd_status* per_item,
                        const std::vector<int>* lvec, bool reuse_words) {
  Job J;
  init_job(J, P, C, A, f);
  std::vector<int> warn;
  make_dims(J, lvec, warn, J.mixed ? NPROBE : 0);
  size_t need = 0;
  if (rsvd_status s = build_job(J, nullptr, JOB_MAIN, reuse_words, &need, nullptr)) return s;
  if (!reuse_words) {
    if (rsvd_status s = grow_ws(P, need)) return s;
  } else if (need > P->ws_cap) {
    return seterr(RSVD_ERR_OOM, "workspace sized for the probe is too small");
  }
  if (rsvd_status s = build_job(J, P->ws, JOB_MAIN, reuse_words, &need, nullptr)) return s;
  if (need > P->ws_cap) return seterr(RSVD_ERR_OOM, "workspace estimate exceeded");
  std::vector<ChanResult> res;
  if (rsvd_status s = execute(J, !reuse_words, res)) return s;
  rsvd_status worst = RSVD_OK;
  if (rsvd_status s = collect(J, res, warn, f, per_item, &worst)) return s;
  if (worst < 0) seterr(worst, "at least one channel failed (see per-item status)");
  return worst;
}

// Probe features (and rank-model predictions when the plan has weights) of C
// channels; sizes the workspace for a decomposition with up to lcap columns.
rsvd_status run_probe(rsvd_plan_s* P, int C, const rsvd_matrix* A, rsvd_factors* f, int lcap,
                      std::vector<float>* feat, std::vector<float>* pred) {
  Job Jp;
  init_job(Jp, P, C, A, f);
  std::vector<int> warn;
  std::vector<int> l16(C, 16);
  make_dims(Jp, &l16, warn, 0);
  size_t need_p = 0, need_m = 0;
  if (rsvd_status s = build_job(Jp, nullptr, JOB_PROBE, false, &need_p, nullptr)) return s;
  {
    Job Jm;
    init_job(Jm, P, C, A, f);
    std::vector<int> lc(C, lcap);
    make_dims(Jm, &lc, warn, Jm.mixed ? NPROBE : 0);
    if (rsvd_status s = build_job(Jm, nullptr, JOB_MAIN, true, &need_m, nullptr)) return s;
  }
  if (rsvd_status s = grow_ws(P, std::max(need_p, need_m))) return s;
  ProbeOut po;
  if (rsvd_status s = build_job(Jp, P->ws, JOB_PROBE, false, &need_p, &po)) return s;
  std::vector<ChanResult> res;
  if (rsvd_status s = execute(Jp, true, res)) return s;
  if (feat) {
    feat->resize((size_t)C * 19);
    CK(cudaMemcpy(feat->data(), po.feat, sizeof(float) * C * 19, cudaMemcpyDeviceToHost));
  }
  if (pred) {
    pred->resize((size_t)C * 2);
    CK(cudaMemcpy(pred->data(), po.pred, sizeof(float) * C * 2, cudaMemcpyDeviceToHost));
  }
  for (int c = 0; c < C; ++c)
    if (res[c].flags & FLAG_NONFINITE) return seterr(RSVD_ERR_NONFINITE, "channel %d has NaN/Inf entries", c);
  return RSVD_OK;
}

// Learned rank: probe -> features -> network -> per-channel
// l = 1.2 (k^ + p^), one fixed-l decomposition (reusing the probe's V words);
// channels whose rank rule misses the tolerance get one retry at 1.5 l, then
// the adaptive loop in the plan's precision (stored channels and tile rules
// alike); every result is accepted only by the rank rule's error check.  A
// channel that already drew all the columns it may (n or l_max) keeps its
// best factors and TOL_NOT_MET.
rsvd_status run_learned(rsvd_plan_s* P, int C, const rsvd_matrix* A, rsvd_factors* f, rsvd_status* per_item) {
  if (!P->o.mlp_weights) return seterr(RSVD_ERR_INVALID_ARG, "learned rank needs mlp_weights");
  const int lcap_opt = P->o.l_max > 0 ? P->o.l_max : 1024;
  int lcap = 16;
  for (int c = 0; c < C; ++c) lcap = std::max(lcap, (int)std::min<int64_t>(A[c].n, lcap_opt));
  const bool dbg = getenv("RSVD_DEBUG") != nullptr;
  auto now = []() { return std::chrono::steady_clock::now(); };
  auto ms_since = [&](std::chrono::steady_clock::time_point t) {
    return std::chrono::duration<double, std::milli>(now() - t).count();
  };
  auto t0 = now();
  std::vector<float> pred;
  if (rsvd_status s = run_probe(P, C, A, f, lcap, nullptr, &pred)) return s;
  std::vector<int> lvec(C);
  for (int c = 0; c < C; ++c) {
    const double k = std::exp((double)pred[2 * c]), p = std::exp((double)pred[2 * c + 1]);
    const int cap = (int)std::min<int64_t>(A[c].n, lcap_opt);
    // 20% headroom over the predicted k + p: a miss costs a second run
    int l = (int)rup((int64_t)std::ceil(1.2 * (k + std::max(p, 1.0))), 16);
    lvec[c] = std::max(16, std::min(l, cap));
  }
  if (dbg) fprintf(stderr, "rsvd learned: probe %.2f ms\n", ms_since(t0));
  t0 = now();
  std::vector<rsvd_status> st(C, RSVD_OK);
  rsvd_status r = run_fixed_l(P, C, A, f, st.data(), &lvec, true);
  if (dbg) {
    fprintf(stderr, "rsvd learned: first run %.2f ms\n", ms_since(t0));
    for (int c = 0; c < C; ++c)
      fprintf(stderr, "rsvd learned: chan %d n %lld pred k %.1f p %.1f l %d k_out %d status %d\n", c,
              (long long)A[c].n, std::exp((double)pred[2 * c]), std::exp((double)pred[2 * c + 1]), lvec[c],
              f[c].k_out, (int)st[c]);
  }
  if (r < 0 && r != RSVD_ERR_TOL_NOT_MET && r != RSVD_ERR_NOT_CONVERGED) return r;
  // channels that missed the tolerance: once more with 1.5x the columns,
  // then the adaptive loop; a channel that already drew every column it may
  // (n or l_max) keeps its best factors and TOL_NOT_MET
  for (int attempt = 0; attempt < 2; ++attempt) {
    std::vector<int> idx;
    for (int c = 0; c < C; ++c)
      if (st[c] == RSVD_ERR_TOL_NOT_MET && lvec[c] < (int)std::min<int64_t>(A[c].n, lcap_opt)) idx.push_back(c);
    if (idx.empty()) break;
    std::vector<rsvd_matrix> As(idx.size());
    std::vector<rsvd_factors> fs(idx.size());
    std::vector<int> ls(idx.size());
    for (size_t i = 0; i < idx.size(); ++i) {
      As[i] = A[idx[i]];
      fs[i] = f[idx[i]];
      ls[i] = std::min<int>((int)std::min<int64_t>(A[idx[i]].n, lcap_opt), (int)rup(3 * lvec[idx[i]] / 2, 16));
      lvec[idx[i]] = ls[i];
    }
    std::vector<rsvd_status> sts(idx.size());
    t0 = now();
    if (attempt == 0) {
      r = run_fixed_l(P, (int)idx.size(), As.data(), fs.data(), sts.data(), &ls, false);
    } else {
      // the plain adaptive loop in the plan's precision (a temporary plan
      // sharing the stream)
      rsvd_plan_s Q;
      Q.o = P->o;
      Q.o.rank_policy = RSVD_RANK_ADAPTIVE;
      Q.slices = P->slices;
      Q.st = P->st;
      Q.d_err = P->d_err;
      Q.d_coop = P->d_coop;
      Q.profiling = P->profiling;
      r = run_adaptive(&Q, (int)idx.size(), As.data(), fs.data(), sts.data());
      P->prof.tc_launches += Q.prof.tc_launches; P->prof.tc_ms += Q.prof.tc_ms;
      P->prof.tc_bytes += Q.prof.tc_bytes; P->prof.tc_flops += Q.prof.tc_flops;
      P->prof.f64_launches += Q.prof.f64_launches; P->prof.f64_ms += Q.prof.f64_ms;
      P->prof.f64_flops += Q.prof.f64_flops;
      if (Q.ws) cudaFree(Q.ws);
      if (Q.hp) cudaFreeHost(Q.hp);
      for (cudaEvent_t e : Q.ev_pool) cudaEventDestroy(e);
    }
    if (r < 0 && r != RSVD_ERR_TOL_NOT_MET && r != RSVD_ERR_NOT_CONVERGED) return r;
    if (dbg) fprintf(stderr, "rsvd learned: %s for %zu channels %.2f ms\n", attempt == 0 ? "retry" : "fallback",
                     idx.size(), ms_since(t0));
    for (size_t i = 0; i < idx.size(); ++i) {
      f[idx[i]] = fs[i];
      st[idx[i]] = sts[i];
    }
  }
  rsvd_status worst = RSVD_OK;
  for (int c = 0; c < C; ++c) {
    if (per_item) per_item[c] = st[c];
    f[c].status = st[c];
    if (st[c] < 0 && (worst >= 0 || st[c] < worst)) worst = st[c];
    else if (worst >= 0 && st[c] > worst) worst = st[c];
  }
  if (worst < 0) seterr(worst, "at least one channel failed (see per-item status)");
  return worst;
}

}  // namespace rsvd_api
