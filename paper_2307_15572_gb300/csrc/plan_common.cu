// Host plumbing shared by the decomposition paths: workspace and pinned
// buffers, event timing, launch-shape autotuner, grouped tile-product step
// builders, tile-rule buffer layout, job layout and argument validation.
#include "api_internal.h"

namespace rsvd_api {

// Bump allocator over the workspace; base == nullptr only measures.

// Descriptor arena: built on the host, uploaded once, referenced by kernels.

rsvd_status grow_pinned(rsvd_plan_s* P, size_t bytes) {
  if (bytes <= P->hp_cap) return RSVD_OK;
  CK(cudaStreamSynchronize(P->st));
  drop_graphs(P);                        // their copy nodes name the old buffer
  if (P->hp) cudaFreeHost(P->hp);
  P->hp = nullptr;
  P->hp_cap = 0;
  size_t cap = std::max(bytes, (size_t)1 << 20);
  CK(cudaHostAlloc((void**)&P->hp, cap, cudaHostAllocDefault));
  P->hp_cap = cap;
  return RSVD_OK;
}

rsvd_status grow_ws(rsvd_plan_s* P, size_t bytes) {
  if (bytes <= P->ws_cap) return RSVD_OK;
  CK(cudaStreamSynchronize(P->st));
  drop_graphs(P);                        // their launches name the old workspace
  if (P->ws) cudaFree(P->ws);
  P->ws = nullptr;
  P->ws_cap = 0;
  size_t cap = rup((int64_t)bytes, (int64_t)1 << 21);
  CK(cudaMalloc((void**)&P->ws, cap));
  P->ws_cap = cap;
  return RSVD_OK;
}

// Event pair for a timed launch (pool grows, events are reused across calls).
void timed_begin(rsvd_plan_s* P, cudaEvent_t* a, cudaEvent_t* b) {
  while (P->ev_pool.size() < P->ev_next + 2) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    P->ev_pool.push_back(e);
  }
  *a = P->ev_pool[P->ev_next++];
  *b = P->ev_pool[P->ev_next++];
  cudaEventRecord(*a, P->st);
}

// Small SVD of every channel's factor: one CTA per channel while the factor
// fits its shared memory, else the cooperative kernel (several CTAs per
// channel; not while the stream is being captured into a graph).
void run_jacobi(const Chan* dch, const std::vector<int>& ls, int fp32, int maxl, int* coop, int* err, cudaStream_t st) {
  const int C = (int)ls.size();
  const int ve = fp32 ? 4 : 2;
  const size_t lp = (size_t)((maxl + 8 * ve - 1) / (8 * ve) * (8 * ve));
  const size_t bytes = (fp32 ? 1 : 2) * (size_t)maxl * lp * (fp32 ? 4 : 8);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (st) cudaStreamIsCapturing(st, &cs);
  if (bytes > 200 * 1024 && cs == cudaStreamCaptureStatusNone &&
      launch_jacobi_coop(dch, ls.data(), C, fp32, coop, err, st) == 0)
    return;
  launch_jacobi(dch, C, fp32, maxl, st);
}

// Cholesky + inverse of every channel's Gram: one CTA per channel while the
// factor fits its shared memory, else the cooperative kernel.
void run_chol(const Chan* dch, const std::vector<int>& ls, int accumulate, int maxl, int f32inv, int f32_chol,
              int conditional, int* coop, int* err, cudaStream_t st) {
  const int C = (int)ls.size();
  const size_t esz = f32_chol ? sizeof(float) : sizeof(double);
  size_t bytes = (size_t)maxl * (maxl + 1) * esz + (size_t)maxl * sizeof(double);
  const size_t b32 = (size_t)maxl * (maxl + 1) * sizeof(float) + 9 * (size_t)maxl * sizeof(float);
  if (b32 > bytes) bytes = b32;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (st) cudaStreamIsCapturing(st, &cs);
  if (bytes > 200 * 1024 && cs == cudaStreamCaptureStatusNone &&
      launch_chol_coop(dch, ls.data(), C, accumulate, f32_chol, conditional, coop, err, st) == 0)
    return;
  launch_chol_inv(dch, C, accumulate, maxl, f32inv, st, f32_chol, conditional);
}

// Fold the timed launches of a finished (synchronised) job into the counters.
void drain_profile(rsvd_plan_s* P) {
  for (auto& t : P->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t.a, t.b);
    if (t.kind == 0) { P->prof.tc_launches++; P->prof.tc_ms += ms; P->prof.tc_bytes += t.bytes; P->prof.tc_flops += t.flops; }
    else if (t.kind == 2) { P->prof.gen_launches++; P->prof.gen_ms += ms; P->prof.gen_flops += t.flops; P->prof.gen_mma_flops += t.bytes; }
    else if (t.kind == 3) { P->prof.cvt_launches++; P->prof.cvt_ms += ms; P->prof.cvt_bytes += t.bytes; }
    else if (t.kind == 6) { P->prof.f64in_launches++; P->prof.f64in_ms += ms; P->prof.f64in_bytes += t.bytes; P->prof.f64in_flops += t.flops; }
    else if (t.kind == 5) { P->prof.nn_launches++; P->prof.nn_ms += ms; P->prof.nn_flops += t.flops; }
    else if (t.kind == 4) { P->prof.gram_launches++; P->prof.gram_ms += ms; P->prof.gram_flops += t.flops; P->prof.gram_mma_flops += t.bytes; }
    else { P->prof.f64_launches++; P->prof.f64_ms += ms; P->prof.f64_flops += t.flops; }
  }
  P->pending.clear();
  P->ev_next = 0;
}

// Split a tile count over k so that the grid covers the GPU `target` tiles
// (by default twice per SM); target 0: no split.
int pick_splits(int64_t tiles, int64_t k, int min_chunk, int64_t target) {
  if (target <= 0 || tiles >= target) return 1;
  int ks = (int)((target + tiles - 1) / tiles);
  int maxk = (int)std::max<int64_t>(1, k / min_chunk);
  return std::max(1, std::min(ks, maxk));
}

// The tensor-core Gram (k_gram_tc) serves the mixed path's n x l Grams when
// every channel has l <= 128 (one 128 x 128 accumulator per level); the
// environment variable RSVD_GRAM=dot2 keeps the CUDA-core compensated Gram.
bool gram_tc_enabled(const Job& J) {
  if (!J.mixed || J.max_l < 1 || J.max_l > 128) return false;
  const char* e = getenv("RSVD_GRAM");
  return !(e && strcmp(e, "dot2") == 0);
}

// The tensor-core tall x small products (k_nn_tc) serve the mixed path's
// products with an l x l (or l x k) right operand when every l <= 128;
// RSVD_NN=simt keeps the CUDA-core FP32 products.
bool nn_tc_enabled(const Job& J) {
  if (!J.mixed || J.max_l < 1 || J.max_l > 128) return false;
  const char* e = getenv("RSVD_NN");
  return !(e && strcmp(e, "simt") == 0);
}

// Everything one batched call needs.

// Tile rule: H words have M padded to whole 64-wide k steps.
int64_t rule_ldh(int M) { return rup(M, 64); }
int rule_panel_rows(int64_t n, int64_t ldb, int nsl) {
  // panel words within ~8 GiB (tunable through RSVD_RULE_PANEL for tests)
  int64_t p = ((int64_t)8 << 30) / std::max<int64_t>(1, (int64_t)nsl * ldb * 2);
  if (const char* e = getenv("RSVD_RULE_PANEL")) p = std::max<int64_t>(128, atoll(e));
  p = std::max<int64_t>(128, p / 128 * 128);
  return (int)std::min<int64_t>(p, rup(n, 128));
}
uint32_t rule_key(uint64_t seed) {
  return lowbias32((uint32_t)seed ^ lowbias32((uint32_t)(seed >> 32)));
}

// Device address of a page-locked host matrix, or null.  On the mixed path V
// is read once (by the conversion to words), so a pinned host V is read in
// place over the CPU-GPU link instead of being staged through a device copy.
const double* host_direct(const rsvd_matrix& A) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, A.data) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type == cudaMemoryTypeHost && at.devicePointer) return (const double*)at.devicePointer;
  return nullptr;
}

// FP64 path: page-locked host channels are read in place by every pass (the
// CPU-GPU link) instead of staged into device memory when their staged copies
// would not fit (free device memory less a quarter kept for the workspace),
// or when the environment sets RSVD_HOST_IN_PLACE=1.  Channels in pageable
// memory are always staged.
bool fp64_reads_host_in_place(const rsvd_matrix* A, int C) {
  if (const char* e = getenv("RSVD_HOST_IN_PLACE"))
    if (atoi(e) == 1) return true;
  size_t need = 0;
  for (int c = 0; c < C; ++c)
    if (A[c].kind == RSVD_DENSE_F64 && A[c].mem == RSVD_MEM_HOST) need += (size_t)A[c].n * A[c].n * sizeof(double);
  if (need == 0) return false;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return need > fr / 4 * 3;
}

// Per-batch tile offsets (prefix sums) uploaded through the arena.
const int* offsets(Job& J, const std::function<int64_t(int)>& per) {
  std::vector<int> off(J.C + 1, 0);
  for (int c = 0; c < J.C; ++c) off[c + 1] = off[c] + (int)per(c);
  return J.ar.put(off.data(), off.size());
}
int total_of(Job& J, const std::function<int64_t(int)>& per) {
  int64_t t = 0;
  for (int c = 0; c < J.C; ++c) t += per(c);
  return (int)t;
}

// ------------------------------------------------------------ autotuner
// A pass with several launch shapes that compute the same result (up to the
// order of FP32/FP64 summation).  Candidate 0 is the fixed default rule.  The
// plan's table maps the pass signature to the chosen candidate; until it has
// one (and while autotuning is on), the first execution outside stream
// capture times every candidate on the caller's data -- one warm-up launch,
// then the better of two timed launches each -- and keeps the fastest unless
// it is within 2% of the default.  Variants only write the pass's output, so
// running several of them in a row leaves the same result.
std::string tune_key(const char* kind, std::initializer_list<int64_t> head, const std::vector<int64_t>& per) {
  std::string k(kind);
  for (int64_t v : head) k.append((const char*)&v, sizeof(v));
  for (int64_t v : per) k.append((const char*)&v, sizeof(v));
  return k;
}

void add_tuned(Job& J, const std::string& key, const std::vector<rsvd_tune_record>& recs,
               const std::vector<std::function<rsvd_status()>>& vars) {
  rsvd_plan_s* P = J.P;
  if (vars.size() == 1) {
    J.steps.push_back(vars[0]);
    return;
  }
  J.tuning = true;
  J.steps.push_back([=]() -> rsvd_status {
    if (const auto* t = P->tuned(key)) return vars[t->rec.choice]();
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (P->st) cudaStreamIsCapturing(P->st, &cs);
    if (cs != cudaStreamCaptureStatusNone) return vars[0]();
    for (auto& e : P->tune_ev)
      if (!e) CK(cudaEventCreate(&e));
    const int prof = P->profiling;
    P->profiling = 0;
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<float> ms(vars.size(), 3.0e38f);
    rsvd_status bad = RSVD_OK;
    if ((bad = vars[0]()) == RSVD_OK) {
      for (int rep = 0; rep < 2 && !bad; ++rep)
        for (size_t i = 0; i < vars.size() && !bad; ++i) {
          cudaEventRecord(P->tune_ev[0], P->st);
          if ((bad = vars[i]())) break;
          cudaEventRecord(P->tune_ev[1], P->st);
          if (cudaEventSynchronize(P->tune_ev[1]) != cudaSuccess) {
            bad = seterr(RSVD_ERR_CUDA, "autotuner: %s", cudaGetErrorString(cudaGetLastError()));
            break;
          }
          float t = 0.f;
          cudaEventElapsedTime(&t, P->tune_ev[0], P->tune_ev[1]);
          ms[i] = std::min(ms[i], t);
        }
    }
    P->profiling = prof;
    if (bad) return bad;
    size_t best = 0;
    for (size_t i = 1; i < vars.size(); ++i)
      if (ms[i] < ms[best]) best = i;
    if (ms[best] > 0.98f * ms[0]) best = 0;
    if (const char* f = getenv("RSVD_TUNE_FORCE")) best = (size_t)std::max(0, atoi(f)) % vars.size();
    rsvd_tune_record r = recs[best];
    r.candidates = (int32_t)vars.size();
    r.choice = (int32_t)best;
    r.ms_default = ms[0];
    r.ms_best = ms[best];
    r.tune_ms = (float)std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    P->tune.push_back({key, r});
    if (getenv("RSVD_DEBUG"))
      fprintf(stderr, "rsvd autotune: kind %d, %d candidates, choice %d (bn %d, split %d, stages %d, order %d): "
              "%.3f ms vs default %.3f ms\n", r.kind, r.candidates, r.choice, r.bn, r.split_target, r.stages,
              r.order, r.ms_best, r.ms_default);
    return vars[best]();
  });
}

// Which candidates to build: the chosen one, all of them (tuning), or the default.
std::vector<int> tune_pick(Job& J, const std::string& key, size_t ncand) {
  if (const auto* t = J.P->tuned(key)) return {t->rec.choice};
  if (J.P->autotune && ncand > 1) {
    std::vector<int> all(ncand);
    for (size_t i = 0; i < ncand; ++i) all[i] = (int)i;
    return all;
  }
  return {0};
}

// ------------------------------------------------------------ step builders
void add_mm(Job& J, MMKind kind, std::vector<MMDesc> md) { J.steps.push_back(make_mm(J, kind, std::move(md))); }

std::function<rsvd_status()> make_mm(Job& J, MMKind kind, std::vector<MMDesc> md) {
  const int tile = tile_of(kind);
  for (auto& m : md) {
    m.tile = tile;
    m.mt = cdiv(m.m, tile);
    m.nt = cdiv(m.n, tile);
  }
  const int C = (int)md.size();               // one descriptor per channel (or per panel)
  std::vector<int> off(C + 1, 0);
  double flops = 0.0;
  for (int c = 0; c < C; ++c) {
    off[c + 1] = off[c] + md[c].mt * md[c].nt * md[c].ks;
    flops += 2.0 * md[c].m * md[c].n * (double)md[c].k;
  }
  const int tiles = off[C];
  const MMDesc* dmd = J.ar.put(md.data(), md.size());
  const int* doff = J.ar.put(off.data(), off.size());
  cudaStream_t st = J.P->st;
  rsvd_plan_s* P = J.P;
  return [=]() {
    const bool timed = P->profiling && kind == MMK_DENSE_F64;
    cudaEvent_t a = nullptr, b = nullptr;
    if (timed) timed_begin(P, &a, &b);
    launch_tile_mm(kind, dmd, doff, C, tiles, st);
    if (timed) {
      cudaEventRecord(b, st);
      P->pending.push_back({a, b, 1, 0.0, flops});
    }
    return RSVD_OK;
  };
}

// Gram-like TN product with split partials and fixed-order reduction:
// out_c (m x n, ld m) = A_c^T B_c over rows_c rows (leading dims ld_c).
void add_tn_ex(Job& J, MMKind kind, std::function<const void*(int)> Ap, std::function<const void*(int)> Bp,
               std::function<double*(int)> outp, std::function<int(int)> mcols, std::function<int(int)> ncols,
               bool sym, std::function<int(int)> rows, std::function<int64_t(int)> ld,
               std::function<int(int)> splits, std::function<const int*(int)> cond) {
  std::vector<MMDesc> md(J.C);
  std::vector<double*> outs(J.C);
  int max_elems = 1;
  for (int c = 0; c < J.C; ++c) {
    const int nr = rows(c);
    MMDesc m{};
    m.A = Ap(c); m.lda = ld(c);
    m.B = Bp(c); m.ldb = ld(c);
    m.m = mcols(c); m.n = ncols(c); m.k = nr;
    m.mt = cdiv(m.m, 64); m.nt = cdiv(m.n, 64);
    m.kchunk = (int)rup(cdiv(nr, splits(c)), 16);
    m.ks = cdiv(nr, m.kchunk);
    m.mode = MM_PARTIAL;
    m.sym = sym ? 1 : 0;
    m.Cm = J.ch[c].gpart;
    m.ldc = m.m;
    m.pstride = (int64_t)m.m * m.n;
    m.cond = cond ? cond(c) : nullptr;
    md[c] = m;
    outs[c] = outp(c);
    max_elems = std::max(max_elems, m.m * m.n);
  }
  add_mm(J, kind, md);
  for (auto& m : md) m.tile = tile_of(kind);
  const MMDesc* dmd = J.ar.put(md.data(), md.size());
  double* const* douts = J.ar.put(outs.data(), outs.size());
  cudaStream_t st = J.P->st;
  const int C = J.C;
  J.steps.push_back([=]() {
    launch_reduce_partials(dmd, douts, C, max_elems, st);
    return RSVD_OK;
  });
}

// The tall case: A_c, B_c are n_c x . panels with leading dim ldt_c, split in
// gsplit_c row chunks.
void add_tn(Job& J, MMKind kind, std::function<const void*(int)> Ap, std::function<const void*(int)> Bp,
            std::function<double*(int)> outp, std::function<int(int)> mcols, std::function<int(int)> ncols,
            bool sym) {
  add_tn_ex(J, kind, Ap, Bp, outp, mcols, ncols, sym, [&](int c) { return J.d[c].n; },
            [&](int c) { return J.d[c].ldt; }, [&](int c) { return J.d[c].gsplit; });
}

std::vector<int> chan_ls(const Job& J) {
  std::vector<int> ls(J.C);
  for (int c = 0; c < J.C; ++c) ls[c] = J.d[c].l;
  return ls;
}

void add_chol(Job& J, int accumulate, int f32_chol) {
  const Chan* dch = J.d_ch;
  const int maxl = J.max_l;
  const int f32inv = J.mixed ? 1 : 0;
  cudaStream_t st = J.P->st;
  const std::vector<int> ls = chan_ls(J);
  int* coop = J.P->d_coop;
  int* derr_w = J.P->d_err;
  J.steps.push_back([=]() {
    run_chol(dch, ls, accumulate, maxl, f32inv, f32_chol, 0, coop, derr_w, st);
    return RSVD_OK;
  });
}

// Tile-rule buffers: factor words per channel, then one panel buffer and
// partial area shared by the channels (they are generated one after another).
// FP64 path: the factor panel in FP64 per channel, one FP64 row panel
// (column-major, panel x n) and the noise kernel's partials.
int rule_panel_rows64(int64_t maxn) {
  int64_t p = ((int64_t)8 << 30) / std::max<int64_t>(1, maxn * 8);
  if (const char* e = getenv("RSVD_RULE_PANEL")) p = std::max<int64_t>(128, atoll(e));
  p = std::max<int64_t>(128, p / 128 * 128);
  return (int)std::min<int64_t>(p, rup(maxn, 128));
}

void lay_rule64(Bump& b, const std::vector<ChanDims>& d, const rsvd_matrix* A, std::vector<Job::RuleDev>& rd,
                double*& p64, double*& part, int& panel) {
  const int C = (int)d.size();
  rd.assign(C, Job::RuleDev{});
  int maxn = 1;
  for (int c = 0; c < C; ++c) {
    Job::RuleDev& r = rd[c];
    r.M = A[c].rule_m;
    r.ldh = rule_ldh(r.M);
    r.H64 = b.take<double>((size_t)d[c].n * r.ldh);
    r.key = rule_key(A[c].rule_seed);
    maxn = std::max(maxn, d[c].n);
  }
  panel = rule_panel_rows64(maxn);
  for (int c = 0; c < C; ++c) {
    const int P = std::min<int>(panel, (int)rup(d[c].n, 128));
    rd[c].psums = b.take<double>(2 * (size_t)cdiv(d[c].n, P));
  }
  p64 = b.take<double>((size_t)panel * maxn);
  part = b.take<double>(2 * (size_t)kRuleNoiseBlocks);
}

void lay_rule(Bump& b, const std::vector<ChanDims>& d, const rsvd_matrix* A, int nsl, std::vector<Job::RuleDev>& rd,
              __nv_bfloat16* (&pw)[3], double*& part, int& panel) {
  const int C = (int)d.size();
  rd.assign(C, Job::RuleDev{});
  int64_t maxldb = 64, maxitems = 1;
  int maxn = 1;
  for (int c = 0; c < C; ++c) {
    Job::RuleDev& r = rd[c];
    r.M = A[c].rule_m;
    r.ldh = rule_ldh(r.M);
    for (int w = 0; w < 2; ++w) r.H[w] = b.take<__half>((size_t)d[c].n * r.ldh);
    r.hscale = rule_hscale(A[c].rule_w, r.M);
    r.key = rule_key(A[c].rule_seed);
    r.amp3 = (float)(A[c].rule_eta * 1.7320508075688772);
    maxldb = std::max<int64_t>(maxldb, d[c].ldb);
    maxn = std::max(maxn, d[c].n);
  }
  panel = rule_panel_rows(maxn, maxldb, nsl);
  for (int c = 0; c < C; ++c) {
    const int P = std::min<int>(panel, (int)rup(d[c].n, 128));
    rd[c].psums = b.take<double>(2 * (size_t)cdiv(d[c].n, P));
    maxitems = std::max<int64_t>(maxitems, (int64_t)cdiv(d[c].n, 128) * cdiv(P, 128));
  }
  for (int w = 0; w < nsl; ++w) pw[w] = b.take<__nv_bfloat16>((size_t)panel * maxldb);
  part = b.take<double>((size_t)maxitems * 8);
}

// ------------------------------------------------------------ layout
// Lay out per-channel buffers; with base == nullptr only measures.  The
// rank-independent part (staged input, V words, partials, results) comes
// first, so a probe job and the decomposition after it (different l) share it.
void layout(Job& J, Bump& b) {
  J.ch.assign(J.C, Chan{});
  J.staged.assign(J.C, 0);
  const bool in_place64 = !J.mixed && J.host_in_place;
  for (int c = 0; c < J.C; ++c) {
    const ChanDims& d = J.d[c];
    Chan& h = J.ch[c];
    const rsvd_matrix& A = J.A[c];
    if (J.rule) {
      h.fro_part = b.take<double>(cdiv(d.n, 8));
      continue;
    }
    if (A.mem == RSVD_MEM_HOST) {
      const double* direct = (J.mixed || in_place64) ? host_direct(A) : nullptr;
      if (direct) { h.A = direct; h.lda = A.ld; }
      else { h.A = b.take<double>((size_t)d.n * d.n); h.lda = d.n; J.staged[c] = 1; }
    } else {
      h.A = A.data; h.lda = A.ld;
    }
    if (J.mixed) {
      for (int s = 0; s < J.nsl; ++s) h.Ab[s] = b.take<__nv_bfloat16>((size_t)d.n * d.ldb);
      h.wres_part = b.take<double>(cdiv(d.n, 8));
    }
    h.fro_part = b.take<double>(cdiv(d.n, 8));
  }
  if (J.rule && J.mixed) lay_rule(b, J.d, J.A, J.nsl, J.rd, J.pw, J.part, J.panel);
  if (J.rule && !J.mixed) lay_rule64(b, J.d, J.A, J.rd, J.p64, J.part, J.panel);
  J.d_res = b.take<ChanResult>(J.C);
  for (int c = 0; c < J.C; ++c) {
    const ChanDims& d = J.d[c];
    Chan& h = J.ch[c];
    const rsvd_factors& F = J.f[c];
    h.n = d.n; h.l = d.l; h.k_cap = d.kcap; h.k_fixed = J.P->o.k;
    h.ldt = d.ldt; h.ldb = d.ldb; h.lw = d.lw; h.nprobe = d.s;
    h.tol = d.tol;
    const size_t L2 = (size_t)d.l * d.l;
    const size_t L2p = (size_t)d.l * (d.l + 32);      // Jacobi's padded working copies when not in smem
    h.G = b.take<double>(L2p); h.R = b.take<double>(L2); h.Ri = b.take<double>(L2p);
    h.M = b.take<double>(L2); h.J = b.take<double>(L2);
    h.sig = b.take<double>(d.l); h.scr = b.take<double>(d.l);
    h.res = J.d_res ? J.d_res + c : nullptr;
    if (!J.mixed) {
      const size_t T = (size_t)d.ldt * d.l;
      h.X = b.take<double>(T); h.Y = b.take<double>(T); h.Q2 = b.take<double>(T);
      h.gpart = b.take<double>((size_t)d.gsplit * L2);
    } else {
      h.Ri32 = b.take<float>(L2);
      for (int s = 0; s < J.nsl; ++s) h.Xb[s] = b.take<__nv_bfloat16>((size_t)d.lw * d.ldb);
      h.Y32 = b.take<float>((size_t)d.ldt * d.lw);
      h.Q32 = b.take<float>((size_t)d.ldt * d.l);
      h.T32 = b.take<float>((size_t)d.ldt * d.l);
      h.gpart = b.take<double>((size_t)d.gsplit * d.l * std::max(d.l, d.s));
      if (gram_tc_enabled(J)) {
        h.gtc_part = b.take<float>((size_t)gram_tc_part_floats(d.n));
        h.gtc_exp = b.take<int>((size_t)cdiv(d.n, 128) * 128);
      }
      if (nn_tc_enabled(J)) {
        h.nn_bimg = b.take<unsigned char>((size_t)nn_tc_img_bytes());
        h.nn_fexp = b.take<int>(128);
      }
      h.C64 = b.take<double>((size_t)d.l * std::max(d.s, 1));
      h.C32 = b.take<float>((size_t)d.l * 32);
      h.est_part = b.take<double>((size_t)std::max(d.s, 1) * (1 + d.l));
    }
    if (F.mem == RSVD_MEM_HOST) {
      h.U = b.take<double>((size_t)d.n * d.kcap); h.ldu = d.n;
      h.V = b.take<double>((size_t)d.n * d.kcap); h.ldv = d.n;
      h.S = b.take<double>(d.kcap);
    } else {
      h.U = F.U; h.ldu = F.ldu; h.V = F.V; h.ldv = F.ldv; h.S = F.S;
      if (!h.U) { h.U = b.take<double>((size_t)d.n * d.kcap); h.ldu = d.n; }
      if (!h.V) { h.V = b.take<double>((size_t)d.n * d.kcap); h.ldv = d.n; }
    }
  }
}

// Parameters of a tile rule: 1 <= rule_m <= 4096 finite centres, widths s > 0,
// weights w >= 0, noise amplitude >= 0.
rsvd_status check_rule(const rsvd_matrix& a) {
  if (a.rule_m < 1 || a.rule_m > 4096) return seterr(RSVD_ERR_INVALID_ARG, "rule_m %d outside [1, 4096]", a.rule_m);
  if (!a.rule_c || !a.rule_s || !a.rule_w) return seterr(RSVD_ERR_INVALID_ARG, "rule parameter array is NULL");
  for (int m = 0; m < a.rule_m; ++m)
    if (!std::isfinite(a.rule_c[m]) || !(a.rule_s[m] > 0.0) || !std::isfinite(a.rule_s[m]) || !(a.rule_w[m] >= 0.0) ||
        !std::isfinite(a.rule_w[m]))
      return seterr(RSVD_ERR_INVALID_ARG, "rule term %d needs finite c, s > 0, w >= 0", m);
  if (!(a.rule_eta >= 0.0) || !std::isfinite(a.rule_eta))
    return seterr(RSVD_ERR_INVALID_ARG, "rule_eta must be finite and >= 0");
  return RSVD_OK;
}

rsvd_status validate(const rsvd_plan_s* P, int C, const rsvd_matrix* A, rsvd_factors* f) {
  if (!P) return seterr(RSVD_ERR_INVALID_ARG, "plan is NULL");
  if (C < 1) return seterr(RSVD_ERR_INVALID_ARG, "channel count %d < 1", C);
  if (!A || !f) return seterr(RSVD_ERR_INVALID_ARG, "matrix or factor array is NULL");
  for (int c = 0; c < C; ++c) {
    const rsvd_matrix& a = A[c];
    const rsvd_factors& F = f[c];
    if (a.kind != RSVD_DENSE_F64 && a.kind != RSVD_TILE_RULE)
      return seterr(RSVD_ERR_INVALID_ARG, "channel %d: matrix kind %d unknown", c, a.kind);
    if (a.kind != A[0].kind)
      return seterr(RSVD_ERR_UNSUPPORTED, "channel %d: stored and tile-rule channels in one call", c);
    if (a.n < 1 || a.n > P->o.n_max)
      return seterr(RSVD_ERR_INVALID_ARG, "channel %d: n = %lld outside [1, n_max = %lld]", c, (long long)a.n,
                    (long long)P->o.n_max);
    if (a.n > 2000000000LL / 64) return seterr(RSVD_ERR_INVALID_ARG, "channel %d: n too large", c);
    if (a.kind == RSVD_TILE_RULE) {
      if (rsvd_status s = check_rule(a)) return s;
    } else {
      if (!a.data) return seterr(RSVD_ERR_INVALID_ARG, "channel %d: data is NULL", c);
      if (a.ld < a.n)
        return seterr(RSVD_ERR_INVALID_ARG, "channel %d: ld %lld < n %lld", c, (long long)a.ld, (long long)a.n);
      if (a.mem != RSVD_MEM_DEVICE && a.mem != RSVD_MEM_HOST)
        return seterr(RSVD_ERR_INVALID_ARG, "channel %d: bad mem", c);
    }
    if (F.mem != RSVD_MEM_DEVICE && F.mem != RSVD_MEM_HOST) return seterr(RSVD_ERR_INVALID_ARG, "channel %d: bad factor mem", c);
    if (F.k_cap < 1) return seterr(RSVD_ERR_INVALID_ARG, "channel %d: k_cap %d < 1", c, F.k_cap);
    if (!F.S) return seterr(RSVD_ERR_INVALID_ARG, "channel %d: S is NULL", c);
    if (F.U && F.ldu < a.n) return seterr(RSVD_ERR_INVALID_ARG, "channel %d: ldu < n", c);
    if (F.V && F.ldv < a.n) return seterr(RSVD_ERR_INVALID_ARG, "channel %d: ldv < n", c);
    if (F.mem == RSVD_MEM_HOST && (!F.U || !F.V))
      return seterr(RSVD_ERR_INVALID_ARG, "channel %d: host factors need U and V", c);
  }
  return RSVD_OK;
}

}  // namespace rsvd_api
