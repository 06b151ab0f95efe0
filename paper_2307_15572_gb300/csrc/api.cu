// C ABI of the library: plan, grouped decomposition of channel blocks,
// exact residual.  Host-side orchestration only; all arithmetic of the
// method runs in the kernels (k_*.cu).
//
// Pipeline per batch (every launch covers all channels):
//   FP64 path  (every step in FP64 on CUDA cores)
//     X = P (Philox, Fig. 1 step 1)          Y = V X
//     Q = CholeskyQR2(Y)                     [Z = Q X of step 1]
//     q rounds: Y = V Q, Q = CQR2(Y); Y = V Q, Q = CQR2(Y)
//     W = V Q  (= Y^T of step 1', V symmetric)
//     W = Q2 R (CQR2, R accumulated), R^T = X Sigma J^T (one-sided Jacobi)
//     so Y^T-SVD: L_Y = X, R_paper = Q2 J; rank k; L = Q X_k (step 3), R = Q2 J_k
//   mixed path (passes over V on tensor cores, V and X as BF16 words)
//     V -> words (+ ||V||^2);  P -> BF16;  Y = V P (tcgen05)
//     Q = CQR2(Y) with compensated (Dot2) Grams, FP64 Cholesky, FP32 solve
//     q rounds as above; [W | V G] = V [Q | G]  (G = 16 probe columns)
//     W^T W = R^T R (Dot2 Gram, FP64 Cholesky); Jacobi on R^T -> X, Sigma
//     rank from the probe estimate; L = Q X_k, R_paper = W X_k Sigma_k^{-1}
#include <math.h>
#include <stdarg.h>
#include <stddef.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <functional>
#include <string>
#include <vector>

#include "kernels.h"
#include "tc_gemm.h"
#include "../../include/rsvd_mlp.h"

using namespace rsvd;

#include <atomic>
namespace rsvd {
static std::atomic<long long> g_launches{0};
void note_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace rsvd

namespace {

thread_local char g_err[1024] = "";

rsvd_status seterr(rsvd_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

#define CK(call)                                                                             \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return seterr(e_ == cudaErrorMemoryAllocation ? RSVD_ERR_OOM : RSVD_ERR_CUDA, "%s: %s", \
                    #call, cudaGetErrorString(e_));                                          \
  } while (0)

}  // namespace

namespace rsvd {
void clear_error_text() { g_err[0] = 0; }
rsvd_status set_error_text(rsvd_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}
}  // namespace rsvd

namespace {

inline int64_t rup(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

constexpr int NPROBE = 32;
constexpr int NSM = 152;

}  // namespace

struct rsvd_plan_s {
  rsvd_opts o;
  cudaStream_t st = nullptr;
  char* ws = nullptr;
  size_t ws_cap = 0;
  char* hp = nullptr;      // pinned host staging
  size_t hp_cap = 0;
  int* d_err = nullptr;    // device error word
  int* d_coop = nullptr;   // scratch of the cooperative Jacobi (after the error word)
  int slices = 2;
  // profiling
  int profiling = 0;
  rsvd_profile prof{};
  std::vector<cudaEvent_t> ev_pool;
  struct Timed { cudaEvent_t a, b; int kind; double bytes, flops; };   // kind 0 tc, 1 FP64, 2 rule generation, 3 conversion
  std::vector<Timed> pending;
  size_t ev_next = 0;
  long long launch_base = 0;
  // CUDA graphs of whole decompositions, keyed by everything that shapes the
  // launch sequence (descriptor contents are re-uploaded by the first node)
  int graphs = 0;
  struct GraphEntry { std::string key; cudaGraphExec_t exec; long long launches; uint64_t used; };
  std::vector<GraphEntry> gcache;
  uint64_t gclock = 0;
  // autotuner: launch-shape choice per pass signature (see add_tuned)
  int autotune = 0;
  struct TuneEntry { std::string key; rsvd_tune_record rec; };
  std::vector<TuneEntry> tune;
  cudaEvent_t tune_ev[2] = {nullptr, nullptr};
  const TuneEntry* tuned(const std::string& k) const {
    for (const auto& t : tune)
      if (t.key == k) return &t;
    return nullptr;
  }
};

void drop_graphs(rsvd_plan_s* P) {
  for (auto& g : P->gcache) cudaGraphExecDestroy(g.exec);
  P->gcache.clear();
}

namespace {

// Bump allocator over the workspace; base == nullptr only measures.
struct Bump {
  char* base;
  size_t off = 0;
  explicit Bump(char* b) : base(b) {}
  template <class T>
  T* take(size_t n) {
    off = (off + 255) & ~(size_t)255;
    T* p = base ? (T*)(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};

// Descriptor arena: built on the host, uploaded once, referenced by kernels.
struct Arena {
  std::vector<char> h;
  char* dbase = nullptr;
  template <class T>
  T* put(const T* src, size_t n, size_t align = 64) {
    size_t o = (h.size() + align - 1) & ~(align - 1);
    h.resize(o + n * sizeof(T));
    memcpy(h.data() + o, src, n * sizeof(T));
    return (T*)(dbase + o);
  }
};

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
    else { P->prof.f64_launches++; P->prof.f64_ms += ms; P->prof.f64_flops += t.flops; }
  }
  P->pending.clear();
  P->ev_next = 0;
}

// Split a tile count over k so that the grid covers the GPU `target` tiles
// (by default twice per SM); target 0: no split.
int pick_splits(int64_t tiles, int64_t k, int min_chunk, int64_t target = 2 * NSM) {
  if (target <= 0 || tiles >= target) return 1;
  int ks = (int)((target + tiles - 1) / tiles);
  int maxk = (int)std::max<int64_t>(1, k / min_chunk);
  return std::max(1, std::min(ks, maxk));
}

struct ChanDims {
  int n, l, lw, s, kcap, gsplit;
  int64_t ldt, ldb;
  double tol;
};

// Everything one batched call needs.
struct Job {
  rsvd_plan_s* P;
  int C;
  const rsvd_matrix* A;
  rsvd_factors* f;
  bool mixed;
  bool measure = true;       // first layout pass: sizes only, no device pointers
  int q, nsl, policy;
  double tol;
  std::vector<ChanDims> d;
  std::vector<Chan> ch;              // host copies of the descriptors
  std::vector<std::function<rsvd_status()>> steps;
  Arena ar;
  Chan* d_ch = nullptr;
  ChanResult* d_res = nullptr;
  int max_l = 0, max_lw = 0, max_kcap = 0;
  // tile-rule channels (all channels of the job, or none)
  bool rule = false;
  bool skip_convert = false;            // V words reused from a probe job
  std::vector<char> staged;             // host V copied to the device (else read in place)
  bool probe_job = false;
  int panel = 0;                        // rows of A generated per panel
  struct RuleDev {
    __half* H[2];                       // factor words (FP16, scaled by hscale)
    double hscale;
    double* H64;                        // FP64 path: the factor panel in FP64
    int64_t ldh;
    int M;
    uint32_t key;
    float amp3;
    double* psums;                      // per panel {sum v^2, sum remainder^2}
  };
  std::vector<RuleDev> rd;
  __nv_bfloat16* pw[3] = {nullptr, nullptr, nullptr};   // panel words (panel x ldb each)
  double* p64 = nullptr;                // FP64 path: generated row panel (column-major, panel x n)
  double* part = nullptr;               // per (item, warp) partials of one generation launch
  bool tuning = false;                  // holds a pass the autotuner still has to time
};

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
std::function<rsvd_status()> make_mm(Job& J, MMKind kind, std::vector<MMDesc> md);
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
               std::function<int(int)> splits, std::function<const int*(int)> cond = nullptr) {
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

void add_chol(Job& J, int accumulate, int f32_chol = 0) {
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

// ---------------------------------------------------------------- FP64 path
// CholeskyQR2 of src (n x l, FP64) using tmp; result back in src.
void cqr2_f64(Job& J, std::function<double*(int)> src, std::function<double*(int)> tmp, bool acc_R) {
  for (int round = 0; round < 2; ++round) {
    auto in = round == 0 ? src : tmp;
    auto out = round == 0 ? tmp : src;
    add_tn(J, MMK_GRAM_F64, [&](int c) { return (const void*)in(c); }, [&](int c) { return (const void*)in(c); },
           [&](int c) { return J.ch[c].G; }, [&](int c) { return J.d[c].l; }, [&](int c) { return J.d[c].l; },
           true);
    add_chol(J, (acc_R && round == 1) ? 1 : 0);
    std::vector<MMDesc> md(J.C);
    for (int c = 0; c < J.C; ++c) {
      const ChanDims& d = J.d[c];
      MMDesc m{};
      m.A = in(c); m.lda = d.ldt;
      m.B = J.ch[c].Ri; m.ldb = d.l;
      m.Cm = out(c); m.ldc = d.ldt;
      m.m = d.n; m.n = d.l; m.k = d.l;
      m.mt = cdiv(d.n, 64); m.nt = cdiv(d.l, 64); m.ks = 1; m.kchunk = (int)rup(d.l, 16);
      m.mode = MM_STORE;
      md[c] = m;
    }
    add_mm(J, MMK_NN_F64, md);
  }
  // Conditional third round for the channels whose Cholesky needed the shift
  // (shifted CholeskyQR3, Fukaya et al. 2020): the shifted factor leaves Q
  // orthonormal only to about kappa(Y)^2 u, one more round restores it (and
  // accumulates its factor into R).  Other channels skip every launch at its
  // first instruction.
  auto flags = [&](int c) {
    return (const int*)((uintptr_t)J.ch[c].res + offsetof(ChanResult, flags));
  };
  add_tn_ex(J, MMK_GRAM_F64, [&](int c) { return (const void*)src(c); }, [&](int c) { return (const void*)src(c); },
            [&](int c) { return J.ch[c].G; }, [&](int c) { return J.d[c].l; }, [&](int c) { return J.d[c].l; }, true,
            [&](int c) { return J.d[c].n; }, [&](int c) { return J.d[c].ldt; },
            [&](int c) { return J.d[c].gsplit; }, flags);
  {
    const Chan* dch = J.d_ch;
    const int maxl = J.max_l;
    cudaStream_t st = J.P->st;
    const std::vector<int> ls = chan_ls(J);
    int* coop = J.P->d_coop;
    int* derr_w = J.P->d_err;
    const int acc = acc_R ? 1 : 0;
    J.steps.push_back([=]() {
      run_chol(dch, ls, acc, maxl, 0, 0, 1, coop, derr_w, st);
      return RSVD_OK;
    });
  }
  std::vector<MMDesc> md(J.C);
  std::vector<CopyDesc> cd(J.C);
  for (int c = 0; c < J.C; ++c) {
    const ChanDims& d = J.d[c];
    MMDesc m{};
    m.A = src(c); m.lda = d.ldt;
    m.B = J.ch[c].Ri; m.ldb = d.l;
    m.Cm = tmp(c); m.ldc = d.ldt;
    m.m = d.n; m.n = d.l; m.k = d.l;
    m.mt = cdiv(d.n, 64); m.nt = cdiv(d.l, 64); m.ks = 1; m.kchunk = (int)rup(d.l, 16);
    m.mode = MM_STORE;
    m.cond = flags(c);
    md[c] = m;
    cd[c] = CopyDesc{tmp(c), src(c), (int64_t)d.ldt * d.l, flags(c)};
  }
  add_mm(J, MMK_NN_F64, md);
  const CopyDesc* dcd = J.ar.put(cd.data(), cd.size());
  const int C = J.C;
  cudaStream_t st = J.P->st;
  J.steps.push_back([=]() {
    launch_copy64_if_shifted(dcd, C, st);
    return RSVD_OK;
  });
}

// Y_c = V_c X_c (dense FP64), split over k with atomic accumulation when the
// batch has too few output tiles to fill the GPU.  Autotuned: the split target
// (1, 2 or 4 tiles per SM, or none) and the shortest split (64 or 128 rows).
void dense_f64(Job& J, std::function<const double*(int)> X, std::function<double*(int)> Y) {
  int64_t tiles = 0;
  for (int c = 0; c < J.C; ++c) tiles += (int64_t)cdiv(J.d[c].n, 64) * cdiv(J.d[c].l, 64);
  struct Cfg { int target, min_chunk; };
  const Cfg all[] = {{2, 128}, {1, 128}, {4, 128}, {4, 64}, {0, 128}};
  auto ks_of = [&](const Cfg& g, int c) {
    const int n = J.d[c].n;
    int ks = pick_splits(tiles, n, g.min_chunk, (int64_t)g.target * NSM);
    const int kchunk = (int)rup(cdiv(n, ks), 16);
    return std::make_pair(cdiv(n, kchunk), kchunk);
  };
  // distinct candidates (by the splits they give every channel)
  std::vector<Cfg> cands;
  std::vector<std::vector<int>> sigs;
  for (const Cfg& g : all) {
    std::vector<int> sg(J.C);
    for (int c = 0; c < J.C; ++c) sg[c] = ks_of(g, c).first;
    if (std::find(sigs.begin(), sigs.end(), sg) == sigs.end()) {
      sigs.push_back(sg);
      cands.push_back(g);
    }
  }
  std::vector<int64_t> per;
  for (int c = 0; c < J.C; ++c) { per.push_back(J.d[c].n); per.push_back(J.d[c].l); }
  const std::string key = tune_key("f64", {}, per);
  std::vector<std::function<rsvd_status()>> vars;
  std::vector<rsvd_tune_record> recs;
  for (int ci : tune_pick(J, key, cands.size())) {
    const Cfg g = cands[ci];
    std::vector<MMDesc> md(J.C);
    std::vector<ZeroDesc> zd(J.C);
    bool any_split = false;
    for (int c = 0; c < J.C; ++c) {
      const ChanDims& d = J.d[c];
      MMDesc m{};
      m.A = J.ch[c].A; m.lda = J.ch[c].lda;
      m.B = X(c); m.ldb = d.ldt;
      m.Cm = Y(c); m.ldc = d.ldt;
      m.m = d.n; m.n = d.l; m.k = d.n;
      m.mt = cdiv(d.n, 64); m.nt = cdiv(d.l, 64);
      const auto kk = ks_of(g, c);
      m.ks = kk.first;
      m.kchunk = kk.second;
      m.mode = m.ks > 1 ? MM_ATOMIC : MM_STORE;
      any_split |= m.ks > 1;
      md[c] = m;
      zd[c] = ZeroDesc{Y(c), d.ldt, d.n, d.l, 8};
    }
    std::function<rsvd_status()> zero;
    if (any_split) {
      const int* off = offsets(J, [&](int c) { return (int64_t)cdiv(J.d[c].n, 64); });
      const int tiles64 = total_of(J, [&](int c) { return (int64_t)cdiv(J.d[c].n, 64); });
      const ZeroDesc* dzd = J.ar.put(zd.data(), zd.size());
      cudaStream_t st = J.P->st;
      const int C = J.C;
      zero = [=]() {
        launch_zero(dzd, off, C, tiles64, st);
        return RSVD_OK;
      };
    }
    auto mm = make_mm(J, MMK_DENSE_F64, md);
    vars.push_back([=]() {
      if (zero) zero();
      return mm();
    });
    rsvd_tune_record r{};
    r.kind = RSVD_TUNE_DENSE_F64;
    r.bn = 64;
    r.split_target = g.target * NSM;
    r.min_split = g.min_chunk;
    recs.push_back(r);
  }
  add_tuned(J, key, recs, vars);
}

void lift(Job& J, MMKind kind, std::function<const void*(int)> basis, std::function<const void*(int)> small,
          std::function<double*(int)> out, std::function<int64_t(int)> ldo, std::function<const double*(int)> scale) {
  std::vector<MMDesc> md(J.C);
  for (int c = 0; c < J.C; ++c) {
    const ChanDims& d = J.d[c];
    MMDesc m{};
    m.A = basis(c); m.lda = d.ldt;
    m.B = small(c); m.ldb = d.l;
    m.Cm = out(c); m.ldc = ldo(c);
    m.m = d.n; m.n = d.kcap; m.k = d.l;
    m.mt = cdiv(d.n, 64); m.nt = cdiv(d.kcap, 64); m.ks = 1; m.kchunk = (int)rup(d.l, 16);
    m.mode = MM_STORE;
    m.colscale = scale(c);
    m.ncols_dev = &J.d_res[c].k_out;
    md[c] = m;
  }
  add_mm(J, kind, md);
}

// FP64 path, tile rule: one pass Y = V X generates V row panel by row panel
// in FP64 -- panel = H_rows H^T (H_jm = sqrt(w_m) g_m(x_j), FP64), plus the
// hash noise -- and multiplies it by X (FP64 CUDA cores throughout; 2M flops
// per generated entry).  `first` also sums ||V||^2 into the channel result.
std::vector<RuleDesc64> rule_descs64(Job& J) {
  std::vector<RuleDesc64> rds(J.C);
  for (int c = 0; c < J.C; ++c) {
    const rsvd_matrix& A = J.A[c];
    const int M = A.rule_m;
    RuleDesc64 r{};
    r.n = J.d[c].n; r.M = M;
    r.c = J.ar.put(A.rule_c, M);
    r.s = J.ar.put(A.rule_s, M);
    r.w = J.ar.put(A.rule_w, M);
    r.H = J.rd[c].H64;
    r.ldh = J.rd[c].ldh;
    rds[c] = r;
  }
  return rds;
}

void rule_pass64(Job& J, std::function<const double*(int)> X, std::function<double*(int)> Y, bool first) {
  cudaStream_t st = J.P->st;
  for (int c = 0; c < J.C; ++c) {
    const ChanDims& d = J.d[c];
    const Job::RuleDev r = J.rd[c];
    const int Pr = std::min<int>(J.panel, (int)rup(d.n, 128));
    const int np = cdiv(d.n, Pr);
    const double amp3 = J.A[c].rule_eta * 1.7320508075688772;
    for (int p = 0; p < np; ++p) {
      const int r0 = p * Pr, rows = std::min(Pr, d.n - r0);
      MMDesc g{};
      g.A = r.H64 + (int64_t)r0 * r.ldh; g.lda = r.ldh;
      g.B = r.H64; g.ldb = r.ldh;
      g.Cm = J.p64; g.ldc = Pr;
      g.m = rows; g.n = d.n; g.k = r.M;
      g.ks = 1; g.kchunk = (int)rup(r.M, 16);
      g.mode = MM_STORE;
      J.steps.push_back(make_mm(J, MMK_DENSE_F64, {g}));
      double* p64 = J.p64;
      double* part = J.part;
      double* psum = r.psums + 2 * p;
      const uint32_t key = r.key;
      const int n = d.n, ldp = Pr;
      J.steps.push_back([=]() {
        launch_rule_noise64(p64, ldp, rows, n, r0, key, amp3, first ? part : nullptr, st);
        if (first) launch_rule_part_sum(part, kRuleNoiseBlocks, psum, st);
        return RSVD_OK;
      });
      MMDesc t{};
      t.A = J.p64; t.lda = Pr;
      t.B = X(c); t.ldb = d.ldt;
      t.Cm = Y(c) + r0; t.ldc = d.ldt;
      t.m = rows; t.n = d.l; t.k = d.n;
      t.ks = 1; t.kchunk = (int)rup(d.n, 16);
      t.mode = MM_STORE;
      J.steps.push_back(make_mm(J, MMK_NN_F64, {t}));
    }
    if (first) {
      ChanResult* res = J.ch[c].res;
      const double* ps = r.psums;
      J.steps.push_back([=]() {
        launch_rule_finish(ps, np, res, st);
        return RSVD_OK;
      });
    }
  }
}

// One FP64 pass over V: the stored matrix, or the generated tile rule.
void pass64(Job& J, std::function<const double*(int)> X, std::function<double*(int)> Y, bool first) {
  if (J.rule) rule_pass64(J, X, Y, first);
  else dense_f64(J, X, Y);
}

void build_fp64(Job& J) {
  auto& ch = J.ch;
  const int C = J.C;
  cudaStream_t st = J.P->st;
  const Chan* dch = J.d_ch;
  const int* off64 = offsets(J, [&](int c) { return (int64_t)cdiv(J.d[c].n, 64); });
  const int t64 = total_of(J, [&](int c) { return (int64_t)cdiv(J.d[c].n, 64); });
  const uint64_t seed = J.P->o.seed;
  if (J.rule) {
    // tile rules: the FP64 factor panel; ||V||^2 comes with the first pass
    const std::vector<RuleDesc64> rds = rule_descs64(J);
    J.steps.push_back([=]() {
      for (const RuleDesc64& r : rds) launch_rule_prep64(r, st);
      launch_omega_f64(dch, off64, C, t64, seed, 0, st);
      return RSVD_OK;
    });
  } else {
    J.steps.push_back([=]() {
      launch_fro2(dch, off64, C, t64, st);
      launch_fro2_reduce(dch, C, st);
      launch_omega_f64(dch, off64, C, t64, seed, 0, st);
      return RSVD_OK;
    });
  }
  auto X = [&](int c) { return ch[c].X; };
  auto Y = [&](int c) { return ch[c].Y; };
  auto Q2 = [&](int c) { return ch[c].Q2; };
  pass64(J, [&](int c) { return (const double*)ch[c].X; }, Y, true);     // Y = V P
  cqr2_f64(J, Y, X, false);                                              // Q in Y
  bool q_in_y = true;
  for (int r = 0; r < 2 * J.q; ++r) {
    if (q_in_y) { pass64(J, [&](int c) { return (const double*)ch[c].Y; }, X, false); cqr2_f64(J, X, Q2, false); }
    else { pass64(J, [&](int c) { return (const double*)ch[c].X; }, Y, false); cqr2_f64(J, Y, Q2, false); }
    q_in_y = !q_in_y;
  }
  auto Qb = [&, q_in_y](int c) { return q_in_y ? ch[c].Y : ch[c].X; };
  auto Wb = [&, q_in_y](int c) { return q_in_y ? ch[c].X : ch[c].Y; };
  pass64(J, [&](int c) { return (const double*)Qb(c); }, Wb, false);     // W = V Q
  const bool rr = J.P->o.rayleigh_ritz != 0;
  if (rr) {
    // T = Q^T W into R (symmetric); Jacobi SVD of T gives T = X Sigma J^T
    add_tn(J, MMK_GRAM_F64, [&](int c) { return (const void*)Qb(c); }, [&](int c) { return (const void*)Wb(c); },
           [&](int c) { return ch[c].R; }, [&](int c) { return J.d[c].l; }, [&](int c) { return J.d[c].l; },
           false);
  } else {
    cqr2_f64(J, Wb, Q2, true);                                            // W = Q2 R, Q2 in Wb
  }
  const int maxl = J.max_l;
  const int policy = J.policy;
  const double tol = J.tol;
  std::vector<int> ls(C);
  for (int c = 0; c < C; ++c) ls[c] = J.d[c].l;
  int* coop = J.P->d_coop;
  int* derr_w = J.P->d_err;
  J.steps.push_back([=]() {
    run_jacobi(dch, ls, 0, maxl, coop, derr_w, st);
    launch_select(dch, C, policy, tol, 0, st);
    return RSVD_OK;
  });
  lift(J, MMK_NN_F64, [&](int c) { return (const void*)Qb(c); }, [&](int c) { return (const double*)ch[c].M; },
       [&](int c) { return ch[c].U; }, [&](int c) { return ch[c].ldu; }, [&](int c) { return (const double*)nullptr; });
  lift(J, MMK_NN_F64, [&, rr](int c) { return (const void*)(rr ? Qb(c) : Wb(c)); },
       [&](int c) { return (const double*)ch[c].J; }, [&](int c) { return ch[c].V; },
       [&](int c) { return ch[c].ldv; }, [&](int c) { return (const double*)nullptr; });
  const int maxk = J.max_kcap;
  J.steps.push_back([=]() {
    launch_signfix(dch, C, maxk, st);
    return RSVD_OK;
  });
}

// --------------------------------------------------------------- mixed path
rsvd_status tc_pass_ex(Job& J, int sa, int sx, std::function<int(int)> ncols_of,
                       std::function<const __nv_bfloat16*(int, int)> xword, std::function<float*(int)> yout) {
  // one grouped tcgen05 launch: Y[:, 0:ncols) = sum words V_a X_b.
  // Default shape: all columns in one tile up to the kernel's register
  // accumulator width (TC_BN_NARROW), else balanced column tiles; k split only when
  // the batch has fewer than two items per SM; as many pipeline stages as
  // shared memory holds; items longest channel first.  Autotuned: one or two
  // more column tiles, the split target (4 items per SM with shorter splits,
  // or none), a 4-stage pipeline, and the plain channel order.
  int maxnc = 16;
  std::vector<int> nc_of(J.C);
  for (int c = 0; c < J.C; ++c) {
    nc_of[c] = ncols_of(c);
    maxnc = std::max(maxnc, nc_of[c]);
  }
  struct Cfg { int bn, target, min_chunk, stages, lpt; };
  std::vector<Cfg> cands;
  {
    const int nt0 = cdiv(maxnc, TC_BN_NARROW);
    std::vector<int> bns;
    for (int nt : {nt0, nt0 + 1, 2 * nt0}) {
      const int bn = (int)rup(cdiv(maxnc, nt), 16);
      if ((nt == nt0 || bn >= 32) && std::find(bns.begin(), bns.end(), bn) == bns.end()) bns.push_back(bn);
    }
    const int splits[3][2] = {{2, 8}, {4, 4}, {0, 8}};
    for (int bn : bns)
      for (const auto& sp : splits)
        for (int stg : {0, 4}) cands.push_back({bn, sp[0], sp[1], stg, 1});
    cands.push_back({bns[0], 2, 8, 0, 0});
  }
  auto ks_of = [&](const Cfg& g, int c) {
    int64_t items0 = 0;
    for (int e = 0; e < J.C; ++e) items0 += (int64_t)cdiv(J.d[e].n, 128) * cdiv(nc_of[e], g.bn);
    const int kt = cdiv(J.d[c].n, 64);
    const int ks = pick_splits(items0, kt, g.min_chunk, (int64_t)g.target * NSM);
    const int kps = cdiv(kt, ks);
    return std::make_pair(cdiv(kt, kps), kps);
  };
  {
    // drop candidates that give the same launch as an earlier one
    std::vector<Cfg> uniq;
    std::vector<std::vector<int>> sigs;
    for (const Cfg& g : cands) {
      std::vector<int> sg = {g.bn, std::min(g.stages ? g.stages : 99, tc_stages(sa, sx, g.bn)), g.lpt};
      for (int c = 0; c < J.C; ++c) sg.push_back(ks_of(g, c).first);
      if (std::find(sigs.begin(), sigs.end(), sg) == sigs.end()) {
        sigs.push_back(sg);
        uniq.push_back(g);
      }
    }
    cands.swap(uniq);
  }
  std::vector<int64_t> per;
  for (int c = 0; c < J.C; ++c) { per.push_back(J.d[c].n); per.push_back(nc_of[c]); }
  const std::string key = tune_key("tc", {sa, sx}, per);
  std::vector<std::function<rsvd_status()>> vars;
  std::vector<rsvd_tune_record> recs;
  for (int ci : tune_pick(J, key, cands.size())) {
    const Cfg g = cands[ci];
    const int bn = g.bn;
    std::vector<TcChan> tcs(J.C);
    bool any_split = false;
    std::vector<ZeroDesc> zd(J.C);
    int item = 0;
    // items numbered longest first: the persistent CTAs take items
    // round-robin, so this order balances them (longest-processing-time-first)
    std::vector<int> order(J.C);
    for (int c = 0; c < J.C; ++c) order[c] = c;
    if (g.lpt) std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return J.d[a].n > J.d[b].n; });
    for (int pos = 0; pos < J.C; ++pos) {
      const int c = order[pos];
      const ChanDims& d = J.d[c];
      const int nc = nc_of[c];
      TcChan& t = tcs[pos];
      memset(&t, 0, sizeof(t));
      const void* A[3] = {J.ch[c].Ab[0], J.ch[c].Ab[1], J.ch[c].Ab[2]};
      const void* X[3] = {xword(c, 0), xword(c, 1), xword(c, 2)};
      if (!J.measure) {
        const int e = tc_encode(&t, A, sa, d.ldb, X, sx, d.ldb, d.n, d.n, nc, bn);
        if (e) return seterr(RSVD_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", e);
      }
      t.Y = yout(c);
      t.ldy = d.ldt;
      t.n = d.n;
      t.m = d.n;
      t.mode = TC_STORE;
      t.ncols = nc;
      t.mt = cdiv(d.n, 128);
      t.nt = cdiv(nc, bn);
      const auto kk = ks_of(g, c);
      t.ks = kk.first;
      t.kt_per_split = kk.second;
      t.atomic = t.ks > 1;
      any_split |= t.atomic != 0;
      t.item0 = item;
      item += t.mt * t.nt * t.ks;
      zd[c] = ZeroDesc{t.Y, d.ldt, d.n, nc, 4};
    }
    const int items = item;
    std::function<rsvd_status()> zero;
    if (any_split) {
      const int* off = offsets(J, [&](int c) { return (int64_t)cdiv(J.d[c].n, 64); });
      const int tiles64 = total_of(J, [&](int c) { return (int64_t)cdiv(J.d[c].n, 64); });
      const ZeroDesc* dzd = J.ar.put(zd.data(), zd.size());
      cudaStream_t st = J.P->st;
      const int C = J.C;
      zero = [=]() {
        launch_zero(dzd, off, C, tiles64, st);
        return RSVD_OK;
      };
    }
    const TcChan* dtc = J.ar.put(tcs.data(), tcs.size(), 128);
    cudaStream_t st = J.P->st;
    int* derr = J.P->d_err;
    const int C = J.C;
    // algorithmic traffic: every V word, X word and Y element once; MMA flops
    double bytes = 0.0, flops = 0.0;
    int npairs = 0;
    for (int a = 0; a < sa; ++a)
      for (int x = 0; x < sx; ++x) npairs += (a + x < std::max(sa, sx));
    for (int c = 0; c < J.C; ++c) {
      const double n = J.d[c].n, nc = nc_of[c];
      bytes += n * n * 2.0 * sa + n * nc * 2.0 * sx + n * nc * 4.0;
      flops += 2.0 * n * n * nc * npairs;
    }
    rsvd_plan_s* P = J.P;
    const int stages = g.stages;
    vars.push_back([=]() {
      if (zero) zero();
      cudaEvent_t ea = nullptr, eb = nullptr;
      if (P->profiling) timed_begin(P, &ea, &eb);
      const int e = tc_launch(dtc, C, items, sa, sx, bn, derr, st, false, stages);
      if (e) return seterr(RSVD_ERR_CUDA, "tcgen05 GEMM launch failed: %s", cudaGetErrorString((cudaError_t)e));
      if (P->profiling) {
        cudaEventRecord(eb, st);
        P->pending.push_back({ea, eb, 0, bytes, flops});
      }
      return RSVD_OK;
    });
    rsvd_tune_record r{};
    r.kind = RSVD_TUNE_TC;
    r.bn = bn;
    r.split_target = g.target * NSM;
    r.min_split = g.min_chunk * 64;
    r.stages = std::min(g.stages ? g.stages : 99, tc_stages(sa, sx, bn));
    r.order = g.lpt;
    recs.push_back(r);
  }
  add_tuned(J, key, recs, vars);
  return RSVD_OK;
}

rsvd_status tc_pass(Job& J, int sa, int sx, int ncols_of_pass /*0: l, 1: lw*/) {
  return tc_pass_ex(
      J, sa, sx, [&](int c) { return ncols_of_pass ? J.d[c].lw : J.d[c].l; },
      [&](int c, int w) { return (const __nv_bfloat16*)J.ch[c].Xb[w]; }, [&](int c) { return J.ch[c].Y32; });
}

// One pass Y = A X over tile-rule channels.  Per channel and row panel: a
// generation launch (H H_panel^T on the tensor core, plus the noise, split
// into the panel's BF16 words) and a product launch (panel words x X words
// -> the panel's rows of Y).  A is symmetric, so the generated block, stored
// with the matrix column index fastest, is exactly the row panel the product
// reads.  `first`: also reduce the entry energies into fro2 and wres2.
rsvd_status rule_pass(Job& J, int sx, std::function<int(int)> ncols_of,
                      std::function<const __nv_bfloat16*(int, int)> xword, std::function<float*(int)> yout,
                      bool first) {
  const int nsl = J.nsl;
  rsvd_plan_s* P = J.P;
  cudaStream_t st = P->st;
  int* derr = P->d_err;
  for (int c = 0; c < J.C; ++c) {
    const ChanDims& d = J.d[c];
    const Job::RuleDev r = J.rd[c];
    const int Pr = std::min<int>(J.panel, (int)rup(d.n, 128));
    const int np = cdiv(d.n, Pr);
    const int nc = ncols_of(c);
    const bool wide = (nsl == 2 && sx == 2) || (nsl == 3 && sx == 3);   // the wide instantiations
    const int ntile = cdiv(std::max(nc, 16), wide ? TC_BN_MAX : TC_BN_NARROW);
    const int bn = (int)rup(cdiv(std::max(nc, 16), ntile), 16);
    for (int p = 0; p < np; ++p) {
      const int r0 = p * Pr, rows = std::min(Pr, d.n - r0);
      const int gbn = std::min(128, (int)rup(rows, 16));
      TcChan g, t;
      memset(&g, 0, sizeof(g));
      memset(&t, 0, sizeof(t));
      if (!J.measure) {
        const void* HA[2] = {r.H[0], r.H[1]};
        const void* HX[2] = {r.H[0] + (int64_t)r0 * r.ldh, r.H[1] + (int64_t)r0 * r.ldh};
        int e = tc_encode(&g, HA, 2, r.ldh, HX, 2, r.ldh, d.n, r.M, rows, gbn, 1);
        if (e) return seterr(RSVD_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", e);
        const void* PA[3] = {J.pw[0], J.pw[1], J.pw[2]};
        const void* X[3] = {xword(c, 0), xword(c, 1), xword(c, 2)};
        e = tc_encode(&t, PA, nsl, d.ldb, X, sx, d.ldb, rows, d.n, nc, bn);
        if (e) return seterr(RSVD_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", e);
      }
      g.n = r.M; g.m = d.n; g.ncols = rows;
      g.mt = cdiv(d.n, 128); g.nt = cdiv(rows, gbn); g.ks = 1; g.kt_per_split = cdiv(r.M, 64);
      g.mode = TC_RULE;
      // each 64-wide k step accumulated from zero, the chunk sums added to
      // nearest: longer chunks let the tensor core's truncating accumulation
      // bias the entries measurably (two steps per chunk raised the exact
      // residual of the n = 200,000 rule from 1.6e-6 to 2.0e-6)
      g.chunk_kt = 1;
      for (int w = 0; w < nsl; ++w) g.W[w] = J.pw[w];
      g.ldw = d.ldb; g.nw = nsl; g.r0 = r0;
      g.eta_key = r.key; g.eta_amp3 = r.amp3;
      g.hinv = (float)(1.0 / r.hscale);
      g.part = first ? J.part : nullptr;
      t.Y = yout(c) + r0; t.ldy = d.ldt;
      t.n = d.n; t.m = rows; t.ncols = nc;
      t.mt = cdiv(rows, 128); t.nt = cdiv(nc, bn);
      {
        // the panel has few output tiles (rows / 128 x 2-3) and a long k
        // extent (n): split k so the persistent CTAs get ~4 items each
        const int kt = cdiv(d.n, 64);
        const int ks = pick_splits((int64_t)t.mt * t.nt, kt, 8, 4 * NSM);
        t.kt_per_split = cdiv(kt, ks);
        t.ks = cdiv(kt, t.kt_per_split);
        t.atomic = t.ks > 1;
      }
      t.mode = TC_STORE;
      const int gitems = g.mt * g.nt, titems = t.mt * t.nt * t.ks;
      const TcChan* dg = J.ar.put(&g, 1, 128);
      const TcChan* dt = J.ar.put(&t, 1, 128);
      const ZeroDesc zd{t.Y, d.ldt, rows, nc, 4};
      const ZeroDesc* dzd = t.atomic ? J.ar.put(&zd, 1) : nullptr;
      const int zoff[2] = {0, cdiv(rows, 64)};
      const int* dzoff = t.atomic ? J.ar.put(zoff, 2) : nullptr;
      const int ztiles = zoff[1];
      const double gflops = 2.0 * d.n * (double)rows * r.M;                // algorithmic
      const double gmma = 2.0 * d.n * (double)rows * r.ldh * 3;            // issued word products
      double tpairs = 0;
      for (int a = 0; a < nsl; ++a)
        for (int x = 0; x < sx; ++x) tpairs += (a + x < std::max(nsl, sx));
      const double tbytes = (double)rows * d.n * 2.0 * nsl + (double)d.n * nc * 2.0 * sx + (double)rows * nc * 4.0;
      const double tflops = 2.0 * rows * (double)d.n * nc * tpairs;
      double* part = J.part;
      double* psum = r.psums + 2 * p;
      J.steps.push_back([=]() {
        cudaEvent_t ea = nullptr, eb = nullptr;
        if (P->profiling) timed_begin(P, &ea, &eb);
        int e = tc_launch(dg, 1, gitems, 2, 2, gbn, derr, st, true);
        if (e) return seterr(RSVD_ERR_CUDA, "tile-rule generation launch failed: %s", cudaGetErrorString((cudaError_t)e));
        if (P->profiling) {
          cudaEventRecord(eb, st);
          P->pending.push_back({ea, eb, 2, gmma, gflops});
        }
        if (first) launch_rule_part_sum(part, gitems * 4, psum, st);
        if (dzd) launch_zero(dzd, dzoff, 1, ztiles, st);     // the k splits accumulate into Y
        if (P->profiling) timed_begin(P, &ea, &eb);
        e = tc_launch(dt, 1, titems, nsl, sx, bn, derr, st);
        if (e) return seterr(RSVD_ERR_CUDA, "tcgen05 GEMM launch failed: %s", cudaGetErrorString((cudaError_t)e));
        if (P->profiling) {
          cudaEventRecord(eb, st);
          P->pending.push_back({ea, eb, 0, tbytes, tflops});
        }
        return RSVD_OK;
      });
    }
    if (first) {
      ChanResult* res = J.ch[c].res;
      const double* ps = r.psums;
      J.steps.push_back([=]() {
        launch_rule_finish(ps, np, res, st);
        return RSVD_OK;
      });
    }
  }
  return RSVD_OK;
}

// One pass over V (dense words) or over the generated rule entries.
rsvd_status pass_over(Job& J, int sa, int sx, int ncols_of_pass, bool first) {
  auto ncols = [&](int c) { return ncols_of_pass ? J.d[c].lw : J.d[c].l; };
  auto xw = [&](int c, int w) { return (const __nv_bfloat16*)J.ch[c].Xb[w]; };
  auto y = [&](int c) { return J.ch[c].Y32; };
  if (J.rule) return rule_pass(J, sx, ncols, xw, y, first);
  return tc_pass_ex(J, sa, sx, ncols, xw, y);
}

// The register Cholesky (l <= 128) also leaves an FP32 copy of R^{-1} in
// Ri32 where the job has that buffer; the triangular solves then read FP32
// operands only (the cp.async tile kernel).
bool ri32_ok(const Job& J) {
  if (J.max_l > 128) return false;
  for (int c = 0; c < J.C; ++c)
    if (!J.ch[c].Ri32) return false;
  return true;
}

// FP32 copy of a small per-channel FP64 operand into Ri32 (count <= l * l).
void add_cvt_f32(Job& J, std::function<const double*(int)> src, std::function<int64_t(int)> count) {
  std::vector<CvtDesc> cd(J.C);
  int64_t mx = 0;
  for (int c = 0; c < J.C; ++c) {
    cd[c] = CvtDesc{src(c), J.ch[c].Ri32, count(c)};
    mx = std::max(mx, cd[c].count);
  }
  const CvtDesc* dcd = J.ar.put(cd.data(), cd.size());
  const int C = J.C;
  cudaStream_t st = J.P->st;
  J.steps.push_back([=]() {
    launch_cvt_f32(dcd, C, mx, st);
    return RSVD_OK;
  });
}

// CholeskyQR2 of Y32[:, 0:l) -> Q32 (FP32) and its BF16 words in Xb[:, 0:l).
void cqr2_mixed(Job& J, int nsl_out) {
  auto& ch = J.ch;
  for (int round = 0; round < 2; ++round) {
    auto in = [&, round](int c) { return round == 0 ? ch[c].Y32 : ch[c].T32; };
    auto out = [&, round](int c) { return round == 0 ? ch[c].T32 : ch[c].Q32; };
    // round 0: Y has kappa up to ~1e5, so the Gram needs FP64-grade accuracy
    // (compensated Dot2); round 1: Q1 is orthonormal to ~1e-2, a plain FP32
    // Gram is accurate enough
    add_tn(J, round == 0 ? MMK_GRAM_DOT2 : MMK_GRAM_F32, [&](int c) { return (const void*)in(c); },
           [&](int c) { return (const void*)in(c); }, [&](int c) { return ch[c].G; },
           [&](int c) { return J.d[c].l; }, [&](int c) { return J.d[c].l; }, true);
    add_chol(J, 0, round == 1 ? 1 : 0);
    const bool b32 = ri32_ok(J);
    std::vector<MMDesc> md(J.C);
    for (int c = 0; c < J.C; ++c) {
      const ChanDims& d = J.d[c];
      MMDesc m{};
      m.A = in(c); m.lda = d.ldt;
      m.B = b32 ? (const void*)ch[c].Ri32 : (const void*)ch[c].Ri; m.ldb = d.l;
      m.Cm = out(c); m.ldc = d.ldt;
      m.m = d.n; m.n = d.l; m.k = d.l;
      m.mt = cdiv(d.n, 64); m.nt = cdiv(d.l, 64); m.ks = 1; m.kchunk = (int)rup(d.l, 16);
      m.mode = MM_STORE;
      if (round == 1) {
        for (int s = 0; s < nsl_out; ++s) m.sl[s] = ch[c].Xb[s];
        m.ldsl = d.ldb;
        m.nsl = nsl_out;
      }
      md[c] = m;
    }
    add_mm(J, b32 ? MMK_NN_F32 : MMK_NN_F32_F64B, md);
  }
  // Conditional third round, only for channels whose Cholesky needed the
  // shift: shifted CholeskyQR leaves Q orthonormal to about kappa(Y)^2 u only,
  // and one more round restores it (shifted CholeskyQR3; Fukaya, Kannan,
  // Nakatsukasa, Yamamoto and Yanagisawa, SIAM J. Sci. Comput. 42 (2020)).
  // Other channels skip every launch of the round at its first instruction.
  auto flags = [&](int c) {
    return (const int*)((uintptr_t)ch[c].res + offsetof(ChanResult, flags));
  };
  add_tn_ex(J, MMK_GRAM_DOT2, [&](int c) { return (const void*)ch[c].Q32; },
            [&](int c) { return (const void*)ch[c].Q32; }, [&](int c) { return ch[c].G; },
            [&](int c) { return J.d[c].l; }, [&](int c) { return J.d[c].l; }, true,
            [&](int c) { return J.d[c].n; }, [&](int c) { return J.d[c].ldt; },
            [&](int c) { return J.d[c].gsplit; }, flags);
  {
    const Chan* dch = J.d_ch;
    const int C = J.C, maxl = J.max_l;
    cudaStream_t st = J.P->st;
    const std::vector<int> ls = chan_ls(J);
    int* coop = J.P->d_coop;
  int* derr_w = J.P->d_err;
    J.steps.push_back([=]() {
      run_chol(dch, ls, 0, maxl, 1, 0, 1, coop, derr_w, st);
      return RSVD_OK;
    });
  }
  const bool b32 = ri32_ok(J);
  std::vector<MMDesc> md(J.C);
  for (int c = 0; c < J.C; ++c) {
    const ChanDims& d = J.d[c];
    MMDesc m{};
    m.A = ch[c].Q32; m.lda = d.ldt;
    m.B = b32 ? (const void*)ch[c].Ri32 : (const void*)ch[c].Ri; m.ldb = d.l;
    m.Cm = ch[c].T32; m.ldc = d.ldt;
    m.m = d.n; m.n = d.l; m.k = d.l;
    m.ks = 1; m.kchunk = (int)rup(d.l, 16);
    m.mode = MM_STORE;
    for (int w = 0; w < nsl_out; ++w) m.sl[w] = ch[c].Xb[w];
    m.ldsl = d.ldb;
    m.nsl = nsl_out;
    m.cond = flags(c);
    md[c] = m;
  }
  add_mm(J, b32 ? MMK_NN_F32 : MMK_NN_F32_F64B, md);
  {
    const Chan* dch = J.d_ch;
    const int C = J.C;
    cudaStream_t st = J.P->st;
    J.steps.push_back([=]() {
      launch_copy_t_to_q_if_shifted(dch, C, st);
      return RSVD_OK;
    });
  }
}

// FP64 CholeskyQR of the small SVD's left vectors X (l x l, in M).  The FP32
// Jacobi stops once every pair is orthogonal to l eps_32 (relative), so at
// large l or tight tolerances U = Q X is measurably not orthonormal and U U^T
// is not a projector.  X = X~ R with R upper triangular keeps
// span(X~_1..k) = span(X_1..k) for every k: the rank rule and the truncation
// see the same nested subspaces, now orthonormal to FP64 rounding.  The
// columns of X are already orthonormal to ~1e-4, so one round suffices and the
// Cholesky never needs its shift.  X~ lands in J (free on the FP32 path);
// the chain after it reads the returned table, whose M is that buffer.
Chan* reorth_x(Job& J) {
  std::vector<Chan> sw(J.ch);
  for (auto& h : sw) h.M = h.J;                     // Cholesky works in (and X~ lands in) J
  Chan* dsw = J.ar.put(sw.data(), sw.size(), 128);
  auto& ch = J.ch;
  if (ri32_ok(J)) {
    // l <= 128: the Jacobi left its columns M unnormalised in FP32 (X = M D).
    // G = D (M^T M) D with M^T M from the compensated (Dot2) Gram, FP32
    // Cholesky R^T R = G, and X~ = M D + M (D (R^{-1} - I)): FP64 where it
    // matters, the small correction as an FP32 product (no FP64 l^3 work).
    add_tn_ex(J, MMK_GRAM_DOT2, [&](int c) { return (const void*)ch[c].M; },
              [&](int c) { return (const void*)ch[c].M; }, [&](int c) { return ch[c].G; },
              [&](int c) { return J.d[c].l; }, [&](int c) { return J.d[c].l; }, true,
              [&](int c) { return J.d[c].l; }, [&](int c) { return (int64_t)J.d[c].l; }, [&](int) { return 1; });
    const int C = J.C, maxl = J.max_l;
    cudaStream_t st = J.P->st;
    const std::vector<int> ls = chan_ls(J);
    int* coop = J.P->d_coop;
  int* derr_w = J.P->d_err;
    const Chan* dch = J.d_ch;
    J.steps.push_back([=]() {
      launch_reorth(0, dch, C, maxl, st);              // G = D (M^T M) D
      run_chol(dsw, ls, 0, maxl, 0, 1, 0, coop, derr_w, st);  // X^T X ~ I: an FP32 factor is enough
      launch_reorth(1, dch, C, maxl, st);              // Ri32 = D (R^{-1} - I)
      return RSVD_OK;
    });
    std::vector<MMDesc> md(J.C);
    for (int c = 0; c < J.C; ++c) {
      const int l = J.d[c].l;
      MMDesc m{};
      m.A = ch[c].M; m.lda = l;                       // FP32 M
      m.B = ch[c].Ri32; m.ldb = l;
      m.Cm = ch[c].J; m.ldc = l;
      m.m = l; m.n = l; m.k = l;
      m.ks = 1; m.kchunk = (int)rup(l, 16);
      m.mode = MM_STORE;
      md[c] = m;
    }
    add_mm(J, MMK_NN_F32_OUT64_B32, md);
    J.steps.push_back([=]() {
      launch_reorth(2, dch, C, maxl, st);              // J += M D
      return RSVD_OK;
    });
    return dsw;
  }
  add_tn_ex(J, MMK_GRAM_F64, [&](int c) { return (const void*)ch[c].M; }, [&](int c) { return (const void*)ch[c].M; },
            [&](int c) { return ch[c].G; }, [&](int c) { return J.d[c].l; }, [&](int c) { return J.d[c].l; }, true,
            [&](int c) { return J.d[c].l; }, [&](int c) { return (int64_t)J.d[c].l; }, [&](int) { return 1; });
  {
    const int C = J.C, maxl = J.max_l;
    cudaStream_t st = J.P->st;
    const std::vector<int> ls = chan_ls(J);
    int* coop = J.P->d_coop;
  int* derr_w = J.P->d_err;
    J.steps.push_back([=]() {
      run_chol(dsw, ls, 0, maxl, 0, 1, 0, coop, derr_w, st);   // X^T X ~ I: an FP32 factor is enough
      return RSVD_OK;
    });
  }
  std::vector<MMDesc> md(J.C);
  for (int c = 0; c < J.C; ++c) {
    const int l = J.d[c].l;
    MMDesc m{};
    m.A = ch[c].M; m.lda = l;
    m.B = ch[c].Ri; m.ldb = l;
    m.Cm = ch[c].J; m.ldc = l;
    m.m = l; m.n = l; m.k = l;
    m.ks = 1; m.kchunk = (int)rup(l, 16);
    m.mode = MM_STORE;
    md[c] = m;
  }
  add_mm(J, MMK_NN_F64, md);
  return dsw;
}

// The factor panel H of each tile rule (its parameters travel in the
// descriptor region).
std::vector<RuleDesc> rule_descs(Job& J) {
  std::vector<RuleDesc> rds(J.C);
  for (int c = 0; c < J.C; ++c) {
    const rsvd_matrix& A = J.A[c];
    const int M = A.rule_m;
    RuleDesc r{};
    r.n = J.d[c].n; r.M = M;
    r.c = J.ar.put(A.rule_c, M);
    r.s = J.ar.put(A.rule_s, M);
    r.w = J.ar.put(A.rule_w, M);
    for (int w = 0; w < 2; ++w) r.H[w] = J.rd[c].H[w];
    r.ldh = J.rd[c].ldh;
    r.hscale = J.rd[c].hscale;
    rds[c] = r;
  }
  return rds;
}

rsvd_status build_mixed(Job& J, bool skip_convert = false) {
  auto& ch = J.ch;
  const int C = J.C;
  cudaStream_t st = J.P->st;
  const Chan* dch = J.d_ch;
  const int nsl = J.nsl;
  const int* off8 = offsets(J, [&](int c) { return (int64_t)cdiv(J.d[c].n, 8); });
  const int t8 = total_of(J, [&](int c) { return (int64_t)cdiv(J.d[c].n, 8); });
  const int* off64 = offsets(J, [&](int c) { return (int64_t)cdiv(J.d[c].n, 64); });
  const int t64 = total_of(J, [&](int c) { return (int64_t)cdiv(J.d[c].n, 64); });
  const uint64_t seed = J.P->o.seed;
  const uint64_t pseed = seed ^ 0x5DEECE66DULL;
  if (J.rule) {
    const std::vector<RuleDesc> rds = rule_descs(J);
    J.steps.push_back([=]() {
      for (const RuleDesc& r : rds) launch_rule_prep(r, st);
      launch_omega_bf16(dch, off64, C, t64, seed, 0, 0, 1 << 30, pseed, nsl, st);   // P and probes
      return RSVD_OK;
    });
  } else {
    // algorithmic traffic of the conversion: V read once (8 B), its words and
    // P's words written once
    double cbytes = 0.0;
    for (int c = 0; c < C; ++c)
      cbytes += (double)J.d[c].n * J.d[c].n * (8.0 + 2.0 * nsl) + (double)J.d[c].n * J.d[c].lw * 2.0 * nsl;
    rsvd_plan_s* P = J.P;
    J.steps.push_back([=]() {
      if (!skip_convert) {
        cudaEvent_t ea = nullptr, eb = nullptr;
        if (P->profiling) timed_begin(P, &ea, &eb);
        launch_convert_omega(dch, off8, t8, off64, t64, C, nsl, seed, pseed, nsl, st);   // words, P and probes
        if (P->profiling) {
          cudaEventRecord(eb, st);
          P->pending.push_back({ea, eb, 3, cbytes, 0.0});
        }
        launch_fro2_reduce_rows(dch, C, 8, st);
      } else {
        launch_fro2_reduce_rows(dch, C, 8, st);       // partials are kept from the probe job's conversion
        launch_omega_bf16(dch, off64, C, t64, seed, 0, 0, 1 << 30, pseed, nsl, st);   // P and probes
      }
      return RSVD_OK;
    });
  }
  // sketch: only the l sketch columns (X word 0 = P exactly)
  if (rsvd_status s = pass_over(J, nsl, 1, 0, true)) return s;
  cqr2_mixed(J, nsl);
  for (int r = 0; r < 2 * J.q; ++r) {
    if (rsvd_status s = pass_over(J, nsl, nsl, 0, false)) return s;
    cqr2_mixed(J, nsl);
  }
  // projection with the probe block: [W | V G] = V [Q | G]
  if (rsvd_status s = pass_over(J, nsl, nsl, 1, false)) return s;
  // C = Q^T (V G) (FP32 accumulate is ample for the error estimate)
  add_tn(J, MMK_GRAM_F32, [&](int c) { return (const void*)ch[c].Q32; },
         [&](int c) { return (const void*)(ch[c].Y32 + (int64_t)J.d[c].l * J.d[c].ldt); },
         [&](int c) { return ch[c].C64; }, [&](int c) { return J.d[c].l; }, [&](int c) { return J.d[c].s; }, false);
  // probe residual R = V G - Q C in place of V G, then its column energies
  {
    bool c32 = ri32_ok(J);                                  // C (l x s) must fit the l x l FP32 scratch
    for (int c = 0; c < J.C; ++c) c32 = c32 && J.d[c].s <= J.d[c].l;
    if (c32) add_cvt_f32(J, [&](int c) { return (const double*)ch[c].C64; },
                         [&](int c) { return (int64_t)J.d[c].l * J.d[c].s; });
    std::vector<MMDesc> md(J.C);
    std::vector<SumsqDesc> sd(J.C);
    for (int c = 0; c < J.C; ++c) {
      const ChanDims& d = J.d[c];
      float* VG = ch[c].Y32 + (int64_t)d.l * d.ldt;
      MMDesc m{};
      m.A = ch[c].Q32; m.lda = d.ldt;
      m.B = c32 ? (const void*)ch[c].Ri32 : (const void*)ch[c].C64; m.ldb = d.l;
      m.Cm = VG; m.ldc = d.ldt;
      m.m = d.n; m.n = d.s; m.k = d.l;
      m.ks = 1; m.kchunk = (int)rup(d.l, 16);
      m.mode = MM_SUB;
      md[c] = m;
      sd[c] = SumsqDesc{VG, d.ldt, d.n, d.s, 4, ch[c].est_part};
    }
    add_mm(J, c32 ? MMK_NN_F32 : MMK_NN_F32_F64B, md);
    const SumsqDesc* dsd = J.ar.put(sd.data(), sd.size());
    const int s_max = NPROBE;
    J.steps.push_back([=]() {
      launch_colsumsq(dsd, C, s_max, st);
      return RSVD_OK;
    });
  }
  const int maxl = J.max_l;
  // W^T W = R^T R
  add_tn(J, MMK_GRAM_DOT2, [&](int c) { return (const void*)ch[c].Y32; }, [&](int c) { return (const void*)ch[c].Y32; },
         [&](int c) { return ch[c].G; }, [&](int c) { return J.d[c].l; }, [&](int c) { return J.d[c].l; }, true);
  add_chol(J, 0);
  const int policy = J.policy;
  const double tol = J.tol;
  std::vector<int> ls(C);
  for (int c = 0; c < C; ++c) ls[c] = J.d[c].l;
  int* coop = J.P->d_coop;
  int* derr_w = J.P->d_err;
  J.steps.push_back([=]() {
    run_jacobi(dch, ls, 1, maxl, coop, derr_w, st);
    return RSVD_OK;
  });
  const Chan* dsw = reorth_x(J);                 // X~ in J
  J.steps.push_back([=]() {
    launch_probe_finish(dsw, C, maxl, st);
    launch_select(dsw, C, policy, tol, 1, st);
    return RSVD_OK;
  });
  // the lifts read X~ in FP32 (the FP32 basis bounds their accuracy anyway)
  const bool b32 = ri32_ok(J);
  if (b32) add_cvt_f32(J, [&](int c) { return (const double*)ch[c].J; }, [&](int c) { return (int64_t)J.d[c].l * J.d[c].l; });
  const MMKind lk = b32 ? MMK_NN_F32_OUT64_B32 : MMK_NN_F32_OUT64;
  auto xs = [&](int c) { return b32 ? (const void*)ch[c].Ri32 : (const void*)ch[c].J; };
  lift(J, lk, [&](int c) { return (const void*)ch[c].Q32; }, xs,
       [&](int c) { return ch[c].U; }, [&](int c) { return ch[c].ldu; }, [&](int c) { return (const double*)nullptr; });
  lift(J, lk, [&](int c) { return (const void*)ch[c].Y32; }, xs,
       [&](int c) { return ch[c].V; }, [&](int c) { return ch[c].ldv; }, [&](int c) { return (const double*)ch[c].scr; });
  const int maxk = J.max_kcap;
  J.steps.push_back([=]() {
    launch_signfix(dch, C, maxk, st);
    return RSVD_OK;
  });
  return RSVD_OK;
}

// ------------------------------------------------------------ probe job
// 16-column probe Y16 = V P16 (P16 from the Philox stream tag 1), its
// singular values, the rank-model features and (with weights) the network's
// predictions.  Mixed path: V is converted to its words here (the
// decomposition that follows reuses them) and the probe pass reads one word.
rsvd_status build_probe(Job& J, float* d_feat, const float* theta, float* d_pred) {
  auto& ch = J.ch;
  const int C = J.C;
  cudaStream_t st = J.P->st;
  const Chan* dch = J.d_ch;
  const uint64_t seed = J.P->o.seed;
  const double tol = J.tol;
  const int* off64 = offsets(J, [&](int c) { return (int64_t)cdiv(J.d[c].n, 64); });
  const int t64 = total_of(J, [&](int c) { return (int64_t)cdiv(J.d[c].n, 64); });
  if (J.mixed && J.rule) {
    // tile rules: the probe is one generated pass with 16 columns
    const std::vector<RuleDesc> rds = rule_descs(J);
    J.steps.push_back([=]() {
      for (const RuleDesc& r : rds) launch_rule_prep(r, st);
      launch_omega_bf16(dch, off64, C, t64, seed, 0, 0, 16, seed, 1, st, TAG_PROBE);
      return RSVD_OK;
    });
    if (rsvd_status s = pass_over(J, J.nsl, 1, 0, true)) return s;
    add_tn(J, MMK_GRAM_DOT2, [&](int c) { return (const void*)ch[c].Y32; },
           [&](int c) { return (const void*)ch[c].Y32; }, [&](int c) { return ch[c].G; },
           [&](int c) { return J.d[c].l; }, [&](int c) { return J.d[c].l; }, true);
  } else if (J.mixed) {
    const int* off8 = offsets(J, [&](int c) { return (int64_t)cdiv(J.d[c].n, 8); });
    const int t8 = total_of(J, [&](int c) { return (int64_t)cdiv(J.d[c].n, 8); });
    const int nsl = J.nsl;
    J.steps.push_back([=]() {
      launch_convert_slices(dch, off8, C, t8, nsl, st);
      launch_omega_bf16(dch, off64, C, t64, seed, 0, 0, 16, seed, 1, st, TAG_PROBE);
      return RSVD_OK;
    });
    if (rsvd_status s = tc_pass(J, 1, 1, 0)) return s;
    add_tn(J, MMK_GRAM_DOT2, [&](int c) { return (const void*)ch[c].Y32; },
           [&](int c) { return (const void*)ch[c].Y32; }, [&](int c) { return ch[c].G; },
           [&](int c) { return J.d[c].l; }, [&](int c) { return J.d[c].l; }, true);
  } else {
    if (J.rule) {
      const std::vector<RuleDesc64> rds = rule_descs64(J);
      J.steps.push_back([=]() {
        for (const RuleDesc64& r : rds) launch_rule_prep64(r, st);
        return RSVD_OK;
      });
    }
    J.steps.push_back([=]() {
      launch_omega_f64(dch, off64, C, t64, seed, 0, st, TAG_PROBE);
      return RSVD_OK;
    });
    pass64(J, [&](int c) { return (const double*)ch[c].X; }, [&](int c) { return ch[c].Y; }, true);
    add_tn(J, MMK_GRAM_F64, [&](int c) { return (const void*)ch[c].Y; },
           [&](int c) { return (const void*)ch[c].Y; }, [&](int c) { return ch[c].G; },
           [&](int c) { return J.d[c].l; }, [&](int c) { return J.d[c].l; }, true);
  }
  add_chol(J, 0);
  const int mixed = J.mixed ? 1 : 0;
  J.steps.push_back([=]() {
    launch_jacobi(dch, C, mixed, 16, st);
    launch_features(dch, C, tol, d_feat, st);
    if (theta && d_pred) {
      if (rsvd_mlp_forward(theta, 19, d_feat, C, d_pred, st) != RSVD_OK)
        return seterr(RSVD_ERR_CUDA, "rank model inference failed");
    }
    return RSVD_OK;
  });
  return RSVD_OK;
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
  for (int c = 0; c < J.C; ++c) {
    const ChanDims& d = J.d[c];
    Chan& h = J.ch[c];
    const rsvd_matrix& A = J.A[c];
    if (J.rule) {
      h.fro_part = b.take<double>(cdiv(d.n, 8));
      continue;
    }
    if (A.mem == RSVD_MEM_HOST) {
      const double* direct = J.mixed ? host_direct(A) : nullptr;
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
      h.C64 = b.take<double>((size_t)d.l * std::max(d.s, 1));
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


// ------------------------------------------------------------ adaptive loop
// Tolerance-driven blocked range finder, randQB_EI of Yu, Gu & Li (SIAM J.
// Matrix Anal. Appl. 39, 2018), all channels advancing in lockstep, one host
// synchronisation per block (to read each channel's error indicator).
// Per block of b columns (global columns col .. col+b of the Philox matrix):
//   Y = V P_i, Y <- (I - Q Q^T) Y (twice), Q_i = CQR2(Y)
//   q rounds: Z = V Q_i, Qh = CQR2(Z); Y = V Qh, Y <- (I - Q Q^T) Y (twice), Q_i = CQR2(Y)
//   Q_i <- CQR2((I - Q Q^T) Q_i) (twice projected);  W_i = V Q_i  (= B_i^T)
//   E <- E - ||W_i||_F^2; stop once E <= tol^2 ||V||_F^2 (or l_max columns)
// then the thin SVD of B = W^T (CQR2 of W with R accumulated, Jacobi on R^T)
// and the rank by the FP64 identity, exactly as the fixed-l path.
struct AdaptBufs {
  double *Q, *W, *Xo, *T2, *Cb, *Q2big, *E;
  double *Gs, *Rs, *Ris, *Ms, *Js, *sigs, *scrs;     // block (b x b) small buffers
  double *Gf, *Rf, *Rif, *Mf, *Jf, *sigf, *scrf;     // final (l x l)
  double *gpart, *fro_part;
  int lmax;
};

void lay_adapt(Bump& b, const std::vector<ChanDims>& d, int bsz, std::vector<AdaptBufs>& ab,
               std::vector<Chan>& base, const rsvd_matrix* A, rsvd_factors* f, int kfixed) {
  const int C = (int)d.size();
  ab.assign(C, AdaptBufs{});
  base.assign(C, Chan{});
  for (int c = 0; c < C; ++c) {
    const ChanDims& dd = d[c];
    AdaptBufs& x = ab[c];
    Chan& h = base[c];
    x.lmax = dd.l;                       // l holds the per-channel column cap here
    const int64_t T = dd.ldt;
    x.Q = b.take<double>(T * x.lmax);
    x.W = b.take<double>(T * x.lmax);
    x.Xo = b.take<double>(T * bsz);
    x.T2 = b.take<double>(T * bsz);
    x.Cb = b.take<double>((size_t)x.lmax * bsz);
    x.Q2big = b.take<double>(T * x.lmax);
    x.E = b.take<double>(1);
    const size_t sb = (size_t)bsz * (bsz + 32);
    x.Gs = b.take<double>(sb); x.Rs = b.take<double>(sb); x.Ris = b.take<double>(sb);
    x.Ms = b.take<double>(sb); x.Js = b.take<double>(sb);
    x.sigs = b.take<double>(bsz); x.scrs = b.take<double>(bsz);
    const size_t sf = (size_t)x.lmax * (x.lmax + 32);
    x.Gf = b.take<double>(sf); x.Rf = b.take<double>(sf); x.Rif = b.take<double>(sf);
    x.Mf = b.take<double>(sf); x.Jf = b.take<double>(sf);
    x.sigf = b.take<double>(x.lmax); x.scrf = b.take<double>(x.lmax);
    x.gpart = b.take<double>((size_t)dd.gsplit * x.lmax * std::max(x.lmax, bsz));
    x.fro_part = b.take<double>(cdiv(dd.n, 64));
    h.n = dd.n; h.k_cap = dd.kcap; h.k_fixed = kfixed; h.ldt = dd.ldt; h.tol = dd.tol;
    if (A[c].kind == RSVD_TILE_RULE) { h.A = nullptr; h.lda = 0; }     // generated in every pass
    else if (A[c].mem == RSVD_MEM_HOST) { h.A = b.take<double>((size_t)dd.n * dd.n); h.lda = dd.n; }
    else { h.A = A[c].data; h.lda = A[c].ld; }
    h.gpart = x.gpart;
    h.fro_part = x.fro_part;
    const rsvd_factors& F = f[c];
    if (F.mem == RSVD_MEM_HOST) {
      h.U = b.take<double>((size_t)dd.n * dd.kcap); h.ldu = dd.n;
      h.V = b.take<double>((size_t)dd.n * dd.kcap); h.ldv = dd.n;
      h.S = b.take<double>(dd.kcap);
    } else {
      h.U = F.U; h.ldu = F.ldu; h.V = F.V; h.ldv = F.ldv; h.S = F.S;
      if (!h.U) { h.U = b.take<double>((size_t)dd.n * dd.kcap); h.ldu = dd.n; }
      if (!h.V) { h.V = b.take<double>((size_t)dd.n * dd.kcap); h.ldv = dd.n; }
    }
  }
}

// Upload a job's arena and run its steps (synchronous at the end).
rsvd_status run_job(Job& J) {
  rsvd_plan_s* P = J.P;
  if (rsvd_status s = grow_pinned(P, J.ar.h.size() + 64)) return s;
  memcpy(P->hp, J.ar.h.data(), J.ar.h.size());
  CK(cudaMemcpyAsync(J.ar.dbase, P->hp, J.ar.h.size(), cudaMemcpyHostToDevice, P->st));
  for (auto& step : J.steps)
    if (rsvd_status s = step()) return s;
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(P->st));
  drain_profile(P);
  return RSVD_OK;
}

// Y_c -= Q_c (Q_c^T Y_c) for the active channels (m_c = columns of Q so far).
void project_out(Job& J, std::function<const double*(int)> Q, std::function<int(int)> m,
                 std::function<double*(int)> Y, std::function<double*(int)> Cb) {
  add_tn(J, MMK_GRAM_F64, [&](int c) { return (const void*)Q(c); }, [&](int c) { return (const void*)Y(c); },
         Cb, m, [&](int c) { return J.d[c].l; }, false);
  std::vector<MMDesc> md(J.C);
  for (int c = 0; c < J.C; ++c) {
    const ChanDims& d = J.d[c];
    MMDesc mm{};
    mm.A = Q(c); mm.lda = d.ldt;
    mm.B = Cb(c); mm.ldb = std::max(1, m(c));
    mm.Cm = Y(c); mm.ldc = d.ldt;
    mm.m = d.n; mm.n = d.l; mm.k = m(c);
    mm.ks = 1; mm.kchunk = (int)rup(std::max(1, m(c)), 16);
    mm.mode = MM_SUB;
    md[c] = mm;
  }
  add_mm(J, MMK_NN_F64, md);
}

rsvd_status run_adaptive_mixed(rsvd_plan_s* P, int C, const rsvd_matrix* A, rsvd_factors* f,
                               rsvd_status* per_item);

rsvd_status run_adaptive(rsvd_plan_s* P, int C, const rsvd_matrix* A, rsvd_factors* f, rsvd_status* per_item) {
  if (P->o.precision != RSVD_PREC_FP64) return run_adaptive_mixed(P, C, A, f, per_item);
  const int bsz = P->o.block_b > 0 ? P->o.block_b : 32;
  const int lcap = P->o.l_max > 0 ? P->o.l_max : 1024;
  const double tol = P->o.tol;
  const int q = P->o.q;
  std::vector<ChanDims> d(C);
  int64_t sum_tiles = 0;
  for (int c = 0; c < C; ++c) {
    d[c].n = (int)A[c].n;
    d[c].l = std::min(d[c].n, lcap);                       // column cap
    d[c].s = 0; d[c].lw = d[c].l;
    d[c].kcap = std::min(f[c].k_cap, d[c].l);
    d[c].ldt = rup(d[c].n, 4);
    d[c].ldb = rup(d[c].n, 64);
    d[c].tol = f[c].tol > 0.0 ? f[c].tol : tol;
    sum_tiles += (int64_t)cdiv(d[c].l, 64) * cdiv(d[c].l, 64);
  }
  for (int c = 0; c < C; ++c) {
    int g = cdiv(d[c].n, 512);
    const int want = (int)((2 * NSM + sum_tiles - 1) / std::max<int64_t>(1, sum_tiles));
    g = std::max(g, std::min(want, cdiv(d[c].n, 64)));
    d[c].gsplit = std::max(1, std::min(g, 64));
  }
  // workspace: buffers, then a descriptor region reused by every job
  std::vector<AdaptBufs> ab;
  std::vector<Chan> base;
  // tile rules: every pass generates FP64 row panels of the rule
  const bool rule = C > 0 && A[0].kind == RSVD_TILE_RULE;
  std::vector<Job::RuleDev> rd;
  double* p64 = nullptr;
  double* rpart = nullptr;
  int rpanel = 0;
  const size_t arena_reserve = (size_t)1 << 20 | 0;
  size_t buf_bytes = 0;
  {
    Bump b(nullptr);
    lay_adapt(b, d, bsz, ab, base, A, f, P->o.k);
    if (rule) lay_rule64(b, d, A, rd, p64, rpart, rpanel);
    b.take<ChanResult>(C);
    buf_bytes = (b.off + 4095) & ~(size_t)4095;
  }
  const size_t arena_bytes = arena_reserve + (size_t)C * 64 * 1024;
  if (rsvd_status s = grow_ws(P, buf_bytes + arena_bytes)) return s;
  Bump b(P->ws);
  lay_adapt(b, d, bsz, ab, base, A, f, P->o.k);
  if (rule) lay_rule64(b, d, A, rd, p64, rpart, rpanel);
  ChanResult* d_res = b.take<ChanResult>(C);
  char* arena_dev = P->ws + buf_bytes;
  for (int c = 0; c < C; ++c) base[c].res = d_res + c;
  CK(cudaMemsetAsync(d_res, 0, sizeof(ChanResult) * C, P->st));
  CK(cudaMemsetAsync(P->d_err, 0, sizeof(int), P->st));
  for (int c = 0; c < C; ++c)
    if (!rule && A[c].mem == RSVD_MEM_HOST)
      CK(cudaMemcpy2DAsync((void*)base[c].A, (size_t)d[c].n * sizeof(double), A[c].data,
                           (size_t)A[c].ld * sizeof(double), (size_t)d[c].n * sizeof(double), d[c].n,
                           cudaMemcpyHostToDevice, P->st));
  // the rule buffers of the job's channels (chan: job channel -> call channel)
  auto set_rule = [&](Job& J, const std::vector<int>* chan) {
    if (!rule) return;
    J.rule = true;
    J.rd.resize(J.C);
    for (int a = 0; a < J.C; ++a) J.rd[a] = rd[chan ? (*chan)[a] : a];
    J.p64 = p64;
    J.part = rpart;
    J.panel = rpanel;
  };

  // ||V||^2 per channel (tile rules: the FP64 factor panels; ||V||^2 comes
  // with the first generated pass)
  std::vector<double> fro2(C, 0.0);
  if (rule) {
    Job J;
    J.P = P; J.C = C; J.A = A; J.f = f; J.mixed = false; J.measure = false;
    J.d = d;
    J.ch = base;
    J.ar.dbase = arena_dev;
    set_rule(J, nullptr);
    J.d_ch = J.ar.put(J.ch.data(), J.ch.size(), 128);
    const std::vector<RuleDesc64> rds = rule_descs64(J);
    cudaStream_t st = P->st;
    J.steps.push_back([=]() {
      for (const RuleDesc64& r : rds) launch_rule_prep64(r, st);
      return RSVD_OK;
    });
    if (J.ar.h.size() > arena_bytes) return seterr(RSVD_ERR_OOM, "descriptor region too small");
    if (rsvd_status s = run_job(J)) return s;
  } else {
    Job J;
    J.P = P; J.C = C; J.A = A; J.f = f; J.mixed = false; J.measure = false;
    J.d = d;
    J.ch = base;
    J.ar.dbase = arena_dev;
    J.d_ch = J.ar.put(J.ch.data(), J.ch.size(), 128);
    const int* off64 = offsets(J, [&](int c) { return (int64_t)cdiv(d[c].n, 64); });
    const int t64 = total_of(J, [&](int c) { return (int64_t)cdiv(d[c].n, 64); });
    const Chan* dch = J.d_ch;
    cudaStream_t st = P->st;
    J.steps.push_back([=]() {
      launch_fro2(dch, off64, C, t64, st);
      launch_fro2_reduce(dch, C, st);
      return RSVD_OK;
    });
    if (rsvd_status s = run_job(J)) return s;
    std::vector<ChanResult> r(C);
    CK(cudaMemcpy(r.data(), d_res, sizeof(ChanResult) * C, cudaMemcpyDeviceToHost));
    for (int c = 0; c < C; ++c) {
      fro2[c] = r[c].fro2;
      if (r[c].flags & FLAG_NONFINITE) {
        f[c].status = RSVD_ERR_NONFINITE;
      }
    }
  }
  std::vector<int> cols(C, 0);
  std::vector<double> E(fro2);
  std::vector<char> active(C, 1);
  for (int c = 0; c < C; ++c)
    if (f[c].status == RSVD_ERR_NONFINITE) active[c] = 0;
  const uint64_t seed = P->o.seed;
  std::vector<double> Ei(C);
  while (true) {
    std::vector<int> idx;
    for (int c = 0; c < C; ++c)
      if (active[c]) idx.push_back(c);
    if (idx.empty()) break;
    const int Ca = (int)idx.size();
    Job J;
    J.P = P; J.C = Ca; J.A = A; J.f = f; J.mixed = false; J.measure = false;
    J.d.resize(Ca);
    J.ch.resize(Ca);
    J.ar.dbase = arena_dev;
    set_rule(J, &idx);
    bool first = true;
    for (int a = 0; a < Ca; ++a) {
      const int c = idx[a];
      ChanDims dd = d[c];
      dd.l = std::min(bsz, ab[c].lmax - cols[c]);
      dd.kcap = dd.l;
      J.d[a] = dd;
      Chan h = base[c];
      h.l = dd.l;
      h.col0 = cols[c];
      h.X = ab[c].Xo;
      h.G = ab[c].Gs; h.R = ab[c].Rs; h.Ri = ab[c].Ris; h.M = ab[c].Ms; h.J = ab[c].Js;
      h.sig = ab[c].sigs; h.scr = ab[c].scrs;
      J.ch[a] = h;
      first &= cols[c] == 0;
    }
    J.d_ch = J.ar.put(J.ch.data(), J.ch.size(), 128);
    J.max_l = bsz;
    auto Yq = [&](int a) { return ab[idx[a]].Q + (int64_t)cols[idx[a]] * J.d[a].ldt; };
    auto Xw = [&](int a) { return ab[idx[a]].W + (int64_t)cols[idx[a]] * J.d[a].ldt; };
    auto T2 = [&](int a) { return ab[idx[a]].T2; };
    auto Qp = [&](int a) { return (const double*)ab[idx[a]].Q; };
    auto mcols = [&](int a) { return cols[idx[a]]; };
    auto Cb = [&](int a) { return ab[idx[a]].Cb; };
    const int* off64 = offsets(J, [&](int a) { return (int64_t)cdiv(J.d[a].n, 64); });
    const int t64 = total_of(J, [&](int a) { return (int64_t)cdiv(J.d[a].n, 64); });
    {
      const Chan* dch = J.d_ch;
      cudaStream_t st = P->st;
      J.steps.push_back([=]() {
        launch_omega_f64(dch, off64, Ca, t64, seed, 0, st);
        return RSVD_OK;
      });
    }
    pass64(J, [&](int a) { return (const double*)ab[idx[a]].Xo; }, Yq, first);    // Y = V P_i
    if (!first) { project_out(J, Qp, mcols, Yq, Cb); project_out(J, Qp, mcols, Yq, Cb); }
    cqr2_f64(J, Yq, T2, false);
    for (int r = 0; r < q; ++r) {
      pass64(J, [&](int a) { return (const double*)Yq(a); }, Xw, false);         // V Q_i
      cqr2_f64(J, Xw, T2, false);
      pass64(J, [&](int a) { return (const double*)Xw(a); }, Yq, false);         // V Qh
      if (!first) { project_out(J, Qp, mcols, Yq, Cb); project_out(J, Qp, mcols, Yq, Cb); }
      cqr2_f64(J, Yq, T2, false);
    }
    if (!first) {
      project_out(J, Qp, mcols, Yq, Cb);
      project_out(J, Qp, mcols, Yq, Cb);
      cqr2_f64(J, Yq, T2, false);
    }
    pass64(J, [&](int a) { return (const double*)Yq(a); }, Xw, false);           // W_i = V Q_i
    {
      std::vector<SumsqDesc> sd(Ca);
      for (int a = 0; a < Ca; ++a) sd[a] = SumsqDesc{Xw(a), J.d[a].ldt, J.d[a].n, J.d[a].l, 8, ab[idx[a]].E};
      const SumsqDesc* dsd = J.ar.put(sd.data(), sd.size());
      cudaStream_t st = P->st;
      J.steps.push_back([=]() {
        launch_sumsq(dsd, Ca, st);
        return RSVD_OK;
      });
    }
    if (J.ar.h.size() > arena_bytes) return seterr(RSVD_ERR_OOM, "descriptor region too small");
    if (rsvd_status s = run_job(J)) return s;
    for (int a = 0; a < Ca; ++a) {
      const int c = idx[a];
      CK(cudaMemcpyAsync(&Ei[c], ab[c].E, sizeof(double), cudaMemcpyDeviceToHost, P->st));
    }
    CK(cudaStreamSynchronize(P->st));
    if (rule && first) {                     // ||V||^2 from the first generated pass
      std::vector<ChanResult> r(C);
      CK(cudaMemcpy(r.data(), d_res, sizeof(ChanResult) * C, cudaMemcpyDeviceToHost));
      for (int c = 0; c < C; ++c) fro2[c] = E[c] = r[c].fro2;
    }
    for (int a = 0; a < Ca; ++a) {
      const int c = idx[a];
      E[c] -= Ei[c];
      cols[c] += J.d[a].l;
      if (E[c] <= d[c].tol * d[c].tol * fro2[c] || cols[c] >= ab[c].lmax) active[c] = 0;
    }
  }
  // final: SVD of B = W^T on the drawn columns, rank by tolerance, lift
  std::vector<int> idx;
  for (int c = 0; c < C; ++c)
    if (cols[c] > 0) idx.push_back(c);
  const int Cf = (int)idx.size();
  if (Cf > 0) {
    Job J;
    J.P = P; J.C = Cf; J.A = A; J.f = f; J.mixed = false; J.measure = false;
    J.d.resize(Cf);
    J.ch.resize(Cf);
    J.ar.dbase = arena_dev;
    J.policy = RSVD_RANK_TOL;
    J.tol = tol;
    for (int a = 0; a < Cf; ++a) {
      const int c = idx[a];
      ChanDims dd = d[c];
      dd.l = cols[c];
      dd.kcap = std::min(f[c].k_cap, dd.l);
      J.d[a] = dd;
      Chan h = base[c];
      h.l = dd.l;
      h.k_cap = dd.kcap;
      h.G = ab[c].Gf; h.R = ab[c].Rf; h.Ri = ab[c].Rif; h.M = ab[c].Mf; h.J = ab[c].Jf;
      h.sig = ab[c].sigf; h.scr = ab[c].scrf;
      J.ch[a] = h;
      J.max_l = std::max(J.max_l, dd.l);
      J.max_kcap = std::max(J.max_kcap, dd.kcap);
    }
    J.d_ch = J.ar.put(J.ch.data(), J.ch.size(), 128);
    J.d_res = nullptr;
    // fro2 is already in res; results land in res[c]
    auto Wb = [&](int a) { return ab[idx[a]].W; };
    auto Q2 = [&](int a) { return ab[idx[a]].Q2big; };
    cqr2_f64(J, Wb, Q2, true);
    const Chan* dch = J.d_ch;
    const int maxl = J.max_l, maxk = J.max_kcap;
    cudaStream_t st = P->st;
    std::vector<int> ls(Cf);
    for (int a = 0; a < Cf; ++a) ls[a] = J.d[a].l;
    int* coop = P->d_coop;
    int* derr_w = P->d_err;
    J.steps.push_back([=]() {
      run_jacobi(dch, ls, 0, maxl, coop, derr_w, st);
      launch_select(dch, Cf, RSVD_RANK_TOL, tol, 0, st);
      return RSVD_OK;
    });
    // lift (k_out from each channel's result)
    for (int pass = 0; pass < 2; ++pass) {
      std::vector<MMDesc> md(Cf);
      for (int a = 0; a < Cf; ++a) {
        const int c = idx[a];
        const ChanDims& dd = J.d[a];
        MMDesc m{};
        m.A = pass == 0 ? (const void*)ab[c].Q : (const void*)ab[c].W; m.lda = dd.ldt;
        m.B = pass == 0 ? ab[c].Mf : ab[c].Jf; m.ldb = dd.l;
        m.Cm = pass == 0 ? J.ch[a].U : J.ch[a].V; m.ldc = pass == 0 ? J.ch[a].ldu : J.ch[a].ldv;
        m.m = dd.n; m.n = dd.kcap; m.k = dd.l;
        m.ks = 1; m.kchunk = (int)rup(dd.l, 16);
        m.mode = MM_STORE;
        m.ncols_dev = &d_res[c].k_out;
        md[a] = m;
      }
      add_mm(J, MMK_NN_F64, md);
    }
    J.steps.push_back([=]() {
      launch_signfix(dch, Cf, maxk, st);
      return RSVD_OK;
    });
    if (J.ar.h.size() > arena_bytes) return seterr(RSVD_ERR_OOM, "descriptor region too small");
    if (rsvd_status s = run_job(J)) return s;
  }
  std::vector<ChanResult> res(C);
  CK(cudaMemcpy(res.data(), d_res, sizeof(ChanResult) * C, cudaMemcpyDeviceToHost));
  int herr = 0;
  CK(cudaMemcpy(&herr, P->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) return seterr(RSVD_ERR_TIMEOUT, "a bounded device wait expired (code %d)", herr);
  rsvd_status worst = RSVD_OK;
  for (int c = 0; c < C; ++c) {
    rsvd_status s = (rsvd_status)res[c].status;
    if (res[c].flags & FLAG_NONFINITE) s = RSVD_ERR_NONFINITE;
    else if (E[c] > d[c].tol * d[c].tol * fro2[c] && s >= 0) s = RSVD_ERR_TOL_NOT_MET;
    f[c].k_out = cols[c] > 0 ? res[c].k_out : 0;
    f[c].l_used = cols[c];
    f[c].err_est = res[c].err_est;
    f[c].status = s;
    if (per_item) per_item[c] = s;
    if (s < 0 && (worst >= 0 || s < worst)) worst = s;
    else if (worst >= 0 && s > worst) worst = s;
    if (f[c].mem == RSVD_MEM_HOST && f[c].k_out > 0) {
      const int k = f[c].k_out, n = d[c].n;
      CK(cudaMemcpy2DAsync(f[c].U, f[c].ldu * sizeof(double), base[c].U, (size_t)n * sizeof(double),
                           (size_t)n * sizeof(double), k, cudaMemcpyDeviceToHost, P->st));
      CK(cudaMemcpy2DAsync(f[c].V, f[c].ldv * sizeof(double), base[c].V, (size_t)n * sizeof(double),
                           (size_t)n * sizeof(double), k, cudaMemcpyDeviceToHost, P->st));
      CK(cudaMemcpyAsync(f[c].S, base[c].S, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, P->st));
    }
  }
  CK(cudaStreamSynchronize(P->st));
  if (worst < 0) seterr(worst, "at least one channel failed (see per-item status)");
  return worst;
}


// ------------------------------------------------------ adaptive loop (mixed)
// The same randQB_EI blocks on the tensor-core path: V words converted once;
// each block's sketch / power / projection is a tcgen05 pass over the words;
// Gram-Schmidt against earlier blocks by FP32 tile products; orthonormality by
// the mixed CholeskyQR2.  The error indicator cannot use ||V||^2 - ||B||^2
// (it cancels at FP32-accurate projections), so 16 probe columns G ride along
// the first block's sketch and R_G = (I - Q Q^T) V G is updated block by block:
// E ~ ||R_G||^2 / 16.  Stop once E <= (tol / 1.1)^2 ||V||^2 (the probe rank
// rule's margin) or l_max columns.
void project_out_f32(Job& J, std::function<const float*(int)> Q, std::function<int(int)> m,
                     std::function<float*(int)> Y, std::function<int(int)> ncols,
                     std::function<double*(int)> Cb) {
  add_tn(J, MMK_GRAM_F32, [&](int c) { return (const void*)Q(c); }, [&](int c) { return (const void*)Y(c); },
         Cb, m, ncols, false);
  std::vector<MMDesc> md(J.C);
  for (int c = 0; c < J.C; ++c) {
    const ChanDims& d = J.d[c];
    MMDesc mm{};
    mm.A = Q(c); mm.lda = d.ldt;
    mm.B = Cb(c); mm.ldb = std::max(1, m(c));
    mm.Cm = Y(c); mm.ldc = d.ldt;
    mm.m = d.n; mm.n = ncols(c); mm.k = m(c);
    mm.ks = 1; mm.kchunk = (int)rup(std::max(1, m(c)), 16);
    mm.mode = MM_SUB;
    md[c] = mm;
  }
  add_mm(J, MMK_NN_F32_F64B, md);
}

struct AdaptBufsM {
  float *Q32, *W32, *Yb32, *T32, *AG, *RG;
  __nv_bfloat16 *Qw[3], *Xo;
  double *Cb, *E;
  double *Gs, *Rs, *Ris, *Ms, *Js, *sigs, *scrs;
  double *Gf, *Rf, *Rif, *Mf, *Jf, *sigf, *scrf, *C64f, *est;
  float *Ri32s, *Ri32f;
  double *gpart;
  int lmax;
};

void lay_adapt_mixed(Bump& b, const std::vector<ChanDims>& d, int bsz, int nsl, std::vector<AdaptBufsM>& ab,
                     std::vector<Chan>& base, const rsvd_matrix* A, rsvd_factors* f, int kfixed) {
  const int C = (int)d.size();
  ab.assign(C, AdaptBufsM{});
  base.assign(C, Chan{});
  for (int c = 0; c < C; ++c) {          // rank-independent prefix: staged input, words, partials
    Chan& h = base[c];
    if (A[c].kind == RSVD_TILE_RULE) {     // generated in every pass: no input, no words
      h.fro_part = b.take<double>(cdiv(d[c].n, 8));
      continue;
    }
    const double* direct = A[c].mem == RSVD_MEM_HOST ? host_direct(A[c]) : nullptr;
    if (A[c].mem == RSVD_MEM_HOST && !direct) { h.A = b.take<double>((size_t)d[c].n * d[c].n); h.lda = d[c].n; }
    else { h.A = direct ? direct : A[c].data; h.lda = A[c].ld; }
    for (int w = 0; w < nsl; ++w) h.Ab[w] = b.take<__nv_bfloat16>((size_t)d[c].n * d[c].ldb);
    h.fro_part = b.take<double>(cdiv(d[c].n, 8));
    h.wres_part = b.take<double>(cdiv(d[c].n, 8));
  }
  for (int c = 0; c < C; ++c) {
    const ChanDims& dd = d[c];
    AdaptBufsM& x = ab[c];
    Chan& h = base[c];
    x.lmax = dd.l;
    const int64_t T = dd.ldt;
    x.Q32 = b.take<float>(T * x.lmax);
    x.W32 = b.take<float>(T * x.lmax);
    for (int w = 0; w < nsl; ++w) x.Qw[w] = b.take<__nv_bfloat16>((size_t)x.lmax * dd.ldb);
    x.Xo = b.take<__nv_bfloat16>((size_t)(bsz + NPROBE) * dd.ldb);
    x.Yb32 = b.take<float>(T * (bsz + NPROBE));
    x.T32 = b.take<float>(T * bsz);
    x.AG = b.take<float>(T * NPROBE);
    x.RG = b.take<float>(T * NPROBE);
    x.Cb = b.take<double>((size_t)x.lmax * std::max(bsz, NPROBE));
    x.E = b.take<double>(NPROBE);
    const size_t sb = (size_t)bsz * (bsz + 32);
    x.Gs = b.take<double>(sb); x.Rs = b.take<double>(sb); x.Ris = b.take<double>(sb);
    x.Ms = b.take<double>(sb); x.Js = b.take<double>(sb);
    x.Ri32s = b.take<float>((size_t)bsz * bsz);
    x.sigs = b.take<double>(bsz); x.scrs = b.take<double>(bsz);
    const size_t sf = (size_t)x.lmax * (x.lmax + 32);
    x.Gf = b.take<double>(sf); x.Rf = b.take<double>(sf); x.Rif = b.take<double>(sf);
    x.Mf = b.take<double>(sf); x.Jf = b.take<double>(sf);
    x.Ri32f = b.take<float>((size_t)x.lmax * std::max(x.lmax, NPROBE));
    x.sigf = b.take<double>(x.lmax); x.scrf = b.take<double>(x.lmax);
    x.C64f = b.take<double>((size_t)x.lmax * NPROBE);
    x.est = b.take<double>((size_t)NPROBE * (1 + x.lmax));
    x.gpart = b.take<double>((size_t)dd.gsplit * x.lmax * std::max(x.lmax, std::max(bsz, NPROBE)));
    h.n = dd.n; h.k_cap = dd.kcap; h.k_fixed = kfixed; h.ldt = dd.ldt; h.ldb = dd.ldb; h.tol = dd.tol;
    h.nprobe = NPROBE;
    h.gpart = x.gpart;
    const rsvd_factors& F = f[c];
    if (F.mem == RSVD_MEM_HOST) {
      h.U = b.take<double>((size_t)dd.n * dd.kcap); h.ldu = dd.n;
      h.V = b.take<double>((size_t)dd.n * dd.kcap); h.ldv = dd.n;
      h.S = b.take<double>(dd.kcap);
    } else {
      h.U = F.U; h.ldu = F.ldu; h.V = F.V; h.ldv = F.ldv; h.S = F.S;
      if (!h.U) { h.U = b.take<double>((size_t)dd.n * dd.kcap); h.ldu = dd.n; }
      if (!h.V) { h.V = b.take<double>((size_t)dd.n * dd.kcap); h.ldv = dd.n; }
    }
  }
}

rsvd_status run_adaptive_mixed(rsvd_plan_s* P, int C, const rsvd_matrix* A, rsvd_factors* f,
                               rsvd_status* per_item) {
  const int bsz = P->o.block_b > 0 ? P->o.block_b : 32;
  const int lcap = P->o.l_max > 0 ? P->o.l_max : 1024;
  const int q = P->o.q;
  const int nsl = P->slices;
  const double stop_margin = 0.98;
  std::vector<ChanDims> d(C);
  int64_t sum_tiles = 0;
  for (int c = 0; c < C; ++c) {
    d[c].n = (int)A[c].n;
    d[c].l = std::min(d[c].n, lcap);
    d[c].s = NPROBE; d[c].lw = d[c].l + NPROBE;
    d[c].kcap = std::min(f[c].k_cap, d[c].l);
    d[c].ldt = rup(d[c].n, 4);
    d[c].ldb = rup(d[c].n, 64);
    d[c].tol = f[c].tol > 0.0 ? f[c].tol : P->o.tol;
    sum_tiles += (int64_t)cdiv(d[c].l, 64) * cdiv(d[c].l, 64);
  }
  for (int c = 0; c < C; ++c) {
    int g = cdiv(d[c].n, 512);
    const int want = (int)((2 * NSM + sum_tiles - 1) / std::max<int64_t>(1, sum_tiles));
    g = std::max(g, std::min(want, cdiv(d[c].n, 64)));
    d[c].gsplit = std::max(1, std::min(g, 64));
  }
  std::vector<AdaptBufsM> ab;
  std::vector<Chan> base;
  // tile rules: every pass generates the entries it reads (no stored words)
  const bool rule = C > 0 && A[0].kind == RSVD_TILE_RULE;
  std::vector<Job::RuleDev> rd;
  __nv_bfloat16* pw[3] = {nullptr, nullptr, nullptr};
  double* rpart = nullptr;
  int rpanel = 0;
  size_t buf_bytes = 0;
  {
    Bump b(nullptr);
    lay_adapt_mixed(b, d, bsz, nsl, ab, base, A, f, P->o.k);
    if (rule) lay_rule(b, d, A, nsl, rd, pw, rpart, rpanel);
    b.take<ChanResult>(C);
    buf_bytes = (b.off + 4095) & ~(size_t)4095;
  }
  const size_t arena_bytes = ((size_t)1 << 20) + (size_t)C * 96 * 1024;
  if (rsvd_status s = grow_ws(P, buf_bytes + arena_bytes)) return s;
  Bump b(P->ws);
  lay_adapt_mixed(b, d, bsz, nsl, ab, base, A, f, P->o.k);
  if (rule) lay_rule(b, d, A, nsl, rd, pw, rpart, rpanel);
  ChanResult* d_res = b.take<ChanResult>(C);
  char* arena_dev = P->ws + buf_bytes;
  for (int c = 0; c < C; ++c) base[c].res = d_res + c;
  CK(cudaMemsetAsync(d_res, 0, sizeof(ChanResult) * C, P->st));
  CK(cudaMemsetAsync(P->d_err, 0, sizeof(int), P->st));
  for (int c = 0; c < C; ++c)
    if (!rule && A[c].mem == RSVD_MEM_HOST && !host_direct(A[c]))        // staged (not read in place)
      CK(cudaMemcpy2DAsync((void*)base[c].A, (size_t)d[c].n * sizeof(double), A[c].data,
                           (size_t)A[c].ld * sizeof(double), (size_t)d[c].n * sizeof(double), d[c].n,
                           cudaMemcpyHostToDevice, P->st));
  // chan: the job's channel a -> the call's channel (for the rule buffers)
  auto new_job = [&](int Cj, const std::vector<int>* chan = nullptr) {
    Job J;
    J.P = P; J.C = Cj; J.A = A; J.f = f; J.mixed = true; J.measure = false; J.nsl = nsl; J.q = q;
    J.tol = P->o.tol;
    J.ar.dbase = arena_dev;
    J.d.resize(Cj);
    J.ch.resize(Cj);
    if (rule) {
      J.rule = true;
      J.rd.resize(Cj);
      for (int a = 0; a < Cj; ++a) J.rd[a] = rd[chan ? (*chan)[a] : a];
      for (int w = 0; w < 3; ++w) J.pw[w] = pw[w];
      J.part = rpart;
      J.panel = rpanel;
    }
    return J;
  };
  // one pass over V: tensor-core product of the stored words, or generation
  // of the rule's entries panel by panel (`gen_first`: also sum ||V||^2 and
  // the words' remainder for the channel results)
  auto vpass = [&](Job& J, int sx, std::function<int(int)> ncols, std::function<const __nv_bfloat16*(int, int)> xw,
                   std::function<float*(int)> y, bool gen_first) -> rsvd_status {
    if (J.rule) return rule_pass(J, sx, ncols, xw, y, gen_first);
    return tc_pass_ex(J, nsl, sx, ncols, xw, y);
  };
  // words + ||V||^2 (tile rules: the factor words; ||V||^2 comes with the first pass)
  std::vector<double> fro2(C, 0.0), wres2(C, 0.0);
  if (rule) {
    Job J = new_job(C);
    J.d = d;
    J.ch = base;
    J.d_ch = J.ar.put(J.ch.data(), J.ch.size(), 128);
    const std::vector<RuleDesc> rds = rule_descs(J);
    cudaStream_t st = P->st;
    J.steps.push_back([=]() {
      for (const RuleDesc& r : rds) launch_rule_prep(r, st);
      return RSVD_OK;
    });
    if (J.ar.h.size() > arena_bytes) return seterr(RSVD_ERR_OOM, "descriptor region too small");
    if (rsvd_status s = run_job(J)) return s;
  } else {
    Job J = new_job(C);
    J.d = d;
    J.ch = base;
    J.d_ch = J.ar.put(J.ch.data(), J.ch.size(), 128);
    const int* off8 = offsets(J, [&](int c) { return (int64_t)cdiv(d[c].n, 8); });
    const int t8 = total_of(J, [&](int c) { return (int64_t)cdiv(d[c].n, 8); });
    const Chan* dch = J.d_ch;
    cudaStream_t st = P->st;
    J.steps.push_back([=]() {
      launch_convert_slices(dch, off8, C, t8, nsl, st);
      launch_fro2_reduce_rows(dch, C, 8, st);
      return RSVD_OK;
    });
    if (rsvd_status s = run_job(J)) return s;
    std::vector<ChanResult> r(C);
    CK(cudaMemcpy(r.data(), d_res, sizeof(ChanResult) * C, cudaMemcpyDeviceToHost));
    for (int c = 0; c < C; ++c) {
      fro2[c] = r[c].fro2;
      wres2[c] = r[c].wres2;
      if (r[c].flags & FLAG_NONFINITE) f[c].status = RSVD_ERR_NONFINITE;
    }
  }
  std::vector<int> cols(C, 0);
  std::vector<char> active(C, 1);
  for (int c = 0; c < C; ++c)
    if (f[c].status == RSVD_ERR_NONFINITE) active[c] = 0;
  const uint64_t seed = P->o.seed;
  const uint64_t pseed = seed ^ 0x5DEECE66DULL;
  std::vector<double> Ei((size_t)C * NPROBE);
  const bool dbg = getenv("RSVD_DEBUG") != nullptr;
  while (true) {
    std::vector<int> idx;
    for (int c = 0; c < C; ++c)
      if (active[c]) idx.push_back(c);
    if (idx.empty()) break;
    const int Ca = (int)idx.size();
    Job J = new_job(Ca, &idx);
    bool first = true;
    for (int a = 0; a < Ca; ++a) {
      const int c = idx[a];
      ChanDims dd = d[c];
      dd.l = std::min(bsz, ab[c].lmax - cols[c]);
      dd.kcap = dd.l;
      J.d[a] = dd;
      first &= cols[c] == 0;
    }
    J.max_l = bsz;
    auto cb = [&](int a) { return ab[idx[a]]; };
    auto bb = [&](int a) { return J.d[a].l; };
    // role tables: omega into Xo; CQR2 of the sketch block into Q_i; CQR2 of Q_i in place
    std::vector<Chan> chO(Ca), chA(Ca), chB(Ca);
    for (int a = 0; a < Ca; ++a) {
      const int c = idx[a];
      const AdaptBufsM& x = ab[c];
      Chan h = base[c];
      h.l = J.d[a].l;
      h.col0 = cols[c];
      h.G = x.Gs; h.R = x.Rs; h.Ri = x.Ris; h.M = x.Ms; h.J = x.Js; h.sig = x.sigs; h.scr = x.scrs;
      h.Ri32 = x.Ri32s;
      h.T32 = x.T32;
      h.Q32 = x.Q32 + (int64_t)cols[c] * d[c].ldt;
      for (int w = 0; w < nsl; ++w) h.Xb[w] = x.Qw[w] + (int64_t)cols[c] * d[c].ldb;
      Chan o = h;
      o.lw = h.l + (first ? NPROBE : 0);
      o.Xb[0] = x.Xo;
      chO[a] = o;
      h.Y32 = x.Yb32;
      chA[a] = h;
      h.Y32 = h.Q32;
      chB[a] = h;
    }
    Chan* dO = J.ar.put(chO.data(), chO.size(), 128);
    Chan* dA = J.ar.put(chA.data(), chA.size(), 128);
    Chan* dB = J.ar.put(chB.data(), chB.size(), 128);
    J.ch = chA;
    J.d_ch = dA;
    const int* off64 = offsets(J, [&](int a) { return (int64_t)cdiv(J.d[a].n, 64); });
    const int t64 = total_of(J, [&](int a) { return (int64_t)cdiv(J.d[a].n, 64); });
    {
      cudaStream_t st = P->st;
      J.steps.push_back([=]() {
        launch_omega_bf16(dO, off64, Ca, t64, seed, 0, 0, 1 << 30, pseed, 1, st);
        return RSVD_OK;
      });
    }
    auto Qb = [&](int a) { return cb(a).Q32 + (int64_t)cols[idx[a]] * J.d[a].ldt; };
    auto Qprev = [&](int a) { return (const float*)cb(a).Q32; };
    auto mprev = [&](int a) { return cols[idx[a]]; };
    auto Cbuf = [&](int a) { return cb(a).Cb; };
    auto Yb = [&](int a) { return cb(a).Yb32; };
    auto qword = [&](int a, int w) { return (const __nv_bfloat16*)(w < nsl ? cb(a).Qw[w] + (int64_t)cols[idx[a]] * J.d[a].ldb : nullptr); };
    // sketch (+ probe columns in the first block)
    if (rsvd_status s = vpass(J, 1, [&](int a) { return bb(a) + (first ? NPROBE : 0); },
                              [&](int a, int w) { return (const __nv_bfloat16*)(w == 0 ? cb(a).Xo : nullptr); },
                              Yb, first)) return s;
    if (first) {
      std::vector<float*> src(Ca), ag(Ca), rg(Ca);
      std::vector<int64_t> ldt(Ca);
      std::vector<int> nrow(Ca);
      for (int a = 0; a < Ca; ++a) {
        src[a] = cb(a).Yb32 + (int64_t)bb(a) * J.d[a].ldt;
        ag[a] = cb(a).AG; rg[a] = cb(a).RG; ldt[a] = J.d[a].ldt; nrow[a] = J.d[a].n;
      }
      cudaStream_t st = P->st;
      J.steps.push_back([=]() {
        for (int a = 0; a < Ca; ++a) {
          const size_t w = (size_t)nrow[a] * sizeof(float), pitch = (size_t)ldt[a] * sizeof(float);
          if (cudaMemcpy2DAsync(ag[a], pitch, src[a], pitch, w, NPROBE, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
              cudaMemcpy2DAsync(rg[a], pitch, src[a], pitch, w, NPROBE, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return seterr(RSVD_ERR_CUDA, "probe copy failed");
        }
        return RSVD_OK;
      });
    } else {
      project_out_f32(J, Qprev, mprev, Yb, bb, Cbuf);
      project_out_f32(J, Qprev, mprev, Yb, bb, Cbuf);
    }
    cqr2_mixed(J, nsl);                                     // Q_i (FP32 + words)
    for (int r = 0; r < q; ++r) {
      if (rsvd_status s = vpass(J, nsl, bb, qword, Yb, false)) return s;
      cqr2_mixed(J, nsl);
      if (rsvd_status s = vpass(J, nsl, bb, qword, Yb, false)) return s;
      if (!first) {
        project_out_f32(J, Qprev, mprev, Yb, bb, Cbuf);
        project_out_f32(J, Qprev, mprev, Yb, bb, Cbuf);
      }
      cqr2_mixed(J, nsl);
    }
    if (!first) {
      project_out_f32(J, Qprev, mprev, Qb, bb, Cbuf);
      project_out_f32(J, Qprev, mprev, Qb, bb, Cbuf);
      J.ch = chB;
      J.d_ch = dB;
      cqr2_mixed(J, nsl);
      J.ch = chA;
      J.d_ch = dA;
    }
    // W_i = V Q_i
    if (rsvd_status s = vpass(J, nsl, bb, qword,
                              [&](int a) { return cb(a).W32 + (int64_t)cols[idx[a]] * J.d[a].ldt; }, false)) return s;
    // R_G <- (I - Q_i Q_i^T) R_G; E_i = ||R_G||^2
    project_out_f32(J, [&](int a) { return (const float*)Qb(a); }, bb, [&](int a) { return cb(a).RG; },
                    [&](int) { return NPROBE; }, Cbuf);
    {
      std::vector<SumsqDesc> sd(Ca);
      for (int a = 0; a < Ca; ++a) sd[a] = SumsqDesc{cb(a).RG, J.d[a].ldt, J.d[a].n, NPROBE, 4, cb(a).E};
      const SumsqDesc* dsd = J.ar.put(sd.data(), sd.size());
      cudaStream_t st = P->st;
      J.steps.push_back([=]() {
        launch_colsumsq(dsd, Ca, NPROBE, st);
        return RSVD_OK;
      });
    }
    if (J.ar.h.size() > arena_bytes) return seterr(RSVD_ERR_OOM, "descriptor region too small");
    if (rsvd_status s = run_job(J)) return s;
    for (int a = 0; a < Ca; ++a)
      CK(cudaMemcpyAsync(&Ei[(size_t)idx[a] * NPROBE], ab[idx[a]].E, NPROBE * sizeof(double), cudaMemcpyDeviceToHost,
                         P->st));
    CK(cudaStreamSynchronize(P->st));
    if (rule && first) {                     // ||V||^2 and the remainder of the generated words
      std::vector<ChanResult> r(C);
      CK(cudaMemcpy(r.data(), d_res, sizeof(ChanResult) * C, cudaMemcpyDeviceToHost));
      for (int c = 0; c < C; ++c) {
        fro2[c] = r[c].fro2;
        wres2[c] = r[c].wres2;
      }
    }
    for (int a = 0; a < Ca; ++a) {
      const int c = idx[a];
      cols[c] += J.d[a].l;
      // the rank rule's bound over the probe columns (see k_select), with a
      // small extra margin so that the final selection agrees with the stop
      const double* e = &Ei[(size_t)c * NPROBE];
      double mean = 0.0, var = 0.0;
      for (int j = 0; j < NPROBE; ++j) mean += e[j];
      mean /= NPROBE;
      for (int j = 0; j < NPROBE; ++j) var += (e[j] - mean) * (e[j] - mean);
      var /= NPROBE - 1;
      const double floor2 = precision_floor2(wres2[c], cols[c], fro2[c]);
      mean += floor2;
      const double ucb = mean + PROBE_Z * std::sqrt(var / NPROBE);
      if (ucb <= stop_margin * d[c].tol * d[c].tol * fro2[c] || cols[c] >= ab[c].lmax) active[c] = 0;
      if (dbg) fprintf(stderr, "rsvd adaptive: chan %d cols %d est %.3e bound %.3e tol %.3e\n", c, cols[c],
                       std::sqrt(mean / std::max(fro2[c], 1e-300)), std::sqrt(ucb / std::max(fro2[c], 1e-300)),
                       d[c].tol);
    }
  }
  // final: probe estimate per rank, SVD of B = W^T, rank, lift
  std::vector<int> idx;
  for (int c = 0; c < C; ++c)
    if (cols[c] > 0) idx.push_back(c);
  const int Cf = (int)idx.size();
  if (Cf > 0) {
    Job J = new_job(Cf, &idx);
    J.policy = RSVD_RANK_TOL;
    for (int a = 0; a < Cf; ++a) {
      const int c = idx[a];
      const AdaptBufsM& x = ab[c];
      ChanDims dd = d[c];
      dd.l = cols[c];
      dd.lw = dd.l + NPROBE;
      dd.kcap = std::min(f[c].k_cap, dd.l);
      J.d[a] = dd;
      Chan h = base[c];
      h.l = dd.l; h.lw = dd.lw; h.k_cap = dd.kcap;
      h.G = x.Gf; h.R = x.Rf; h.Ri = x.Rif; h.M = x.Mf; h.J = x.Jf; h.sig = x.sigf; h.scr = x.scrf;
      h.Ri32 = x.Ri32f;
      h.Q32 = x.Q32; h.Y32 = x.W32; h.C64 = x.C64f; h.est_part = x.est;
      J.ch[a] = h;
      J.max_l = std::max(J.max_l, dd.l);
      J.max_kcap = std::max(J.max_kcap, dd.kcap);
    }
    J.d_ch = J.ar.put(J.ch.data(), J.ch.size(), 128);
    auto& ch = J.ch;
    add_tn(J, MMK_GRAM_F32, [&](int a) { return (const void*)ch[a].Q32; },
           [&](int a) { return (const void*)ab[idx[a]].AG; }, [&](int a) { return ch[a].C64; },
           [&](int a) { return J.d[a].l; }, [&](int) { return NPROBE; }, false);
    {
      std::vector<MMDesc> md(Cf);
      std::vector<SumsqDesc> sd(Cf);
      for (int a = 0; a < Cf; ++a) {
        const ChanDims& dd = J.d[a];
        MMDesc m{};
        m.A = ch[a].Q32; m.lda = dd.ldt;
        m.B = ch[a].C64; m.ldb = dd.l;
        m.Cm = ab[idx[a]].AG; m.ldc = dd.ldt;
        m.m = dd.n; m.n = NPROBE; m.k = dd.l;
        m.ks = 1; m.kchunk = (int)rup(dd.l, 16);
        m.mode = MM_SUB;                                   // AG <- V G - Q C
        md[a] = m;
        sd[a] = SumsqDesc{ab[idx[a]].AG, dd.ldt, dd.n, NPROBE, 4, ch[a].est_part};
      }
      add_mm(J, MMK_NN_F32_F64B, md);
      const SumsqDesc* dsd = J.ar.put(sd.data(), sd.size());
      cudaStream_t st = P->st;
      J.steps.push_back([=]() {
        launch_colsumsq(dsd, Cf, NPROBE, st);
        return RSVD_OK;
      });
    }
    add_tn(J, MMK_GRAM_DOT2, [&](int a) { return (const void*)ch[a].Y32; }, [&](int a) { return (const void*)ch[a].Y32; },
           [&](int a) { return ch[a].G; }, [&](int a) { return J.d[a].l; }, [&](int a) { return J.d[a].l; }, true);
    add_chol(J, 0);
    const int maxl = J.max_l, maxk = J.max_kcap;
    const double tol = P->o.tol;
    cudaStream_t st = P->st;
    {
      const Chan* d0 = J.d_ch;
      std::vector<int> ls(Cf);
      for (int a = 0; a < Cf; ++a) ls[a] = J.d[a].l;
      int* coop = P->d_coop;
    int* derr_w = P->d_err;
      J.steps.push_back([=]() {
        run_jacobi(d0, ls, 1, maxl, coop, derr_w, st);
        return RSVD_OK;
      });
    }
    const Chan* dch = reorth_x(J);
    J.steps.push_back([=]() {
      launch_probe_finish(dch, Cf, maxl, st);
      launch_select(dch, Cf, RSVD_RANK_TOL, tol, 1, st);
      return RSVD_OK;
    });
    J.d_res = d_res;
    for (int pass = 0; pass < 2; ++pass) {
      std::vector<MMDesc> md(Cf);
      for (int a = 0; a < Cf; ++a) {
        const int c = idx[a];
        const ChanDims& dd = J.d[a];
        MMDesc m{};
        m.A = pass == 0 ? (const void*)ch[a].Q32 : (const void*)ch[a].Y32; m.lda = dd.ldt;
        m.B = ch[a].J; m.ldb = dd.l;          // X~ (see reorth_x)
        m.Cm = pass == 0 ? ch[a].U : ch[a].V; m.ldc = pass == 0 ? ch[a].ldu : ch[a].ldv;
        m.m = dd.n; m.n = dd.kcap; m.k = dd.l;
        m.ks = 1; m.kchunk = (int)rup(dd.l, 16);
        m.mode = MM_STORE;
        m.colscale = pass == 0 ? nullptr : ch[a].scr;
        m.ncols_dev = &d_res[c].k_out;
        md[a] = m;
      }
      add_mm(J, MMK_NN_F32_OUT64, md);
    }
    J.steps.push_back([=]() {
      launch_signfix(dch, Cf, maxk, st);
      return RSVD_OK;
    });
    if (J.ar.h.size() > arena_bytes) return seterr(RSVD_ERR_OOM, "descriptor region too small");
    if (rsvd_status s = run_job(J)) return s;
  }
  std::vector<ChanResult> res(C);
  CK(cudaMemcpy(res.data(), d_res, sizeof(ChanResult) * C, cudaMemcpyDeviceToHost));
  int herr = 0;
  CK(cudaMemcpy(&herr, P->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) return seterr(RSVD_ERR_TIMEOUT, "a bounded device wait expired (code %d)", herr);
  rsvd_status worst = RSVD_OK;
  for (int c = 0; c < C; ++c) {
    rsvd_status s = (rsvd_status)res[c].status;
    if (res[c].flags & FLAG_NONFINITE) s = RSVD_ERR_NONFINITE;
    if (dbg)
      fprintf(stderr,
              "rsvd adaptive: chan %d final l %d k %d flags %d sweeps %d err_est %.3e status %d words %.3e\n", c,
              cols[c], res[c].k_out, res[c].flags, res[c].sweeps, res[c].err_est, res[c].status,
              std::sqrt(res[c].wres2 / std::max(res[c].fro2, 1e-300)));
    f[c].k_out = cols[c] > 0 ? res[c].k_out : 0;
    f[c].l_used = cols[c];
    f[c].err_est = res[c].err_est;
    f[c].status = s;
    if (per_item) per_item[c] = s;
    if (s < 0 && (worst >= 0 || s < worst)) worst = s;
    else if (worst >= 0 && s > worst) worst = s;
    if (f[c].mem == RSVD_MEM_HOST && f[c].k_out > 0) {
      const int k = f[c].k_out, n = d[c].n;
      CK(cudaMemcpy2DAsync(f[c].U, f[c].ldu * sizeof(double), base[c].U, (size_t)n * sizeof(double),
                           (size_t)n * sizeof(double), k, cudaMemcpyDeviceToHost, P->st));
      CK(cudaMemcpy2DAsync(f[c].V, f[c].ldv * sizeof(double), base[c].V, (size_t)n * sizeof(double),
                           (size_t)n * sizeof(double), k, cudaMemcpyDeviceToHost, P->st));
      CK(cudaMemcpyAsync(f[c].S, base[c].S, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, P->st));
    }
  }
  CK(cudaStreamSynchronize(P->st));
  if (worst < 0) seterr(worst, "at least one channel failed (see per-item status)");
  return worst;
}

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

enum JobKind { JOB_MAIN = 0, JOB_PROBE = 1 };

// One layout pass + step building; base == nullptr only measures.  Returns
// the bytes the job needs.
struct ProbeOut { float* feat = nullptr; float* pred = nullptr; };
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
  put64(J.policy); put(&J.tol, sizeof(J.tol)); put64(P->o.rayleigh_ritz); put64((int64_t)(uintptr_t)P->o.mlp_weights);
  for (int c = 0; c < J.C; ++c) {
    const ChanDims& d = J.d[c];
    const int64_t v[] = {d.n, d.l, d.lw, d.s, d.kcap, d.gsplit, d.ldt, d.ldb};
    put(v, sizeof(v));
    if (stage_inputs && J.staged[c]) { put64((int64_t)(uintptr_t)J.A[c].data); put64(J.A[c].ld); }
  }
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
  const bool use_graph = P->graphs && !P->profiling && !J.rule && !J.tuning && P->st != nullptr;
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

}  // namespace

// =================================================================== ABI
extern "C" {

const char* rsvd_last_error_string(void) { return g_err; }
int32_t rsvd_version(void) { return 100; }

rsvd_status rsvd_plan(rsvd_plan_t* out, const rsvd_opts* o) {
  g_err[0] = 0;
  if (!out) return seterr(RSVD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!o) return seterr(RSVD_ERR_INVALID_ARG, "opts is NULL");
  if (o->n_max < 1) return seterr(RSVD_ERR_INVALID_ARG, "n_max %lld < 1", (long long)o->n_max);
  if (o->p < 0) return seterr(RSVD_ERR_INVALID_ARG, "p %d < 0", o->p);
  if (o->q < 0 || o->q > 16) return seterr(RSVD_ERR_INVALID_ARG, "q %d outside [0, 16]", o->q);
  if (o->precision != RSVD_PREC_FP64 && o->precision != RSVD_PREC_BF16X)
    return seterr(RSVD_ERR_INVALID_ARG, "precision %d unknown", o->precision);
  if (o->rank_policy < RSVD_RANK_FIXED || o->rank_policy > RSVD_RANK_LEARNED)
    return seterr(RSVD_ERR_INVALID_ARG, "rank_policy %d unknown", o->rank_policy);
  if (o->rank_policy == RSVD_RANK_FIXED && o->k < 1) return seterr(RSVD_ERR_INVALID_ARG, "fixed rank needs k >= 1");
  if (o->rank_policy != RSVD_RANK_FIXED && !(o->tol > 0.0 && o->tol < 1.0))
    return seterr(RSVD_ERR_INVALID_ARG, "tolerance %g outside (0, 1)", o->tol);
  if (o->rank_policy == RSVD_RANK_TOL && o->k + o->p < 1)
    return seterr(RSVD_ERR_INVALID_ARG, "tolerance mode needs k + p >= 1 columns");
  if (o->slices < 0 || o->slices > 3) return seterr(RSVD_ERR_INVALID_ARG, "slices %d outside [0, 3]", o->slices);
  if (o->block_b < 0 || o->l_max < 0) return seterr(RSVD_ERR_INVALID_ARG, "negative block_b or l_max");
  if (o->rayleigh_ritz && (o->precision != RSVD_PREC_FP64 || o->rank_policy != RSVD_RANK_FIXED))
    return seterr(RSVD_ERR_UNSUPPORTED, "Rayleigh-Ritz is built for the FP64 path with a fixed rank");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return seterr(RSVD_ERR_CUDA, "no CUDA device");
  if (o->precision == RSVD_PREC_BF16X) {
    cudaDeviceProp pr;
    if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return seterr(RSVD_ERR_CUDA, "device query failed");
    if (pr.major != 10 || pr.minor != 3)
      return seterr(RSVD_ERR_UNSUPPORTED, "mixed path needs sm_103 (found sm_%d%d)", pr.major, pr.minor);
  }
  rsvd_plan_s* P = new rsvd_plan_s();
  P->o = *o;
  P->st = (cudaStream_t)o->stream;
  P->slices = o->slices ? o->slices : 2;
  if (cudaMalloc((void**)&P->d_err, sizeof(int) * (64 + (size_t)kCoopWsInts)) != cudaSuccess) {
    delete P;
    return seterr(RSVD_ERR_OOM, "cudaMalloc of the error word failed");
  }
  P->d_coop = P->d_err + 64;
  cudaMemsetAsync(P->d_err, 0, sizeof(int), P->st);
  *out = P;
  return RSVD_OK;
}

void rsvd_plan_destroy(rsvd_plan_t P) {
  if (!P) return;
  cudaStreamSynchronize(P->st);
  drop_graphs(P);
  if (P->ws) cudaFree(P->ws);
  if (P->hp) cudaFreeHost(P->hp);
  if (P->d_err) cudaFree(P->d_err);
  for (cudaEvent_t e : P->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : P->tune_ev)
    if (e) cudaEventDestroy(e);
  delete P;
}

int64_t rsvd_plan_workspace_bytes(rsvd_plan_t P) { return P ? (int64_t)P->ws_cap : 0; }

rsvd_status rsvd_plan_set_profiling(rsvd_plan_t P, int32_t enable) {
  if (!P) return seterr(RSVD_ERR_INVALID_ARG, "plan is NULL");
  P->profiling = enable ? 1 : 0;
  return RSVD_OK;
}

rsvd_status rsvd_plan_set_autotune(rsvd_plan_t P, int32_t enable) {
  if (!P) return seterr(RSVD_ERR_INVALID_ARG, "plan is NULL");
  if (enable && !P->autotune) {
    if (cudaStreamSynchronize(P->st) != cudaSuccess)
      return seterr(RSVD_ERR_CUDA, "stream synchronisation failed: %s", cudaGetErrorString(cudaGetLastError()));
    drop_graphs(P);                      // captured with the default shapes
  }
  P->autotune = enable ? 1 : 0;
  return RSVD_OK;
}

rsvd_status rsvd_plan_tune_records(rsvd_plan_t P, rsvd_tune_record* out, int32_t cap, int32_t* count) {
  if (!P || !count || cap < 0 || (cap > 0 && !out)) return seterr(RSVD_ERR_INVALID_ARG, "bad argument");
  *count = (int32_t)P->tune.size();
  for (int32_t i = 0; i < cap && i < *count; ++i) out[i] = P->tune[i].rec;
  return RSVD_OK;
}

rsvd_status rsvd_plan_set_graphs(rsvd_plan_t P, int32_t enable) {
  if (!P) return seterr(RSVD_ERR_INVALID_ARG, "plan is NULL");
  P->graphs = enable ? 1 : 0;
  if (!enable) {
    cudaStreamSynchronize(P->st);
    drop_graphs(P);
  }
  return RSVD_OK;
}

rsvd_status rsvd_plan_profile(rsvd_plan_t P, rsvd_profile* out, int32_t reset) {
  if (!P || !out) return seterr(RSVD_ERR_INVALID_ARG, "NULL argument");
  *out = P->prof;
  out->launches = launch_count() - P->launch_base;
  if (reset) {
    P->prof = rsvd_profile{};
    P->launch_base = launch_count();
  }
  return RSVD_OK;
}

rsvd_status rsvd_decompose_batched(rsvd_plan_t P, int32_t C, const rsvd_matrix* A, rsvd_factors* f,
                                   rsvd_status* per_item) {
  g_err[0] = 0;
  if (rsvd_status s = validate(P, C, A, f)) return s;
  if (P->o.rank_policy == RSVD_RANK_ADAPTIVE) return run_adaptive(P, C, A, f, per_item);
  if (P->o.rank_policy == RSVD_RANK_LEARNED) return run_learned(P, C, A, f, per_item);
  return run_fixed_l(P, C, A, f, per_item, nullptr, false);
}

rsvd_status rsvd_probe_features(rsvd_plan_t P, int32_t C, const rsvd_matrix* A, const double* tol,
                                float* features) {
  g_err[0] = 0;
  if (!features) return seterr(RSVD_ERR_INVALID_ARG, "features is NULL");
  std::vector<rsvd_factors> f(C > 0 ? C : 1);
  for (int c = 0; c < C; ++c) {
    memset(&f[c], 0, sizeof(rsvd_factors));
    f[c].k_cap = 16;
    f[c].S = (double*)features;           // placeholder: validate() wants a non-null S
    f[c].tol = tol ? tol[c] : 0.0;
  }
  if (rsvd_status s = validate(P, C, A, f.data())) return s;
  std::vector<float> feat;
  const float* saved = P->o.mlp_weights;
  P->o.mlp_weights = nullptr;
  rsvd_status s = run_probe(P, C, A, f.data(), 16, &feat, nullptr);
  P->o.mlp_weights = saved;
  if (s) return s;
  CK(cudaMemcpy(features, feat.data(), sizeof(float) * C * 19, cudaMemcpyHostToDevice));
  return RSVD_OK;
}

rsvd_status rsvd_rule_rows(rsvd_plan_t P, const rsvd_matrix* A, int64_t r0, int32_t rows, float* out,
                           int64_t ldo) {
  g_err[0] = 0;
  if (!P || !A || !out) return seterr(RSVD_ERR_INVALID_ARG, "NULL argument");
  if (A->kind != RSVD_TILE_RULE) return seterr(RSVD_ERR_INVALID_ARG, "matrix is not a tile rule");
  const rsvd_matrix& a = *A;
  if (a.n < 1 || a.n > 2000000000LL / 64) return seterr(RSVD_ERR_INVALID_ARG, "n = %lld out of range", (long long)a.n);
  if (rsvd_status s = check_rule(a)) return s;
  if (r0 < 0 || rows < 1 || r0 + rows > a.n)
    return seterr(RSVD_ERR_INVALID_ARG, "rows [%lld, %lld) outside [0, n)", (long long)r0, (long long)(r0 + rows));
  if (ldo < a.n) return seterr(RSVD_ERR_INVALID_ARG, "ldo < n");
  const int n = (int)a.n, M = a.rule_m;
  const int64_t ldh = rule_ldh(M);
  // workspace: H words, parameters, one descriptor
  const size_t hbytes = ((size_t)n * ldh * sizeof(__half) + 255) & ~(size_t)255;
  const size_t pbytes = ((3 * (size_t)M * sizeof(double)) + 255) & ~(size_t)255;
  if (rsvd_status s = grow_ws(P, 2 * hbytes + pbytes + sizeof(TcChan) + 256)) return s;
  __half* H[2];
  for (int w = 0; w < 2; ++w) H[w] = (__half*)(P->ws + w * hbytes);
  double* dpar = (double*)(P->ws + 2 * hbytes);
  TcChan* dtc = (TcChan*)(P->ws + 2 * hbytes + pbytes);
  if (rsvd_status s = grow_pinned(P, pbytes + sizeof(TcChan) + 64)) return s;
  double* hpar = (double*)P->hp;
  memcpy(hpar, a.rule_c, sizeof(double) * M);
  memcpy(hpar + M, a.rule_s, sizeof(double) * M);
  memcpy(hpar + 2 * M, a.rule_w, sizeof(double) * M);
  TcChan* htc = (TcChan*)(P->hp + pbytes);
  memset(htc, 0, sizeof(TcChan));
  const int gbn = std::min(128, (int)rup(rows, 16));
  const void* HA[2] = {H[0], H[1]};
  const void* HX[2] = {H[0] + r0 * ldh, H[1] + r0 * ldh};
  if (int e = tc_encode(htc, HA, 2, ldh, HX, 2, ldh, n, M, rows, gbn, 1))
    return seterr(RSVD_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", e);
  htc->Y = out; htc->ldy = ldo;
  htc->n = M; htc->m = n; htc->ncols = rows;
  htc->mt = cdiv(n, 128); htc->nt = cdiv(rows, gbn); htc->ks = 1; htc->kt_per_split = cdiv(M, 64);
  htc->mode = TC_RULE;
  htc->chunk_kt = 1;
  htc->nw = 0; htc->r0 = (int)r0;
  htc->eta_key = rule_key(a.rule_seed);
  htc->eta_amp3 = (float)(a.rule_eta * 1.7320508075688772);
  const double hscale = rule_hscale(a.rule_w, M);
  htc->hinv = (float)(1.0 / hscale);
  CK(cudaMemcpyAsync(dpar, hpar, pbytes, cudaMemcpyHostToDevice, P->st));
  CK(cudaMemcpyAsync(dtc, htc, sizeof(TcChan), cudaMemcpyHostToDevice, P->st));
  CK(cudaMemsetAsync(P->d_err, 0, sizeof(int), P->st));
  RuleDesc rdsc{};
  rdsc.n = n; rdsc.M = M; rdsc.c = dpar; rdsc.s = dpar + M; rdsc.w = dpar + 2 * M;
  for (int w = 0; w < 2; ++w) rdsc.H[w] = H[w];
  rdsc.ldh = ldh;
  rdsc.hscale = hscale;
  launch_rule_prep(rdsc, P->st);
  if (int e = tc_launch(dtc, 1, htc->mt * htc->nt, 2, 2, gbn, P->d_err, P->st, true))
    return seterr(RSVD_ERR_CUDA, "tile-rule generation launch failed: %s", cudaGetErrorString((cudaError_t)e));
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, P->st));
  CK(cudaStreamSynchronize(P->st));
  if (herr) return seterr(RSVD_ERR_TIMEOUT, "a bounded device wait expired (code %d)", herr);
  return RSVD_OK;
}

rsvd_status rsvd_decompose(rsvd_plan_t P, const rsvd_matrix* A, rsvd_factors* f) {
  return rsvd_decompose_batched(P, 1, A, f, nullptr);
}

rsvd_status rsvd_transform_factors(rsvd_plan_t P, const rsvd_factors* f, int64_t n, const double* B, int64_t ldb,
                                   int64_t m, double* Lt, int64_t ldl, double* Rt, int64_t ldr) {
  g_err[0] = 0;
  if (!P || !f) return seterr(RSVD_ERR_INVALID_ARG, "NULL argument");
  const int k = f->k_out;
  if (n < 1 || m < 1 || n > 2000000000LL / 64 || m > 2000000000LL / 64)
    return seterr(RSVD_ERR_INVALID_ARG, "n = %lld, m = %lld outside [1, 3.1e7]", (long long)n, (long long)m);
  if (k < 0 || k > f->k_cap) return seterr(RSVD_ERR_INVALID_ARG, "k_out %d outside [0, k_cap]", k);
  if (f->mem != RSVD_MEM_DEVICE) return seterr(RSVD_ERR_INVALID_ARG, "factors must be in device memory");
  if (!B || ldb < n) return seterr(RSVD_ERR_INVALID_ARG, "bad basis matrix");
  if (k == 0) return RSVD_OK;
  if (!f->U || !f->V || f->ldu < n || f->ldv < n) return seterr(RSVD_ERR_INVALID_ARG, "bad factors");
  if (!Lt || !Rt || ldl < m || ldr < m) return seterr(RSVD_ERR_INVALID_ARG, "bad outputs");
  if (rsvd_status s = grow_ws(P, 1 << 16)) return s;
  Job J;
  J.P = P; J.C = 1; J.measure = false;
  J.ar.dbase = P->ws;
  // Lt = B^T U_k, Rt = B^T V_k: B read as the rows of B^T (the FP64 tile
  // kernel's row-operand form), one launch each
  auto desc = [&](const double* X, int64_t ldx, double* out, int64_t ldo) {
    MMDesc d{};
    d.A = B; d.lda = ldb;
    d.B = X; d.ldb = ldx;
    d.Cm = out; d.ldc = ldo;
    d.m = (int)m; d.n = k; d.k = (int)n;
    d.ks = 1; d.kchunk = (int)rup(n, 16);
    d.mode = MM_STORE;
    return d;
  };
  J.steps.push_back(make_mm(J, MMK_GRAM_F64, {desc(f->U, f->ldu, Lt, ldl)}));
  J.steps.push_back(make_mm(J, MMK_GRAM_F64, {desc(f->V, f->ldv, Rt, ldr)}));
  return run_job(J);
}

rsvd_status rsvd_symmetric_signs(rsvd_plan_t P, const rsvd_factors* f, int64_t n, double* signs) {
  g_err[0] = 0;
  if (!P || !f) return seterr(RSVD_ERR_INVALID_ARG, "NULL argument");
  const int k = f->k_out;
  if (n < 1 || n > 2000000000LL / 64) return seterr(RSVD_ERR_INVALID_ARG, "n = %lld outside [1, 3.1e7]", (long long)n);
  if (k < 0 || k > f->k_cap) return seterr(RSVD_ERR_INVALID_ARG, "k_out %d outside [0, k_cap]", k);
  if (f->mem != RSVD_MEM_DEVICE) return seterr(RSVD_ERR_INVALID_ARG, "factors must be in device memory");
  if (k == 0) return RSVD_OK;
  if (!f->U || !f->V || f->ldu < n || f->ldv < n || !signs) return seterr(RSVD_ERR_INVALID_ARG, "bad factors");
  launch_sym_signs(f->U, f->ldu, f->V, f->ldv, (int)n, k, signs, P->st);
  CK(cudaGetLastError());
  return RSVD_OK;
}

double rsvd_compression_ratio(int64_t n, int32_t k, int32_t one_factor) {
  if (n < 1 || k < 1) return 0.0;
  const double N = (double)n, R = (double)k;
  return N * N / ((one_factor ? 1.0 : 2.0) * N * R + R);
}

rsvd_status rsvd_reconstruct_error(rsvd_plan_t P, const rsvd_matrix* A, const rsvd_factors* f,
                                   double* rel_err) {
  g_err[0] = 0;
  if (!P || !A || !f || !rel_err) return seterr(RSVD_ERR_INVALID_ARG, "NULL argument");
  if (A->kind != RSVD_DENSE_F64 && A->kind != RSVD_TILE_RULE)
    return seterr(RSVD_ERR_INVALID_ARG, "matrix kind %d unknown", A->kind);
  const bool rule = A->kind == RSVD_TILE_RULE;
  const int64_t n = A->n;
  const int k = f->k_out;
  if (n < 1 || n > P->o.n_max) return seterr(RSVD_ERR_INVALID_ARG, "bad matrix size");
  if (rule) {
    if (n > 2000000000LL / 64) return seterr(RSVD_ERR_INVALID_ARG, "n too large");
    if (rsvd_status s = check_rule(*A)) return s;
  } else if (!A->data || A->ld < n) {
    return seterr(RSVD_ERR_INVALID_ARG, "bad matrix");
  }
  if (k < 0 || k > f->k_cap) return seterr(RSVD_ERR_INVALID_ARG, "k_out %d outside [0, k_cap]", k);
  if (k > 0 && (!f->U || !f->V || !f->S || f->ldu < n || f->ldv < n))
    return seterr(RSVD_ERR_INVALID_ARG, "bad factors");
  const int blocks = resid_blocks(n);
  const bool hA = !rule && A->mem == RSVD_MEM_HOST, hF = f->mem == RSVD_MEM_HOST;
  const int M = rule ? A->rule_m : 0;
  const int64_t ldh = rule ? rup(M, 16) : 0;
  for (int pass = 0; pass < 2; ++pass) {
    Bump bb(pass == 0 ? nullptr : P->ws);
    double* a = hA ? bb.take<double>((size_t)n * n) : nullptr;
    double* u = hF ? bb.take<double>((size_t)n * std::max(k, 1)) : nullptr;
    double* v = hF ? bb.take<double>((size_t)n * std::max(k, 1)) : nullptr;
    double* s = hF ? bb.take<double>(std::max(k, 1)) : nullptr;
    double* H = rule ? bb.take<double>((size_t)n * ldh) : nullptr;
    double* par = rule ? bb.take<double>(3 * (size_t)M) : nullptr;
    double* part = bb.take<double>(2 * (size_t)blocks);
    if (pass == 0) {
      if (rsvd_status st = grow_ws(P, bb.off + 4096)) return st;
      continue;
    }
    if (rsvd_status st = grow_pinned(P, std::max(2 * (size_t)blocks, 3 * (size_t)M) * sizeof(double) + 64))
      return st;
    const double *dU = f->U, *dV = f->V, *dS = f->S;
    int64_t ldu = f->ldu, ldv = f->ldv;
    if (hF && k > 0) {
      CK(cudaMemcpy2DAsync(u, n * sizeof(double), f->U, f->ldu * sizeof(double), n * sizeof(double), k,
                           cudaMemcpyHostToDevice, P->st));
      CK(cudaMemcpy2DAsync(v, n * sizeof(double), f->V, f->ldv * sizeof(double), n * sizeof(double), k,
                           cudaMemcpyHostToDevice, P->st));
      CK(cudaMemcpyAsync(s, f->S, k * sizeof(double), cudaMemcpyHostToDevice, P->st));
      dU = u; dV = v; dS = s; ldu = n; ldv = n;
    }
    if (rule) {
      // every entry regenerated in FP64 from the rule's definition
      double* hpar = (double*)P->hp;
      memcpy(hpar, A->rule_c, sizeof(double) * M);
      memcpy(hpar + M, A->rule_s, sizeof(double) * M);
      memcpy(hpar + 2 * M, A->rule_w, sizeof(double) * M);
      CK(cudaMemcpyAsync(par, hpar, 3 * sizeof(double) * M, cudaMemcpyHostToDevice, P->st));
      RuleDesc64 rd{};
      rd.n = (int)n; rd.M = M; rd.c = par; rd.s = par + M; rd.w = par + 2 * M;
      rd.H = H; rd.ldh = ldh;
      launch_rule_prep64(rd, P->st);
      launch_resid_rule(H, ldh, M, rule_key(A->rule_seed), A->rule_eta * 1.7320508075688772, dU, ldu, dV, ldv,
                        dS, (int)n, k, part, P->st);
    } else {
      const double* dA = A->data;
      int64_t lda = A->ld;
      if (hA) {
        CK(cudaMemcpy2DAsync(a, n * sizeof(double), A->data, A->ld * sizeof(double), n * sizeof(double), n,
                             cudaMemcpyHostToDevice, P->st));
        dA = a; lda = n;
      }
      launch_resid(dA, lda, dU, ldu, dV, ldv, dS, (int)n, k, part, P->st);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(P->hp, part, 2 * (size_t)blocks * sizeof(double), cudaMemcpyDeviceToHost, P->st));
    CK(cudaStreamSynchronize(P->st));
  }
  const double* hp = (const double*)P->hp;
  double r2 = 0.0, a2 = 0.0;
  for (int t = 0; t < blocks; ++t) { r2 += hp[2 * t]; a2 += hp[2 * t + 1]; }
  *rel_err = a2 > 0.0 ? sqrt(r2 / a2) : sqrt(r2);
  return RSVD_OK;
}

}  // extern "C"
