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
#include <atomic>

#include "api_internal.h"

namespace rsvd {
static std::atomic<long long> g_launches{0};
void note_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace rsvd

namespace rsvd_api {

thread_local char g_err[1024] = "";

rsvd_status seterr(rsvd_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

}  // namespace rsvd_api

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

void drop_graphs(rsvd_plan_s* P) {
  for (auto& g : P->gcache) cudaGraphExecDestroy(g.exec);
  P->gcache.clear();
}


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
  if (P->side) {
    cudaStreamSynchronize(P->side);
    cudaStreamDestroy(P->side);
  }
  if (P->fork_ev) cudaEventDestroy(P->fork_ev);
  if (P->join_ev) cudaEventDestroy(P->join_ev);
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

rsvd_status rsvd_gram_f32(rsvd_plan_t P, const float* Y, int64_t ldy, int64_t n, int32_t l, double* G,
                          int32_t method) {
  g_err[0] = 0;
  if (!P || !Y || !G) return seterr(RSVD_ERR_INVALID_ARG, "NULL argument");
  if (n < 1 || n > 2000000000LL / 64 || l < 1 || l > 4096 || ldy < n)
    return seterr(RSVD_ERR_INVALID_ARG, "n = %lld, l = %d, ldy = %lld out of range", (long long)n, l, (long long)ldy);
  const int nn = (int)n;
  if (method == RSVD_GRAM_TC || method == RSVD_GRAM_TC_F32) {
    if (l > 128) return seterr(RSVD_ERR_UNSUPPORTED, "tensor-core Gram needs l <= 128 (l = %d)", l);
    if ((ldy % 4) != 0 || ((uintptr_t)Y % 16) != 0)
      return seterr(RSVD_ERR_UNSUPPORTED, "tensor-core Gram needs ldy %% 4 == 0 and a 16-byte aligned Y");
    const int nt = cdiv(nn, 128);
    const size_t pb = ((size_t)gram_tc_part_floats(nn) * sizeof(float) + 255) & ~(size_t)255;
    const size_t eb = ((size_t)nt * 128 * sizeof(int) + 255) & ~(size_t)255;
    if (rsvd_status s = grow_ws(P, pb + eb + sizeof(GramTcDesc) + 256)) return s;
    if (rsvd_status s = grow_pinned(P, sizeof(GramTcDesc))) return s;
    GramTcDesc* hd = (GramTcDesc*)P->hp;
    *hd = GramTcDesc{Y, ldy, nn, l, 0, nt, (float*)P->ws, (int*)(P->ws + pb), G};
    GramTcDesc* dd = (GramTcDesc*)(P->ws + pb + eb);
    CK(cudaMemcpyAsync(dd, hd, sizeof(GramTcDesc), cudaMemcpyHostToDevice, P->st));
    CK(cudaMemsetAsync(P->d_err, 0, sizeof(int), P->st));
    if (int e = launch_gram_tc(dd, 1, nt, method == RSVD_GRAM_TC_F32 ? 1 : 0, P->d_err, P->st))
      return seterr(RSVD_ERR_CUDA, "tensor-core Gram launch failed: %s", cudaGetErrorString((cudaError_t)e));
  } else if (method == RSVD_GRAM_DOT2) {
    const int gs = std::max(1, std::min(cdiv(nn, 512), 64));
    MMDesc m{};
    m.A = Y; m.lda = ldy; m.B = Y; m.ldb = ldy;
    m.m = l; m.n = l; m.k = nn;
    m.mt = cdiv(l, 64); m.nt = cdiv(l, 64);
    m.kchunk = (int)rup(cdiv(nn, gs), 16);
    m.ks = cdiv(nn, m.kchunk);
    m.mode = MM_PARTIAL; m.sym = 1;
    m.ldc = l; m.pstride = (int64_t)l * l;
    m.tile = tile_of(MMK_GRAM_DOT2);
    const int tiles = m.mt * m.nt * m.ks;
    const size_t gb = ((size_t)m.ks * l * l * sizeof(double) + 255) & ~(size_t)255;
    if (rsvd_status s = grow_ws(P, gb + 256 + 256)) return s;
    if (rsvd_status s = grow_pinned(P, 256)) return s;
    m.Cm = P->ws;
    char* hp = (char*)P->hp;
    memcpy(hp, &m, sizeof(MMDesc));
    const int off[2] = {0, tiles};
    memcpy(hp + 192, off, sizeof(off));
    memcpy(hp + 208, &G, sizeof(double*));
    static_assert(sizeof(MMDesc) <= 192, "descriptor block");
    CK(cudaMemcpyAsync(P->ws + gb, hp, 256, cudaMemcpyHostToDevice, P->st));
    CK(cudaMemsetAsync(P->d_err, 0, sizeof(int), P->st));
    const MMDesc* dm = (const MMDesc*)(P->ws + gb);
    launch_tile_mm(MMK_GRAM_DOT2, dm, (const int*)(P->ws + gb + 192), 1, tiles, P->st);
    launch_reduce_partials(dm, (double* const*)(P->ws + gb + 208), 1, l * l, P->st);
  } else {
    return seterr(RSVD_ERR_INVALID_ARG, "unknown Gram method %d", method);
  }
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, P->st));
  CK(cudaStreamSynchronize(P->st));
  CK(cudaGetLastError());
  if (herr) return seterr(RSVD_ERR_TIMEOUT, "a bounded device wait expired (code %d)", herr);
  return RSVD_OK;
}

rsvd_status rsvd_panel_product(rsvd_plan_t P, const float* A, int64_t lda, int64_t n, int32_t K, const void* B,
                               int64_t ldb, int32_t b_fp64, int32_t N, void* Cout, int64_t ldc, int32_t c_fp64) {
  g_err[0] = 0;
  if (!P || !A || !B || !Cout) return seterr(RSVD_ERR_INVALID_ARG, "NULL argument");
  if (n < 1 || n > 2000000000LL / 64 || K < 1 || N < 1 || lda < n || ldb < K || ldc < n)
    return seterr(RSVD_ERR_INVALID_ARG, "n = %lld, K = %d, N = %d or a leading dimension out of range", (long long)n,
                  K, N);
  if (K > 128 || N > 128) return seterr(RSVD_ERR_UNSUPPORTED, "tensor-core product needs K, N <= 128");
  const size_t ib = ((size_t)nn_tc_img_bytes() + 255) & ~(size_t)255;
  if (rsvd_status s = grow_ws(P, ib + 512 + 256 + sizeof(NnTcDesc))) return s;
  if (rsvd_status s = grow_pinned(P, sizeof(NnTcDesc))) return s;
  NnTcDesc* hd = (NnTcDesc*)P->hp;
  memset(hd, 0, sizeof(NnTcDesc));
  hd->A = A; hd->lda = lda;
  hd->n = (int)n; hd->K = K; hd->N = N;
  hd->B = B; hd->ldb = ldb; hd->b64 = b_fp64 ? 1 : 0;
  hd->bimg = P->ws;
  hd->fexp = (int*)(P->ws + ib);
  if (c_fp64) hd->C64 = (double*)Cout; else hd->C32 = (float*)Cout;
  hd->ldc = ldc;
  NnTcDesc* dd = (NnTcDesc*)(P->ws + ib + 512);
  CK(cudaMemcpyAsync(dd, hd, sizeof(NnTcDesc), cudaMemcpyHostToDevice, P->st));
  CK(cudaMemsetAsync(P->d_err, 0, sizeof(int), P->st));
  if (int e = launch_nn_tc(dd, 1, cdiv((int)n, 128), P->d_err, P->st))
    return seterr(RSVD_ERR_CUDA, "tensor-core product launch failed: %s", cudaGetErrorString((cudaError_t)e));
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
