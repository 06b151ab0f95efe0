// Adaptive rank (randQB_EI of Yu, Gu & Li, SIAM J. Matrix Anal. Appl. 39,
// 2018): blocks of columns until each channel's error indicator is under
// its tolerance, on the FP64 path and on the mixed path.
#include "api_internal.h"

namespace rsvd_api {

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

void lay_adapt(Bump& b, const std::vector<ChanDims>& d, int bsz, std::vector<AdaptBufs>& ab,
               std::vector<Chan>& base, const rsvd_matrix* A, rsvd_factors* f, int kfixed, bool in_place) {
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
    else if (A[c].mem == RSVD_MEM_HOST && !(in_place && host_direct(A[c]))) {
      h.A = b.take<double>((size_t)dd.n * dd.n); h.lda = dd.n;
    } else {
      h.A = A[c].mem == RSVD_MEM_HOST ? host_direct(A[c]) : A[c].data; h.lda = A[c].ld;
    }
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
  const bool in_place = !rule && fp64_reads_host_in_place(A, C);
  std::vector<Job::RuleDev> rd;
  double* p64 = nullptr;
  double* rpart = nullptr;
  int rpanel = 0;
  const size_t arena_reserve = (size_t)1 << 20 | 0;
  size_t buf_bytes = 0;
  {
    Bump b(nullptr);
    lay_adapt(b, d, bsz, ab, base, A, f, P->o.k, in_place);
    if (rule) lay_rule64(b, d, A, rd, p64, rpart, rpanel);
    b.take<ChanResult>(C);
    buf_bytes = (b.off + 4095) & ~(size_t)4095;
  }
  const size_t arena_bytes = arena_reserve + (size_t)C * 64 * 1024;
  if (rsvd_status s = grow_ws(P, buf_bytes + arena_bytes)) return s;
  Bump b(P->ws);
  lay_adapt(b, d, bsz, ab, base, A, f, P->o.k, in_place);
  if (rule) lay_rule64(b, d, A, rd, p64, rpart, rpanel);
  ChanResult* d_res = b.take<ChanResult>(C);
  char* arena_dev = P->ws + buf_bytes;
  for (int c = 0; c < C; ++c) base[c].res = d_res + c;
  CK(cudaMemsetAsync(d_res, 0, sizeof(ChanResult) * C, P->st));
  CK(cudaMemsetAsync(P->d_err, 0, sizeof(int), P->st));
  for (int c = 0; c < C; ++c)
    if (!rule && A[c].mem == RSVD_MEM_HOST && !(in_place && host_direct(A[c])))
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

}  // namespace rsvd_api
