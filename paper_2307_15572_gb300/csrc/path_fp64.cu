// All-FP64 path (every step on the CUDA cores): CholeskyQR2 with a
// conditional third round, the grouped FP64 passes over V (stored or
// generated from a tile rule), lifts, and the whole fixed-l pipeline.
#include "api_internal.h"

namespace rsvd_api {

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
  if (J.mixed) add_nn(J, kind, md);      // the tensor-core product where it applies
  else add_mm(J, kind, md);
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

}  // namespace rsvd_api
