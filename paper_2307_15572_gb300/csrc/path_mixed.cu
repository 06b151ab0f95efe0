// Mixed path: tensor-core passes over the BF16 words of V (stored, or
// generated per row panel from a tile rule), CholeskyQR with compensated
// Grams, the small SVD and its re-orthonormalisation, the probe rank rule,
// and the learned rank's probe job.
#include "api_internal.h"

namespace rsvd_api {

// --------------------------------------------------------------- mixed path
rsvd_status tc_pass_ex(Job& J, int sa, int sx, std::function<int(int)> ncols_of,
                       std::function<const __nv_bfloat16*(int, int)> xword, std::function<float*(int)> yout,
                       std::function<bool(int)> sel) {
  // one grouped tcgen05 launch: Y[:, 0:ncols) = sum words V_a X_b.
  // Default shape: all columns in one tile up to the kernel's register
  // accumulator width (TC_BN_NARROW), else balanced column tiles; k split only when
  // the batch has fewer than two items per SM; as many pipeline stages as
  // shared memory holds; items longest channel first.  Autotuned: one or two
  // more column tiles, the split target (4 items per SM with shorter splits,
  // or none), a 4-stage pipeline, and the plain channel order.
  // the channels of this launch (all of them, or those sel picks)
  std::vector<int> chans;
  for (int c = 0; c < J.C; ++c)
    if (!sel || sel(c)) chans.push_back(c);
  if (chans.empty()) return RSVD_OK;
  const int CC = (int)chans.size();
  int maxnc = 16;
  std::vector<int> nc_of(J.C, 0);
  for (int c : chans) {
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
    for (int e : chans) items0 += (int64_t)cdiv(J.d[e].n, 128) * cdiv(nc_of[e], g.bn);
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
      for (int c : chans) sg.push_back(ks_of(g, c).first);
      if (std::find(sigs.begin(), sigs.end(), sg) == sigs.end()) {
        sigs.push_back(sg);
        uniq.push_back(g);
      }
    }
    cands.swap(uniq);
  }
  std::vector<int64_t> per;
  for (int c : chans) { per.push_back(J.d[c].n); per.push_back(nc_of[c]); }
  const std::string key = tune_key("tc", {sa, sx}, per);
  std::vector<std::function<rsvd_status()>> vars;
  std::vector<rsvd_tune_record> recs;
  for (int ci : tune_pick(J, key, cands.size())) {
    const Cfg g = cands[ci];
    const int bn = g.bn;
    std::vector<TcChan> tcs(CC);
    bool any_split = false;
    std::vector<ZeroDesc> zd(J.C);
    int item = 0;
    // items numbered longest first: the persistent CTAs take items
    // round-robin, so this order balances them (longest-processing-time-first)
    std::vector<int> order(chans);
    if (g.lpt) std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return J.d[a].n > J.d[b].n; });
    for (int pos = 0; pos < CC; ++pos) {
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
      auto rows64 = [&](int c) { return (sel && !sel(c)) ? (int64_t)0 : (int64_t)cdiv(J.d[c].n, 64); };
      const int* off = offsets(J, rows64);
      const int tiles64 = total_of(J, rows64);
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
    const int C = CC;
    // algorithmic traffic: every V word, X word and Y element once; MMA flops
    double bytes = 0.0, flops = 0.0;
    int npairs = 0;
    for (int a = 0; a < sa; ++a)
      for (int x = 0; x < sx; ++x) npairs += (a + x < std::max(sa, sx));
    for (int c : chans) {
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
// The FP64-input passes (k_tc_f64), an alternative for the mixed path
// without power iterations: two passes reading V in FP64 (16 bytes per
// entry) instead of the conversion to words plus two passes over the words
// (20).  On this part they lose: each pass must round V to FP32 on the
// integer pipe again at ~2.7 values per clock per SM to keep up with HBM,
// and with two 64 KiB stages beside the MMA operands the rounding, the MMAs
// and the loads do not overlap enough (3.8-4.0 TB/s measured, against the
// conversion kernel's 6.1 at 12 bytes per entry); so they are taken only on
// request (RSVD_F64PASS=1).  A channel qualifies if its V is in device
// memory with an even leading dimension and a 16-byte aligned base (the
// TMA's row stride); the others keep the words.  The pass needs two words,
// one column tile, and at least one 128-row tile per SM over its channels
// (no k split).  Returns the per-channel choice (all zero: none).
std::vector<char> f64pass_channels(const Job& J) {
  std::vector<char> use(J.C, 0);
  if (!J.mixed || J.rule || J.skip_convert || J.probe_job || J.q != 0 || J.nsl != 2) return use;
  const char* e = getenv("RSVD_F64PASS");
  if (!e || strcmp(e, "1") != 0) return use;
  int64_t items = 0;
  for (int c = 0; c < J.C; ++c) {
    const rsvd_matrix& A = J.A[c];
    if (J.d[c].lw > TC_BN_NARROW) return std::vector<char>(J.C, 0);
    if (A.mem != RSVD_MEM_DEVICE || (A.ld & 1) || ((uintptr_t)A.data & 15)) continue;
    use[c] = 1;
    items += cdiv(J.d[c].n, 128);
  }
  if (items < NSM) use.assign(J.C, 0);
  return use;
}

// One FP64-input pass Y[:, 0:ncols) = V X (sx X words); `stats` also writes
// the channels' ||V||^2 and remainder partials and the Inf/NaN flag.
rsvd_status f64_pass(Job& J, int sx, std::function<int(int)> ncols_of, bool stats, const std::vector<char>& use) {
  std::vector<int> order;
  int maxnc = 16;
  for (int c = 0; c < J.C; ++c)
    if (use[c]) {
      order.push_back(c);
      maxnc = std::max(maxnc, ncols_of(c));
    }
  const int CC = (int)order.size();
  if (CC == 0) return RSVD_OK;
  const int bn = (int)rup(maxnc, 16);
  // longest channel first: the persistent CTAs take items round-robin
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return J.d[a].n > J.d[b].n; });
  std::vector<TcChan> tcs(CC);
  int item = 0;
  double bytes = 0.0, flops = 0.0;
  for (int pos = 0; pos < CC; ++pos) {
    const int c = order[pos];
    const ChanDims& d = J.d[c];
    const int nc = ncols_of(c);
    TcChan& t = tcs[pos];
    memset(&t, 0, sizeof(t));
    if (!J.measure) {
      const void* X[2] = {J.ch[c].Xb[0], J.ch[c].Xb[1]};
      const int e = f64pass_encode(&t, J.ch[c].A, J.ch[c].lda, d.n, X, sx, d.ldb, nc, bn);
      if (e) return seterr(RSVD_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", e);
    }
    t.Y = J.ch[c].Y32;
    t.ldy = d.ldt;
    t.n = d.n;
    t.m = d.n;
    t.ncols = nc;
    t.mt = cdiv(d.n, 128);
    t.nt = 1;
    t.ks = 1;
    t.kt_per_split = cdiv(d.n, 64);
    t.item0 = item;
    item += t.mt;
    if (stats) {
      t.fro_part = J.ch[c].fro_part;
      t.wres_part = J.ch[c].wres_part;
      t.flags = J.d_res ? (int*)((uintptr_t)(J.d_res + c) + offsetof(ChanResult, flags)) : nullptr;
    }
    bytes += (double)d.n * d.n * 8.0 + (double)d.n * nc * (2.0 * sx + 4.0);
    flops += 2.0 * d.n * d.n * nc * (sx == 1 ? 2 : 3);
  }
  const int items = item;
  const TcChan* dtc = J.ar.put(tcs.data(), tcs.size(), 128);
  rsvd_plan_s* P = J.P;
  cudaStream_t st = P->st;
  int* derr = P->d_err;
  const int C = CC;
  J.steps.push_back([=]() {
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (P->profiling) timed_begin(P, &ea, &eb);
    const int e = f64pass_launch(dtc, C, items, sx, bn, stats, derr, st);
    if (e) return seterr(RSVD_ERR_CUDA, "FP64-input tensor-core pass failed: %s", cudaGetErrorString((cudaError_t)e));
    if (P->profiling) {
      cudaEventRecord(eb, st);
      P->pending.push_back({ea, eb, 6, bytes, flops});
    }
    return RSVD_OK;
  });
  return RSVD_OK;
}

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

// Tall x small products C = A B of the mixed path (CholeskyQR's Y R^{-1},
// the lifts, the re-orthonormalisation of X): on the tensor cores
// (k_nn_tc, exact BF16 slices, FP32-grade) where the job allows it and every
// product is a plain store with k, n <= 128, else the CUDA-core FP32 kernel.
void add_nn(Job& J, MMKind kind, std::vector<MMDesc> md) {
  const bool out64 = kind == MMK_NN_F32_OUT64 || kind == MMK_NN_F32_OUT64_B32;
  const bool b64 = kind == MMK_NN_F32_F64B || kind == MMK_NN_F32_OUT64;
  bool tc = nn_tc_enabled(J) && (out64 || kind == MMK_NN_F32 || kind == MMK_NN_F32_F64B) &&
            (int)md.size() == J.C;
  for (int c = 0; c < (int)md.size() && tc; ++c) {
    const MMDesc& m = md[c];
    tc = m.mode == MM_STORE && m.k >= 1 && m.k <= 128 && m.n >= 1 && m.n <= 128 && m.m >= 1 &&
         J.ch[c].nn_bimg && J.ch[c].nn_fexp && (!out64 || m.nsl == 0);
  }
  if (!tc) {
    add_mm(J, kind, std::move(md));
    return;
  }
  std::vector<NnTcDesc> nd(J.C);
  int tiles = 0;
  double flops = 0.0;
  for (int c = 0; c < J.C; ++c) {
    const MMDesc& m = md[c];
    NnTcDesc x{};
    x.A = (const float*)m.A; x.lda = m.lda;
    x.n = m.m; x.K = m.k; x.N = m.n;
    x.tile0 = tiles;
    x.B = m.B; x.ldb = m.ldb; x.b64 = b64 ? 1 : 0;
    x.colscale = m.colscale;
    x.bimg = J.ch[c].nn_bimg; x.fexp = J.ch[c].nn_fexp;
    if (out64) x.C64 = (double*)m.Cm; else x.C32 = (float*)m.Cm;
    x.ldc = m.ldc;
    for (int w = 0; w < 3; ++w) x.sl[w] = m.sl[w];
    x.ldsl = m.ldsl; x.nsl = m.nsl;
    x.ncols_dev = m.ncols_dev;
    x.cond = m.cond;
    nd[c] = x;
    tiles += cdiv(m.m, 128);
    flops += 2.0 * m.m * (double)m.n * m.k;
  }
  const NnTcDesc* dnd = J.ar.put(nd.data(), nd.size());
  const int C = J.C;
  rsvd_plan_s* P = J.P;
  cudaStream_t st = P->st;
  int* derr = P->d_err;
  J.steps.push_back([=]() {
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (P->profiling) timed_begin(P, &ea, &eb);
    if (int e = launch_nn_tc(dnd, C, tiles, derr, st))
      return seterr(RSVD_ERR_CUDA, "tensor-core product launch failed: %s", cudaGetErrorString((cudaError_t)e));
    if (P->profiling) {
      cudaEventRecord(eb, st);
      P->pending.push_back({ea, eb, 5, 0.0, flops});
    }
    return RSVD_OK;
  });
}

// G = Y^T Y of each channel's n x l FP32 panel (leading dim ldt) into its G:
// on the tensor cores (k_gram_tc, split into exact BF16 slices) where the job
// allows it, else with the compensated (Dot2) Gram on the CUDA cores.  Both
// are FP64-grade; fp32_grade asks only for FP32 accuracy (the tensor-core
// form then takes three slices instead of six).
void add_gram32(Job& J, std::function<const float*(int)> src, bool fp32_grade) {
  auto& ch = J.ch;
  bool tc = gram_tc_enabled(J);
  for (int c = 0; c < J.C && tc; ++c)
    tc = ch[c].gtc_part && ch[c].gtc_exp && (J.d[c].ldt % 4) == 0 && ((uintptr_t)src(c) % 16) == 0;
  if (!tc) {
    add_tn(J, MMK_GRAM_DOT2, [&](int c) { return (const void*)src(c); }, [&](int c) { return (const void*)src(c); },
           [&](int c) { return ch[c].G; }, [&](int c) { return J.d[c].l; }, [&](int c) { return J.d[c].l; }, true);
    return;
  }
  std::vector<GramTcDesc> gd(J.C);
  int tiles = 0;
  double flops = 0.0, mma = 0.0;
  for (int c = 0; c < J.C; ++c) {
    const ChanDims& d = J.d[c];
    const int nt = cdiv(d.n, 128);
    gd[c] = GramTcDesc{src(c), d.ldt, d.n, d.l, tiles, nt, ch[c].gtc_part, ch[c].gtc_exp, ch[c].G};
    tiles += nt;
    flops += 2.0 * d.n * d.l * d.l;
    mma += (fp32_grade ? 6.0 : 21.0) * 2.0 * 128.0 * 128.0 * 128.0 * nt;
  }
  const GramTcDesc* dgd = J.ar.put(gd.data(), gd.size());
  const int C = J.C;
  rsvd_plan_s* P = J.P;
  cudaStream_t st = P->st;
  int* derr = P->d_err;
  J.steps.push_back([=]() {
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (P->profiling) timed_begin(P, &ea, &eb);
    if (int e = launch_gram_tc(dgd, C, tiles, fp32_grade ? 1 : 0, derr, st))
      return seterr(RSVD_ERR_CUDA, "tensor-core Gram launch failed: %s", cudaGetErrorString((cudaError_t)e));
    if (P->profiling) {
      cudaEventRecord(eb, st);
      P->pending.push_back({ea, eb, 4, mma, flops});
    }
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
    // (tensor-core slices or compensated Dot2); round 1: Q1 is orthonormal to
    // ~1e-2 and an FP32 Gram would do, but the tensor-core Gram is faster
    // than the CUDA-core FP32 one as well
    if (round == 0 || gram_tc_enabled(J))
      add_gram32(J, [&](int c) { return (const float*)in(c); }, round == 1);
    else
      add_tn(J, MMK_GRAM_F32, [&](int c) { return (const void*)in(c); },
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
    add_nn(J, b32 ? MMK_NN_F32 : MMK_NN_F32_F64B, md);
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
  add_nn(J, b32 ? MMK_NN_F32 : MMK_NN_F32_F64B, md);
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
    add_nn(J, MMK_NN_F32_OUT64_B32, md);
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

rsvd_status build_mixed(Job& J, bool skip_convert) {
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
  const std::vector<char> f64use = J.rule ? std::vector<char>(C, 0) : f64pass_channels(J);
  bool f64p = false, words = false;             // some channels read FP64 V, some read words
  for (int c = 0; c < C; ++c) (f64use[c] ? f64p : words) = true;
  auto wsel = [f64use](int c) { return f64use[c] == 0; };
  if (J.rule) {
    const std::vector<RuleDesc> rds = rule_descs(J);
    J.steps.push_back([=]() {
      for (const RuleDesc& r : rds) launch_rule_prep(r, st);
      launch_omega_bf16(dch, off64, C, t64, seed, 0, 0, 1 << 30, pseed, nsl, st);   // P and probes
      return RSVD_OK;
    });
  } else if (f64p) {
    // P and the probe block, and the words of the channels that keep them;
    // the other channels' sketch pass reads V in FP64 and sums its energies
    const int* offw = offsets(J, [&](int c) { return f64use[c] ? (int64_t)0 : (int64_t)cdiv(J.d[c].n, 8); });
    const int tw = total_of(J, [&](int c) { return f64use[c] ? (int64_t)0 : (int64_t)cdiv(J.d[c].n, 8); });
    double cbytes = 0.0;
    for (int c = 0; c < C; ++c)
      cbytes += (f64use[c] ? 0.0 : (double)J.d[c].n * J.d[c].n * (8.0 + 2.0 * nsl)) +
                (double)J.d[c].n * J.d[c].lw * 2.0 * nsl;
    rsvd_plan_s* P = J.P;
    J.steps.push_back([=]() {
      cudaEvent_t ea = nullptr, eb = nullptr;
      if (P->profiling) timed_begin(P, &ea, &eb);
      launch_convert_omega(dch, offw, tw, off64, t64, C, nsl, seed, pseed, nsl, st);
      if (P->profiling) {
        cudaEventRecord(eb, st);
        P->pending.push_back({ea, eb, 3, cbytes, 0.0});
      }
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
  if (f64p) {
    if (rsvd_status s = f64_pass(J, 1, [&](int c) { return J.d[c].l; }, true, f64use)) return s;
    if (words)
      if (rsvd_status s = tc_pass_ex(J, nsl, 1, [&](int c) { return J.d[c].l; },
                                     [&](int c, int w) { return (const __nv_bfloat16*)J.ch[c].Xb[w]; },
                                     [&](int c) { return J.ch[c].Y32; }, wsel))
        return s;
    J.steps.push_back([=]() {
      launch_fro2_reduce_rows(dch, C, 8, st);
      return RSVD_OK;
    });
  } else if (rsvd_status s = pass_over(J, nsl, 1, 0, true)) {
    return s;
  }
  cqr2_mixed(J, nsl);
  for (int r = 0; r < 2 * J.q; ++r) {
    if (rsvd_status s = pass_over(J, nsl, nsl, 0, false)) return s;
    cqr2_mixed(J, nsl);
  }
  // projection with the probe block: [W | V G] = V [Q | G]
  if (f64p) {
    if (rsvd_status s = f64_pass(J, nsl, [&](int c) { return J.d[c].lw; }, false, f64use)) return s;
    if (words)
      if (rsvd_status s = tc_pass_ex(J, nsl, nsl, [&](int c) { return J.d[c].lw; },
                                     [&](int c, int w) { return (const __nv_bfloat16*)J.ch[c].Xb[w]; },
                                     [&](int c) { return J.ch[c].Y32; }, wsel))
        return s;
  } else if (rsvd_status s = pass_over(J, nsl, nsl, 1, false)) {
    return s;
  }
  // C = Q^T (V G) and the probe residual R = V G - Q C in place of V G
  // (FP32 accumulate is ample for the error estimate), then R's column
  // energies
  bool narrow = true;                                     // the narrow probe kernels: s <= 32, 32 <= l <= 256
  for (int c = 0; c < J.C; ++c)
    narrow = narrow && J.d[c].s <= 32 && J.d[c].l >= 32 && J.d[c].l <= 256 && ch[c].C32;
  std::vector<SumsqDesc> sd(J.C);
  for (int c = 0; c < J.C; ++c)
    sd[c] = SumsqDesc{ch[c].Y32 + (int64_t)J.d[c].l * J.d[c].ldt, J.d[c].ldt, J.d[c].n, J.d[c].s, 4, ch[c].est_part};
  const ProbeDesc* dtn = nullptr;
  const ProbeDesc* dnn = nullptr;
  int ptb = 0, pnb = 0;
  if (narrow) {
    std::vector<ProbeDesc> tn(J.C), nn(J.C);
    int tb = 0, nb = 0;
    for (int c = 0; c < J.C; ++c) {
      const ChanDims& d = J.d[c];
      ProbeDesc p{};
      p.Q = ch[c].Q32; p.ldq = d.ldt;
      p.Z = ch[c].Y32 + (int64_t)d.l * d.ldt; p.ldz = d.ldt;
      p.n = d.n; p.l = d.l; p.s = d.s;
      p.split_rows = (int)rup(cdiv(d.n, d.gsplit), 32);    // the Gram's row splits
      p.splits = cdiv(d.n, p.split_rows);
      p.part = ch[c].gpart;
      p.C = ch[c].C64;
      p.C32 = ch[c].C32;
      p.tile0 = tb;
      tn[c] = p;
      tb += p.splits * cdiv(d.l, 128);
      p.tile0 = nb;
      nn[c] = p;
      nb += cdiv(d.n, 128);
    }
    dtn = J.ar.put(tn.data(), tn.size());
    dnn = J.ar.put(nn.data(), nn.size());
    ptb = tb;
    pnb = nb;
  } else {
    add_tn(J, MMK_GRAM_F32, [&](int c) { return (const void*)ch[c].Q32; },
           [&](int c) { return (const void*)(ch[c].Y32 + (int64_t)J.d[c].l * J.d[c].ldt); },
           [&](int c) { return ch[c].C64; }, [&](int c) { return J.d[c].l; }, [&](int c) { return J.d[c].s; }, false);
    bool c32 = ri32_ok(J);                                  // C (l x s) must fit the l x l FP32 scratch
    for (int c = 0; c < J.C; ++c) c32 = c32 && J.d[c].s <= J.d[c].l;
    if (c32) add_cvt_f32(J, [&](int c) { return (const double*)ch[c].C64; },
                         [&](int c) { return (int64_t)J.d[c].l * J.d[c].s; });
    std::vector<MMDesc> md(J.C);
    for (int c = 0; c < J.C; ++c) {
      const ChanDims& d = J.d[c];
      MMDesc m{};
      m.A = ch[c].Q32; m.lda = d.ldt;
      m.B = c32 ? (const void*)ch[c].Ri32 : (const void*)ch[c].C64; m.ldb = d.l;
      m.Cm = ch[c].Y32 + (int64_t)d.l * d.ldt; m.ldc = d.ldt;
      m.m = d.n; m.n = d.s; m.k = d.l;
      m.ks = 1; m.kchunk = (int)rup(d.l, 16);
      m.mode = MM_SUB;
      md[c] = m;
    }
    add_mm(J, c32 ? MMK_NN_F32 : MMK_NN_F32_F64B, md);
  }
  const SumsqDesc* dsd = J.ar.put(sd.data(), sd.size());
  const int s_max = NPROBE;
  if (!narrow)
    J.steps.push_back([=]() {
      launch_colsumsq(dsd, C, s_max, st);
      return RSVD_OK;
    });
  const int maxl = J.max_l;
  // W^T W = R^T R
  add_gram32(J, [&](int c) { return (const float*)ch[c].Y32; }, false);
  // The narrow probe block runs on a second stream beside the Cholesky and
  // the Jacobi of W (one CTA per channel each): it reads Q and the probe
  // columns of Y32, writes C, its FP32 copy, the Gram partials (consumed by
  // now) and the probe columns, none of which those two read or write; the
  // main stream waits for it before the next use of the partials.
  // Only with l <= 128 (the one-CTA shared-memory Cholesky and Jacobi; the
  // cooperative forms for large l need every CTA resident at once).
  rsvd_plan_s* P = J.P;
  const bool overlap = narrow && maxl <= 128;
  if (narrow && !overlap)
    J.steps.push_back([=]() {
      launch_probe_block(dtn, dnn, C, ptb, pnb, st);
      launch_colsumsq(dsd, C, s_max, st);
      return RSVD_OK;
    });
  if (overlap) {
    if (!P->side) {
      CK(cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&P->fork_ev, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&P->join_ev, cudaEventDisableTiming));
    }
    cudaStream_t side = P->side;
    cudaEvent_t fork_ev = P->fork_ev, join_ev = P->join_ev;
    J.steps.push_back([=]() {
      CK(cudaEventRecord(fork_ev, st));
      CK(cudaStreamWaitEvent(side, fork_ev, 0));
      launch_probe_block(dtn, dnn, C, ptb, pnb, side);
      launch_colsumsq(dsd, C, s_max, side);
      CK(cudaEventRecord(join_ev, side));
      return RSVD_OK;
    });
  }
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
  if (overlap) {                                 // join before the re-orthonormalisation (its Gram uses the partials)
    cudaEvent_t join_ev = P->join_ev;
    J.steps.push_back([=]() {
      CK(cudaStreamWaitEvent(st, join_ev, 0));
      return RSVD_OK;
    });
  }
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

}  // namespace rsvd_api
