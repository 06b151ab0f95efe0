// Internal declarations shared by the host orchestration files of the C ABI
// (plan_common.cu, path_fp64.cu, path_mixed.cu, adaptive.cu, job.cu,
// api.cu).  Not part of the ABI; every arithmetic step of the method runs in
// the kernels (k_*.cu).
#pragma once

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

namespace rsvd_api {

// Thread-local text of the last error (rsvd_last_error_string).
extern thread_local char g_err[1024];
rsvd_status seterr(rsvd_status s, const char* fmt, ...);

#define CK(call)                                                                             \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return seterr(e_ == cudaErrorMemoryAllocation ? RSVD_ERR_OOM : RSVD_ERR_CUDA, "%s: %s", \
                    #call, cudaGetErrorString(e_));                                          \
  } while (0)

inline int64_t rup(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

constexpr int NPROBE = 32;
constexpr int NSM = 152;

}  // namespace rsvd_api

using namespace rsvd_api;

struct rsvd_plan_s {
  rsvd_opts o;
  cudaStream_t st = nullptr;
  // a second stream (and its fork/join events) for work that overlaps the
  // per-channel kernels of the same decomposition; created on first use
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
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

void drop_graphs(rsvd_plan_s* P);

namespace rsvd_api {

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

struct ChanDims {
  int n, l, lw, s, kcap, gsplit;
  int64_t ldt, ldb;
  double tol;
};

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
  bool host_in_place = false;           // FP64 path: page-locked host V read in place (fp64_reads_host_in_place)
};

struct AdaptBufs {
  double *Q, *W, *Xo, *T2, *Cb, *Q2big, *E;
  double *Gs, *Rs, *Ris, *Ms, *Js, *sigs, *scrs;     // block (b x b) small buffers
  double *Gf, *Rf, *Rif, *Mf, *Jf, *sigf, *scrf;     // final (l x l)
  double *gpart, *fro_part;
  int lmax;
};

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

enum JobKind { JOB_MAIN = 0, JOB_PROBE = 1 };

struct ProbeOut { float* feat = nullptr; float* pred = nullptr; };

bool gram_tc_enabled(const Job& J);
bool nn_tc_enabled(const Job& J);
void add_nn(Job& J, MMKind kind, std::vector<MMDesc> md);
rsvd_status grow_pinned(rsvd_plan_s* P, size_t bytes);
rsvd_status grow_ws(rsvd_plan_s* P, size_t bytes);
void timed_begin(rsvd_plan_s* P, cudaEvent_t* a, cudaEvent_t* b);
void run_jacobi(const Chan* dch, const std::vector<int>& ls, int fp32, int maxl, int* coop, int* err, cudaStream_t st);
void run_chol(const Chan* dch, const std::vector<int>& ls, int accumulate, int maxl, int f32inv, int f32_chol,
              int conditional, int* coop, int* err, cudaStream_t st);
void drain_profile(rsvd_plan_s* P);
int pick_splits(int64_t tiles, int64_t k, int min_chunk, int64_t target = 2 * NSM);
int64_t rule_ldh(int M);
int rule_panel_rows(int64_t n, int64_t ldb, int nsl);
uint32_t rule_key(uint64_t seed);
const double* host_direct(const rsvd_matrix& A);
const int* offsets(Job& J, const std::function<int64_t(int)>& per);
int total_of(Job& J, const std::function<int64_t(int)>& per);
std::string tune_key(const char* kind, std::initializer_list<int64_t> head, const std::vector<int64_t>& per);
void add_tuned(Job& J, const std::string& key, const std::vector<rsvd_tune_record>& recs,
               const std::vector<std::function<rsvd_status()>>& vars);
std::vector<int> tune_pick(Job& J, const std::string& key, size_t ncand);
void add_mm(Job& J, MMKind kind, std::vector<MMDesc> md);
std::function<rsvd_status()> make_mm(Job& J, MMKind kind, std::vector<MMDesc> md);
void add_tn_ex(Job& J, MMKind kind, std::function<const void*(int)> Ap, std::function<const void*(int)> Bp,
               std::function<double*(int)> outp, std::function<int(int)> mcols, std::function<int(int)> ncols,
               bool sym, std::function<int(int)> rows, std::function<int64_t(int)> ld,
               std::function<int(int)> splits, std::function<const int*(int)> cond = nullptr);
void add_tn(Job& J, MMKind kind, std::function<const void*(int)> Ap, std::function<const void*(int)> Bp,
            std::function<double*(int)> outp, std::function<int(int)> mcols, std::function<int(int)> ncols,
            bool sym);
std::vector<int> chan_ls(const Job& J);
void add_chol(Job& J, int accumulate, int f32_chol = 0);
void cqr2_f64(Job& J, std::function<double*(int)> src, std::function<double*(int)> tmp, bool acc_R);
void dense_f64(Job& J, std::function<const double*(int)> X, std::function<double*(int)> Y);
void lift(Job& J, MMKind kind, std::function<const void*(int)> basis, std::function<const void*(int)> small,
          std::function<double*(int)> out, std::function<int64_t(int)> ldo, std::function<const double*(int)> scale);
std::vector<RuleDesc64> rule_descs64(Job& J);
void rule_pass64(Job& J, std::function<const double*(int)> X, std::function<double*(int)> Y, bool first);
void pass64(Job& J, std::function<const double*(int)> X, std::function<double*(int)> Y, bool first);
void build_fp64(Job& J);
rsvd_status tc_pass_ex(Job& J, int sa, int sx, std::function<int(int)> ncols_of,
                       std::function<const __nv_bfloat16*(int, int)> xword, std::function<float*(int)> yout,
                       std::function<bool(int)> sel = nullptr);
rsvd_status tc_pass(Job& J, int sa, int sx, int ncols_of_pass /*0: l, 1: lw*/);
rsvd_status rule_pass(Job& J, int sx, std::function<int(int)> ncols_of,
                      std::function<const __nv_bfloat16*(int, int)> xword, std::function<float*(int)> yout,
                      bool first);
rsvd_status pass_over(Job& J, int sa, int sx, int ncols_of_pass, bool first);
bool ri32_ok(const Job& J);
void add_cvt_f32(Job& J, std::function<const double*(int)> src, std::function<int64_t(int)> count);
void cqr2_mixed(Job& J, int nsl_out);
Chan* reorth_x(Job& J);
std::vector<RuleDesc> rule_descs(Job& J);
rsvd_status build_mixed(Job& J, bool skip_convert = false);
rsvd_status build_probe(Job& J, float* d_feat, const float* theta, float* d_pred);
int rule_panel_rows64(int64_t maxn);
void lay_rule64(Bump& b, const std::vector<ChanDims>& d, const rsvd_matrix* A, std::vector<Job::RuleDev>& rd,
                double*& p64, double*& part, int& panel);
void lay_rule(Bump& b, const std::vector<ChanDims>& d, const rsvd_matrix* A, int nsl, std::vector<Job::RuleDev>& rd,
              __nv_bfloat16* (&pw)[3], double*& part, int& panel);
void layout(Job& J, Bump& b);
rsvd_status check_rule(const rsvd_matrix& a);
bool fp64_reads_host_in_place(const rsvd_matrix* A, int C);
rsvd_status validate(const rsvd_plan_s* P, int C, const rsvd_matrix* A, rsvd_factors* f);
void lay_adapt(Bump& b, const std::vector<ChanDims>& d, int bsz, std::vector<AdaptBufs>& ab,
               std::vector<Chan>& base, const rsvd_matrix* A, rsvd_factors* f, int kfixed, bool in_place);
rsvd_status run_job(Job& J);
void project_out(Job& J, std::function<const double*(int)> Q, std::function<int(int)> m,
                 std::function<double*(int)> Y, std::function<double*(int)> Cb);
rsvd_status run_adaptive(rsvd_plan_s* P, int C, const rsvd_matrix* A, rsvd_factors* f, rsvd_status* per_item);
void project_out_f32(Job& J, std::function<const float*(int)> Q, std::function<int(int)> m,
                     std::function<float*(int)> Y, std::function<int(int)> ncols,
                     std::function<double*(int)> Cb);
void lay_adapt_mixed(Bump& b, const std::vector<ChanDims>& d, int bsz, int nsl, std::vector<AdaptBufsM>& ab,
                     std::vector<Chan>& base, const rsvd_matrix* A, rsvd_factors* f, int kfixed);
rsvd_status run_adaptive_mixed(rsvd_plan_s* P, int C, const rsvd_matrix* A, rsvd_factors* f,
                               rsvd_status* per_item);
void init_job(Job& J, rsvd_plan_s* P, int C, const rsvd_matrix* A, rsvd_factors* f);
void make_dims(Job& J, const std::vector<int>* lvec, std::vector<int>& warn, int probe_cols);
rsvd_status build_job(Job& J, char* base, JobKind kind, bool skip_convert, size_t* need, ProbeOut* po);
std::string graph_key(const Job& J, bool stage_inputs);
rsvd_status execute(Job& J, bool stage_inputs, std::vector<ChanResult>& res);
rsvd_status collect(Job& J, const std::vector<ChanResult>& res, const std::vector<int>& warn, rsvd_factors* f,
                    rsvd_status* per_item, rsvd_status* worst_out);
rsvd_status run_fixed_l(rsvd_plan_s* P, int C, const rsvd_matrix* A, rsvd_factors* f, rsvd_status* per_item,
                        const std::vector<int>* lvec, bool reuse_words);
rsvd_status run_probe(rsvd_plan_s* P, int C, const rsvd_matrix* A, rsvd_factors* f, int lcap,
                      std::vector<float>* feat, std::vector<float>* pred);
rsvd_status run_learned(rsvd_plan_s* P, int C, const rsvd_matrix* A, rsvd_factors* f, rsvd_status* per_item);

}  // namespace rsvd_api
