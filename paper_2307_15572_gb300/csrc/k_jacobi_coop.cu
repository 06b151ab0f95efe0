// One-sided Jacobi SVD of M = R^T for large l, with several CTAs per channel.
//
// The single-CTA kernel (k_small.cu) keeps the l x l factor in shared memory;
// past ~110 (FP64 with right vectors) or ~220 (FP32) columns it falls back to
// global memory on one SM, and at l ~ 800 an FP64 SVD then takes seconds (one
// SM delivers 1/152 of the part's FP64 rate).  Here the same sweep -- Hestenes
// rotations (Golub & Van Loan, 4th ed., Sec. 8.6.3) in the round-robin order of
// Brent & Luk (1985), whose m/2 pairs per round are disjoint -- runs on a
// cooperative grid: the pairs of a round are spread over the CTAs given to the
// channel (in proportion to l^2), the columns live in global memory (L2), and a
// grid-wide barrier separates rounds.  Every channel advances in lockstep;
// converged channels idle.  The barrier's spin is bounded (an expired wait sets
// an error word and every CTA returns).  A second kernel normalises, sorts and
// writes X (= M_i / sigma_i), J and sigma exactly as the single-CTA kernel does.
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "kernels.h"

namespace rsvd {

struct CoopMap {
  int C;
  int nblocks;
  int first[kCoopMaxChannels + 1];   // CTAs [first[c], first[c+1]) serve channel c
};

// coop workspace (ints): [0] barrier count, [1] barrier generation, [2] error,
// [3] sweeps done, [4 + s * C + c] channel c rotated in sweep s.
static constexpr int kCoopSweeps = 60;

// Grid barrier with a bounded spin.  A wait that exceeds ctl.budget clocks
// records the expiry (ws[2] for the grid, DERR_TIMEOUT_BARRIER in the plan's
// error word for the host) and every CTA returns at its next barrier.  The
// verdict is taken once per CTA, by thread 0, and shared, so all threads of a
// CTA return together.
RSVD_DEV bool coop_barrier(int* ws, unsigned int nblocks, const CoopCtl& ctl) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    unsigned int* cnt = (unsigned int*)ws;
    volatile unsigned int* gen = (volatile unsigned int*)(ws + 1);
    __threadfence();
    const unsigned int g = *gen;
    if (atomicAdd(cnt, 1u) == nblocks - 1) {
      atomicExch(cnt, 0u);
      __threadfence();
      atomicAdd((unsigned int*)(ws + 1), 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (clock64() - t0 > ctl.budget) {
          ok = 0;
          atomicExch(ws + 2, 1);
          set_err(ctl.err, DERR_TIMEOUT_BARRIER);
          break;
        }
      }
    }
    __threadfence();
    if (*(volatile int*)(ws + 2) != 0) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// Test hook (ctl.stall): CTA 0 leaves before its first barrier, like a
// participant that never arrives; the others' bounded waits then expire.
RSVD_DEV bool coop_stalled(const CoopCtl& ctl) { return ctl.stall && blockIdx.x == 0; }

template <typename T> struct CVec;
template <> struct CVec<float> { typedef float4 V; static constexpr int N = 4; };
template <> struct CVec<double> { typedef double2 V; static constexpr int N = 2; };

RSVD_DEV float cget(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
RSVD_DEV double cget(const double2& v, int i) { return i == 0 ? v.x : v.y; }

// Working copies: M in h.G, J in h.Ri (both l x (l + 32) doubles, free at
// this point of the pipeline), columns of stride lp = round_up(l, 8 vectors).
template <typename T, bool WANT_J>
__global__ void __launch_bounds__(256) k_jacobi_coop(const Chan* __restrict__ ch, const __grid_constant__ CoopMap map,
                                                     int* __restrict__ ws, const CoopCtl ctl) {
  typedef typename CVec<T>::V V;
  constexpr int VE = CVec<T>::N;
  // channel of this CTA
  int c = 0;
  while (c + 1 < map.C && map.first[c + 1] <= (int)blockIdx.x) ++c;
  const int rank = blockIdx.x - map.first[c], ncta = map.first[c + 1] - map.first[c];
  const Chan& h = ch[c];
  const int l = h.l;
  const int m = l + (l & 1);
  const int lp = (l + 8 * VE - 1) / (8 * VE) * (8 * VE);
  const int nv = lp / VE;
  T* Mw = (T*)h.G;
  T* Jw = (T*)h.Ri;
  // initial M = R^T (zero rows l..lp-1), J = I; each CTA a slice of columns
  for (int j = rank; j < l; j += ncta)
    for (int i = threadIdx.x; i < lp; i += blockDim.x) {
      __stcg(Mw + i + (int64_t)j * lp, (i < l) ? (T)h.R[j + (int64_t)i * l] : (T)0);
      if (WANT_J) __stcg(Jw + i + (int64_t)j * lp, (T)(i == j ? 1.0 : 0.0));
    }
  // rounds per sweep: the longest channel's
  int mmax = 2;
  for (int cc = 0; cc < map.C; ++cc) mmax = max(mmax, ch[cc].l + (ch[cc].l & 1));
  if (coop_stalled(ctl)) return;
  if (!coop_barrier(ws, map.nblocks, ctl)) return;
  const T eps = (sizeof(T) == 8) ? (T)1.1102230246251565e-16 : (T)5.9604645e-8;
  const T thr = (T)l * eps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane >> 3, gl = lane & 7;
  const int groups = (blockDim.x >> 5) * 4;
  const int npairs = m / 2;
  bool active = true;                      // this channel not yet converged
  int sweep = 0;
  for (; sweep < ctl.max_sweeps; ++sweep) {
    int rotated = 0;
    for (int r = 0; r < mmax - 1; ++r) {
      if (active && r < m - 1) {
        // the group loop is uniform across a warp (shuffles take all lanes);
        // groups past the last pair carry a = b = -1 and skip the work
        for (int base = rank * groups; base < npairs; base += ncta * groups) {
          const int pi = base + warp * 4 + grp;
          int a = -1, b = -1;
          if (pi < npairs) {
            if (pi == 0) { a = r; b = m - 1; }
            else {
              a = r + pi; if (a >= m - 1) a -= m - 1;
              b = r - pi; if (b < 0) b += m - 1;
            }
            if (a > b) { const int t = a; a = b; b = t; }
            if (b >= l) a = b = -1;                // the zero column of an odd l
          }
          V* ca = (V*)(Mw + (int64_t)(a < 0 ? 0 : a) * lp);
          V* cb = (V*)(Mw + (int64_t)(b < 0 ? 0 : b) * lp);
          T al = 0, be = 0, ga = 0;
          if (a >= 0)
            for (int v = gl; v < nv; v += 8) {
              const V x = __ldcg(ca + v), y = __ldcg(cb + v);
#pragma unroll
              for (int q = 0; q < VE; ++q) {
                const T xq = cget(x, q), yq = cget(y, q);
                al = fma(xq, xq, al); be = fma(yq, yq, be); ga = fma(xq, yq, ga);
              }
            }
#pragma unroll
          for (int o = 4; o > 0; o >>= 1) {
            al += __shfl_xor_sync(0xffffffffu, al, o);
            be += __shfl_xor_sync(0xffffffffu, be, o);
            ga += __shfl_xor_sync(0xffffffffu, ga, o);
          }
          if (a < 0 || ga == (T)0 || fabs(ga) <= thr * sqrt(al * be)) continue;
          const T zeta = (be - al) / (2 * ga);
          T t;
          if (fabs(zeta) > (T)1e15) t = (T)0.5 / zeta;
          else t = (zeta >= 0 ? (T)1 : (T)-1) / (fabs(zeta) + sqrt((T)1 + zeta * zeta));
          const T cs = (T)1 / sqrt((T)1 + t * t), sn = cs * t;
          for (int v = gl; v < nv; v += 8) {
            const V x = __ldcg(ca + v), y = __ldcg(cb + v);
            V nx, ny;
            T* px = (T*)&nx;
            T* py = (T*)&ny;
#pragma unroll
            for (int q = 0; q < VE; ++q) {
              const T xq = cget(x, q), yq = cget(y, q);
              px[q] = cs * xq - sn * yq;
              py[q] = sn * xq + cs * yq;
            }
            __stcg(ca + v, nx);
            __stcg(cb + v, ny);
          }
          if (WANT_J) {
            V* ja = (V*)(Jw + (int64_t)a * lp);
            V* jb = (V*)(Jw + (int64_t)b * lp);
            for (int v = gl; v < nv; v += 8) {
              const V x = __ldcg(ja + v), y = __ldcg(jb + v);
              V nx, ny;
              T* px = (T*)&nx;
              T* py = (T*)&ny;
#pragma unroll
              for (int q = 0; q < VE; ++q) {
                const T xq = cget(x, q), yq = cget(y, q);
                px[q] = cs * xq - sn * yq;
                py[q] = sn * xq + cs * yq;
              }
              __stcg(ja + v, nx);
              __stcg(jb + v, ny);
            }
          }
          rotated = 1;
        }
      }
      if (!coop_barrier(ws, map.nblocks, ctl)) return;
    }
    // sweep done: record, agree, stop when every channel is converged
    if (__syncthreads_or(rotated) && threadIdx.x == 0) atomicOr(ws + 4 + sweep * map.C + c, 1);
    if (!coop_barrier(ws, map.nblocks, ctl)) return;
    __shared__ int any;
    if (threadIdx.x == 0) {
      any = 0;
      for (int cc = 0; cc < map.C; ++cc) any |= *(volatile int*)(ws + 4 + sweep * map.C + cc);
    }
    __syncthreads();
    if (active && !*(volatile int*)(ws + 4 + sweep * map.C + c)) active = false;
    if (!any) { ++sweep; break; }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ws[3] = sweep;
}

// Column norms, sort (descending, ties by index), X = M_i / sigma_i, J, sigma.
template <typename T, bool WANT_J>
__global__ void __launch_bounds__(512) k_jacobi_coop_finish(const Chan* __restrict__ ch, const int* __restrict__ ws,
                                                             int max_sweeps) {
  constexpr int VE = CVec<T>::N;
  const Chan& h = ch[blockIdx.x];
  const int l = h.l;
  const int lp = (l + 8 * VE - 1) / (8 * VE) * (8 * VE);
  const T* Mw = (const T*)h.G;
  const T* Jw = (const T*)h.Ri;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const int sweeps = ws[3];
  if (threadIdx.x == 0) {
    h.res->sweeps = sweeps;
    if (sweeps >= max_sweeps && ws[4 + (max_sweeps - 1) * gridDim.x + blockIdx.x])
      atomicOr(&h.res->flags, FLAG_JACOBI_CAP);
    if (ws[2]) atomicOr(&h.res->flags, FLAG_JACOBI_CAP);
  }
  for (int cidx = warp; cidx < l; cidx += nwarp) {
    const T* cc = Mw + (int64_t)cidx * lp;
    double s = 0.0;
    for (int rr = lane; rr < l; rr += 32) s += (double)cc[rr] * (double)cc[rr];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) h.scr[cidx] = sqrt(s);
  }
  __syncthreads();
  for (int cidx = warp; cidx < l; cidx += nwarp) {
    const double si = h.scr[cidx];
    int rank = 0;
    for (int o = lane; o < l; o += 32) {
      const double so = h.scr[o];
      rank += (so > si) || (so == si && o < cidx);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
    const T* cc = Mw + (int64_t)cidx * lp;
    const double inv = si > 0.0 ? 1.0 / si : 0.0;
    for (int rr = lane; rr < l; rr += 32) h.M[rr + (int64_t)rank * l] = (double)cc[rr] * inv;
    if (WANT_J) {
      const T* jc = Jw + (int64_t)cidx * lp;
      for (int rr = lane; rr < l; rr += 32) h.J[rr + (int64_t)rank * l] = (double)jc[rr];
    }
    if (lane == 0) h.sig[rank] = si;
  }
}

// ---------------------------------------------------------------------------
// Cholesky G = R^T R (upper R, with the shifted retry of the single-CTA
// kernel), R -> h.R (or R_acc <- R R_acc) and R^{-1} (FP64) -> h.Ri, for
// large l on a cooperative grid.  Right-looking, one column per step: the
// channel's CTAs scale row j of the factor, then update the trailing upper
// triangle (one warp per column), a grid barrier after each phase.  The
// working factor lives in h.M (T, column-major, ld = l), read and written
// through L2.  ws: [0..2] barrier, [4 + a * C + c] channel c failed in attempt a.
template <typename T>
__global__ void __launch_bounds__(256) k_chol_coop(const Chan* __restrict__ ch, const __grid_constant__ CoopMap map,
                                                   int* __restrict__ ws, int accumulate, int conditional,
                                                   const CoopCtl ctl) {
  int c = 0;
  while (c + 1 < map.C && map.first[c + 1] <= (int)blockIdx.x) ++c;
  const int rank = blockIdx.x - map.first[c], ncta = map.first[c + 1] - map.first[c];
  const Chan& h = ch[c];
  const int l = h.l;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
  const int gt = rank * nt + tid, gstride = ncta * nt;
  const int gw = rank * nwarp + warp, wstride = ncta * nwarp;
  T* Ms = (T*)h.M;
  const double* G = h.G;
  int lmax = 1;
  for (int cc = 0; cc < map.C; ++cc) lmax = max(lmax, ch[cc].l);
  const bool on = !conditional || (h.res->flags & FLAG_SHIFTED);
  double shift = 0.0;
  {
    double tr = 0.0;
    for (int i = 0; i < l; ++i) tr += G[i + (int64_t)i * l];
    shift = 11.0 * ((double)h.n * l + (double)l * (l + 1)) *
            (sizeof(T) == 8 ? 1.1102230246251565e-16 : 5.9604644775390625e-08) * tr;
  }
  bool failed = false;
  for (int attempt = 0; attempt < 2; ++attempt) {
    // attempt 1 only for channels that failed attempt 0 (all CTAs agree)
    const bool work = on && (attempt == 0 || *(volatile int*)(ws + 4 + c) != 0);
    if (attempt == 1) {
      __shared__ int anyf;
      if (tid == 0) {
        anyf = 0;
        for (int cc = 0; cc < map.C; ++cc) anyf |= *(volatile int*)(ws + 4 + cc);
      }
      __syncthreads();
      if (!anyf) break;                                 // uniform across the grid
    }
    failed = false;
    if (work)
      for (int e = gt; e < l * l; e += gstride) {
        const int i = e % l, j = e / l;
        const double g = G[e] + ((attempt == 1 && i == j) ? shift : 0.0);
        __stcg(Ms + e, (T)g);
      }
    if (attempt == 0 && coop_stalled(ctl)) return;
    if (!coop_barrier(ws, map.nblocks, ctl)) return;
    for (int j = 0; j < lmax; ++j) {
      const bool act = work && !failed && j < l;
      if (act) {
        const T d = __ldcg(Ms + j + (int64_t)j * l);
        if (!(d > (T)0) || !isfinite(d)) {
          failed = true;
          if (rank == 0 && tid == 0) atomicExch(ws + 4 + attempt * map.C + c, 1);
        } else {
          const T rjj = sqrt(d), inv = (T)1 / rjj;
          for (int b = j + 1 + gt; b < l; b += gstride) {
            T* p = Ms + j + (int64_t)b * l;
            __stcg(p, __ldcg(p) * inv);
          }
        }
      }
      if (!coop_barrier(ws, map.nblocks, ctl)) return;
      if (act && !failed) {
        // the pivot is replaced only now: every CTA of the channel has read it
        if (rank == 0 && tid == 0) {
          T* pj = Ms + j + (int64_t)j * l;
          __stcg(pj, (T)sqrt(__ldcg(pj)));
        }
        for (int b = j + 1 + gw; b < l; b += wstride) {
          const T rb = __ldcg(Ms + j + (int64_t)b * l);
          T* colb = Ms + (int64_t)b * l;
          for (int a = j + 1 + lane; a <= b; a += 32)
            __stcg(colb + a, fma(-__ldcg(Ms + j + (int64_t)a * l), rb, __ldcg(colb + a)));
        }
      }
      if (!coop_barrier(ws, map.nblocks, ctl)) return;
    }
    if (work && attempt == 0 && failed && rank == 0 && tid == 0) atomicOr(&h.res->flags, FLAG_SHIFTED);
    // no early exit: if any channel retries, every CTA takes part in the
    // retry's barriers (the channels that succeeded idle through it)
    if (attempt == 0 && failed) failed = false;
  }
  if (!on) return;
  if (failed) {
    if (rank == 0 && tid == 0) atomicOr(&h.res->flags, FLAG_CHOL_FAIL);
    return;
  }
  // R (upper, zero below) -> h.R, or R_acc <- R R_acc (through h.G, free now)
  if (accumulate) {
    for (int e = gt; e < l * l; e += gstride) {
      const int i = e % l, jj = e / l;
      double s = 0.0;
      if (i <= jj)
        for (int k = i; k <= jj; ++k) s = fma((double)__ldcg(Ms + i + (int64_t)k * l), h.R[k + (int64_t)jj * l], s);
      h.G[e] = s;
    }
  }
  // R^{-1}: one warp per column (back substitution), FP64
  for (int cc = gw; cc < l; cc += wstride) {
    double* x = h.Ri + (int64_t)cc * l;
    for (int k = lane; k < l; k += 32) x[k] = (k == cc) ? 1.0 : 0.0;
    __syncwarp();
    for (int i = cc; i >= 0; --i) {
      const double xi = x[i] / (double)__ldcg(Ms + i + (int64_t)i * l);
      __syncwarp();
      if (lane == 0) x[i] = xi;
      const T* ri = Ms + (int64_t)i * l;
      for (int k = lane; k < i; k += 32) x[k] = fma(-(double)__ldcg(ri + k), xi, x[k]);
      __syncwarp();
    }
  }
  if (!accumulate)
    for (int e = gt; e < l * l; e += gstride) {
      const int i = e % l, jj = e / l;
      h.R[e] = (i <= jj) ? (double)__ldcg(Ms + e) : 0.0;
    }
}

// R_acc <- the product staged in h.G (after the grid-wide kernel boundary).
__global__ void __launch_bounds__(256) k_chol_coop_copy(const Chan* __restrict__ ch, int conditional) {
  const Chan& h = ch[blockIdx.y];
  if (conditional && !(h.res->flags & FLAG_SHIFTED)) return;
  if (h.res->flags & FLAG_CHOL_FAIL) return;
  const int64_t n = (int64_t)h.l * h.l;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    h.R[e] = h.G[e];
}

int jacobi_max_sweeps() {
  int v = 60;
  if (const char* e = getenv("RSVD_JACOBI_MAX_SWEEPS")) v = atoi(e);
  return v < 1 ? 1 : v > 60 ? 60 : v;
}

CoopCtl coop_ctl(int* err) {
  CoopCtl c{err, 1ll << 32, 0, jacobi_max_sweeps()};
  if (const char* e = getenv("RSVD_WAIT_CLOCKS")) {
    const long long v = atoll(e);
    if (v >= 0) c.budget = v;
  }
  if (const char* e = getenv("RSVD_TEST_STALL_BARRIER")) c.stall = atoi(e) == 1;
  return c;
}

static bool coop_map(const void* fn, const int* h_l, int C, CoopMap& map) {
  if (C < 1 || C > kCoopMaxChannels) return false;
  int dev = 0, nsm = 0, coop = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop || nsm < 1) return false;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, 256, 0) != cudaSuccess || per < 1) {
    cudaGetLastError();
    return false;
  }
  const int G = nsm * std::min(per, 2);
  if (G < C) return false;
  map = CoopMap{};
  map.C = C;
  double tot = 0.0;
  for (int c = 0; c < C; ++c) tot += (double)h_l[c] * h_l[c];
  std::vector<int> n(C);
  int given = 0;
  for (int c = 0; c < C; ++c) {
    n[c] = std::max(1, (int)((G - C) * ((double)h_l[c] * h_l[c] / tot)) + 1);
    given += n[c];
  }
  while (given > G) {
    int big = 0;
    for (int c = 1; c < C; ++c) if (n[c] > n[big]) big = c;
    --n[big];
    --given;
  }
  map.first[0] = 0;
  for (int c = 0; c < C; ++c) map.first[c + 1] = map.first[c] + n[c];
  map.nblocks = map.first[C];
  return true;
}

int launch_chol_coop(const Chan* d_ch, const int* h_l, int C, int accumulate, int f32_chol, int conditional,
                     int* coop_ws, int* err, cudaStream_t st) {
  if (!coop_ws) return -1;
  const void* fn = f32_chol ? (const void*)k_chol_coop<float> : (const void*)k_chol_coop<double>;
  CoopMap map;
  if (!coop_map(fn, h_l, C, map)) return -1;
  if (cudaMemsetAsync(coop_ws, 0, sizeof(int) * (4 + 2 * (size_t)C), st) != cudaSuccess) return -1;
  CoopCtl ctl = coop_ctl(err);
  void* args[] = {(void*)&d_ch, (void*)&map, (void*)&coop_ws, (void*)&accumulate, (void*)&conditional, (void*)&ctl};
  if (cudaLaunchCooperativeKernel(fn, dim3(map.nblocks), dim3(256), args, 0, st) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  note_launch();
  if (accumulate) {
    k_chol_coop_copy<<<dim3(32, C), 256, 0, st>>>(d_ch, conditional);
    note_launch();
  }
  return 0;
}

int launch_jacobi_coop(const Chan* d_ch, const int* h_l, int C, int fp32, int* coop_ws, int* err, cudaStream_t st) {
  if (!coop_ws) return -1;
  const void* fn = fp32 ? (const void*)k_jacobi_coop<float, false> : (const void*)k_jacobi_coop<double, true>;
  CoopMap map;
  if (!coop_map(fn, h_l, C, map)) return -1;
  const size_t wsb = sizeof(int) * (4 + (size_t)kCoopSweeps * C);
  if (cudaMemsetAsync(coop_ws, 0, wsb, st) != cudaSuccess) return -1;
  CoopCtl ctl = coop_ctl(err);
  if (ctl.max_sweeps > kCoopSweeps) ctl.max_sweeps = kCoopSweeps;   // the workspace holds kCoopSweeps flags
  void* args[] = {(void*)&d_ch, (void*)&map, (void*)&coop_ws, (void*)&ctl};
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(map.nblocks), dim3(256), args, 0, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  note_launch();
  if (fp32) k_jacobi_coop_finish<float, false><<<C, 512, 0, st>>>(d_ch, coop_ws, ctl.max_sweeps);
  else k_jacobi_coop_finish<double, true><<<C, 512, 0, st>>>(d_ch, coop_ws, ctl.max_sweeps);
  note_launch();
  return 0;
}

}  // namespace rsvd
