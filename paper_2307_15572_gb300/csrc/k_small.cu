// Per-channel kernels of the pipeline: ||V||_F^2, the FP64 random projection
// matrix, CholeskyQR's l x l factorisation, the one-sided Jacobi SVD of the
// small factor, rank selection and the sign convention.
#include <math.h>

#include "kernels.h"

namespace rsvd {

template <typename T>
RSVD_DEV T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum (fixed tree) of one value per thread; blockDim <= 1024.
RSVD_DEV double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (lane < nw) ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  if (threadIdx.x == 0) sh[0] = r;
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------- ||V||_F^2
__global__ void __launch_bounds__(256) k_fro2(const Chan* __restrict__ ch,
                                              const int* __restrict__ off, int C) {
  __shared__ double sh[32];
  const int t = blockIdx.x;
  const int c = find_chan(off, C, t);
  const Chan& h = ch[c];
  const int b = t - off[c];
  const int r0 = b * 64, r1 = min(h.n, r0 + 64);
  double s = 0.0;
  bool bad = false;
  for (int r = r0; r < r1; ++r) {
    const double* row = h.A + (int64_t)r * h.lda;
    for (int j = threadIdx.x; j < h.n; j += blockDim.x) {
      const double a = row[j];
      bad |= !isfinite(a);
      s = fma(a, a, s);
    }
  }
  s = block_sum(s, sh);
  if (bad) atomicOr(&h.res->flags, FLAG_NONFINITE);
  if (threadIdx.x == 0) h.fro_part[b] = s;
}

__global__ void k_fro2_reduce(const Chan* __restrict__ ch, int nparts_per_row_block) {
  __shared__ double sh[32];
  const Chan& h = ch[blockIdx.x];
  const int nb = (h.n + nparts_per_row_block - 1) / nparts_per_row_block;
  double s = 0.0, w = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    s += h.fro_part[i];
    if (h.wres_part) w += h.wres_part[i];
  }
  s = block_sum(s, sh);
  w = block_sum(w, sh);
  if (threadIdx.x == 0) {
    h.res->fro2 = s;
    h.res->wres2 = w;
  }
}

void launch_fro2(const Chan* d_ch, const int* d_off, int C, int tiles, cudaStream_t st) {
  if (tiles > 0) { k_fro2<<<tiles, 256, 0, st>>>(d_ch, d_off, C); note_launch(); }
}
void launch_fro2_reduce(const Chan* d_ch, int C, cudaStream_t st) {
  k_fro2_reduce<<<C, 256, 0, st>>>(d_ch, 64);
  note_launch();
}
void launch_fro2_reduce_rows(const Chan* d_ch, int C, int rows_per_part, cudaStream_t st) {
  k_fro2_reduce<<<C, 256, 0, st>>>(d_ch, rows_per_part);
  note_launch();
}

// ------------------------------------------------------------- Omega (FP64)
__global__ void __launch_bounds__(256) k_omega_f64(const Chan* __restrict__ ch,
                                                   const int* __restrict__ off, int C,
                                                   uint64_t seed, int col0, uint32_t tag) {
  const int t = blockIdx.x;
  const int c = find_chan(off, C, t);
  const Chan& h = ch[c];
  const int r0 = (t - off[c]) * 64;
  const int rows = min(64, h.n - r0);
  for (int e = threadIdx.x; e < 64 * h.l; e += blockDim.x) {
    const int rr = e & 63, j = e >> 6;
    if (rr < rows)
      h.X[(r0 + rr) + (int64_t)j * h.ldt] =
          gauss_f64(seed, (uint32_t)(r0 + rr), (uint32_t)(col0 + h.col0 + j), tag);
  }
}

void launch_omega_f64(const Chan* d_ch, const int* d_off, int C, int tiles, uint64_t seed,
                      int col0, cudaStream_t st, uint32_t tag) {
  if (tiles > 0) { k_omega_f64<<<tiles, 256, 0, st>>>(d_ch, d_off, C, seed, col0, tag); note_launch(); }
}

// ------------------------------------------------- Cholesky + inverse (FP64)
// G = R^T R with R upper triangular, right-looking: at step j, R_jj =
// sqrt(G_jj), row j of R = row j of the updated G / R_jj, and the trailing
// block is updated G_ab -= R_ja R_jb (independent FMAs, no long chains).  A
// non-positive pivot is a breakdown; the factorisation is then retried on
// G + s I with the shift of Fukaya, Kannan, Nakatsukasa, Yamamoto &
// Yanagisawa (SIAM J. Sci. Comput. 42, 2020), s = 11 (m l + l (l+1)) u tr(G),
// which keeps the shifted CholeskyQR well defined for kappa up to ~u^{-1}.
// Then R^{-1}: in FP64 (one thread per column, back substitution), or, for
// the mixed path, in FP32 row by row with all columns in parallel -- any
// invertible right factor leaves range(Y R^{-1}) = range(Y), and the second
// CholeskyQR round restores orthogonality.  If asked, R_acc <- R R_acc (the
// triangular factor of a repeated CholeskyQR).
// T = double: the ill-conditioned Grams (first CholeskyQR round, W^T W);
// T = float: the second CholeskyQR round, whose Gram is within ~1e-2 of I.
// In-place inverse of the upper triangular l x l matrix A (column-major,
// leading dimension lda, shared memory) by the whole block; rinv (l entries
// of shared memory) receives the reciprocals of the diagonal first.
// Column j: X_jj = 1 / A_jj, X[0:j, j] = -X_jj X[0:j, 0:j] A[0:j, j], where
// the leading block already holds X.  Each row of the product is split over g
// threads (2 while 2 l rows fit the block), reduced by shuffle.
// Rows are dealt to at most two passes of the block (l <= 2 nt; the callers'
// shared-memory bound keeps l below 256).
template <typename T>
RSVD_DEV void tri_inv_inplace(T* A, int lda, T* rinv, int l, int tid, int nt) {
  for (int i = tid; i < l; i += nt) rinv[i] = (T)1 / A[i + (int64_t)i * lda];
  __syncthreads();
  if (tid == 0) A[0] = rinv[0];
  __syncthreads();
  const int g = (2 * l <= nt) ? 2 : 1;
  const int p = tid % g;
  const int rstride = nt / g;
  for (int j = 1; j < l; ++j) {
    const T* aj = A + (int64_t)j * lda;
    T acc[2] = {(T)0, (T)0};
    int nrow = 0;
    for (int i = tid / g; i < j && nrow < 2; i += rstride, ++nrow) {
      T s0 = 0, s1 = 0;
      int k = i + p;
      for (; k + g < j; k += 2 * g) {
        s0 = fma(A[i + (int64_t)k * lda], aj[k], s0);
        s1 = fma(A[i + (int64_t)(k + g) * lda], aj[k + g], s1);
      }
      if (k < j) s0 = fma(A[i + (int64_t)k * lda], aj[k], s0);
      acc[nrow] = s0 + s1;
    }
    if (g == 2) {
      acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
      acc[1] += __shfl_xor_sync(0xffffffffu, acc[1], 1);
    }
    __syncthreads();                        // every read of column j is done
    const T xjj = rinv[j];
    nrow = 0;
    for (int i = tid / g; i < j && nrow < 2; i += rstride, ++nrow)
      if (p == 0) A[i + (int64_t)j * lda] = -acc[nrow] * xjj;
    if (tid == 0) A[j + (int64_t)j * lda] = xjj;   // column j is X from here on
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_chol_inv(const Chan* __restrict__ ch, int accumulate,
                                                  int use_smem, int f32_inverse, int conditional) {
  extern __shared__ __align__(16) unsigned char craw[];
  const Chan& h = ch[blockIdx.x];
  if (conditional && !(h.res->flags & FLAG_SHIFTED)) return;
  const int l = h.l;
  const int ld = use_smem ? l + 1 : l;       // odd stride: conflict-free column access
  T* Ms = use_smem ? (T*)craw : (T*)h.M;     // working copy of G -> R (column-major)
  const double* G = h.G;
  __shared__ int fail, s_bad;
  __shared__ double shift;
  __shared__ T s_rjj, s_inv;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) {
    fail = 0;
    double tr = 0.0;
    for (int i = 0; i < l; ++i) tr += G[i + (int64_t)i * l];
    shift = 11.0 * ((double)h.n * l + (double)l * (l + 1)) *
            (sizeof(T) == 8 ? 1.1102230246251565e-16 : 5.9604644775390625e-08) * tr;
  }
  __syncthreads();
  for (int attempt = 0; attempt < 2; ++attempt) {
    for (int e = tid; e < l * l; e += nt) {
      const int i = e % l, j = e / l;
      const double g = G[e] + ((attempt == 1 && i == j) ? shift : 0.0);
      Ms[i + (int64_t)j * ld] = (sizeof(T) == 8) ? (T)g : (T)f64_to_f32_rn(g);
    }
    int bad = 0;
    for (int j = 0; j < l; ++j) {
      __syncthreads();
      // the pivot's square root and reciprocal once, by one thread: on this
      // GPU an FP64 warp instruction costs the same with one lane or 32
      if (tid == 0) {
        const T d = Ms[j + (int64_t)j * ld];
        const int b = !(d > (T)0) || !isfinite(d);
        s_bad = b;
        if (!b) {
          const T r = sqrt(d);
          s_rjj = r;
          s_inv = (T)1 / r;
        }
      }
      __syncthreads();
      if (s_bad) { bad = 1; break; }                                // uniform across the block
      const T rjj = s_rjj, inv = s_inv;
      for (int i = j + tid; i < l; i += nt)
        Ms[j + (int64_t)i * ld] = (i == j) ? rjj : Ms[j + (int64_t)i * ld] * inv;
      __syncthreads();
      // trailing update, upper triangle: one warp per column b, lanes over a
      {
        const int w = tid >> 5, ln = tid & 31, nw = nt >> 5;
        for (int b = j + 1 + w; b < l; b += nw) {
          const T rb = Ms[j + (int64_t)b * ld];
          T* colb = Ms + (int64_t)b * ld;
          for (int a = j + 1 + ln; a <= b; a += 32) colb[a] = fma(-Ms[j + (int64_t)a * ld], rb, colb[a]);
        }
      }
    }
    __syncthreads();
    if (!bad) break;
    if (tid == 0) {
      if (attempt == 0) atomicOr(&h.res->flags, FLAG_SHIFTED);
      else { fail = 1; atomicOr(&h.res->flags, FLAG_CHOL_FAIL); }
    }
    __syncthreads();
    if (fail) break;
  }
  __syncthreads();
  if (fail) return;
  // R (upper, zero below) -> h.R, or R_acc <- R R_acc
  if (accumulate) {
    for (int e = tid; e < l * l; e += nt) {
      const int i = e % l, j = e / l;
      double s = 0.0;
      if (i <= j)
        for (int k = i; k <= j; ++k) s = fma((double)Ms[i + (int64_t)k * ld], h.R[k + (int64_t)j * l], s);
      h.G[e] = s;                               // G is free now
    }
    __syncthreads();
    for (int e = tid; e < l * l; e += nt) h.R[e] = h.G[e];
  } else {
    for (int e = tid; e < l * l; e += nt) {
      const int i = e % l, j = e / l;
      h.R[e] = (i <= j) ? (double)Ms[i + (int64_t)j * ld] : 0.0;
    }
  }
  __syncthreads();
  // R^{-1}.  In shared memory: in place, column by column from the left
  // (the unblocked triangular inverse): with the leading j x j block already
  // inverted, X_jj = 1 / R_jj and X[0:j, j] = -X_jj X[0:j, 0:j] R[0:j, j],
  // the rows of that triangular matrix-vector product in parallel (two
  // threads per row, each half of its terms, while rows fit).  Otherwise
  // (l past shared memory) one warp per column by back substitution.
  const int warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
  if ((f32_inverse || sizeof(T) == 4) && use_smem && l <= 2 * nt) {
    // FP32 arithmetic on an FP32 copy of R (stride l+1) in shared memory
    float* Rs;
    if (sizeof(T) == 4) {
      Rs = (float*)Ms;
    } else {
      // Ms is dead once h.R holds R: rebuild R in FP32 in the same space
      Rs = (float*)craw;
      for (int e = tid; e < l * l; e += nt) {
        const int i = e % l, j = e / l;
        h.Ri[e] = (i <= j) ? (double)Ms[i + (int64_t)j * ld] : 0.0;   // stage through global
      }
      __syncthreads();
      for (int e = tid; e < l * l; e += nt) {
        const int i = e % l, j = e / l;
        Rs[i + (int64_t)j * (l + 1)] = f64_to_f32_rn(h.Ri[e]);
      }
      __syncthreads();
    }
    float* rinv = Rs + (int64_t)l * (l + 1);
    tri_inv_inplace<float>(Rs, l + 1, rinv, l, tid, nt);
    for (int e = tid; e < l * l; e += nt) {
      const int i = e % l, j = e / l;
      h.Ri[e] = (i <= j) ? f32_to_f64(Rs[i + (int64_t)j * (l + 1)]) : 0.0;
    }
    return;
  }
  if (use_smem && sizeof(T) == 8 && l <= 2 * nt) {
    // FP64 in place; the reciprocals of the diagonal after the factor
    double* rinv = (double*)((unsigned char*)craw + (size_t)l * ld * sizeof(T));
    tri_inv_inplace<T>(Ms, ld, (T*)rinv, l, tid, nt);
    for (int e = tid; e < l * l; e += nt) {
      const int i = e % l, j = e / l;
      h.Ri[e] = (i <= j) ? (double)Ms[i + (int64_t)j * ld] : 0.0;
    }
    return;
  }
  // large l, R in global memory: the column itself (in h.Ri) as the work
  // vector; the reciprocals of the diagonal in G (free once R exists)
  double* rinv = (double*)h.G;
  for (int i = tid; i < l; i += nt) rinv[i] = 1.0 / (double)Ms[i + (int64_t)i * ld];
  __syncthreads();
  for (int c = warp; c < l; c += nwarp) {
    double* x = h.Ri + (int64_t)c * l;
    for (int k = lane; k < l; k += 32) x[k] = (k == c) ? 1.0 : 0.0;
    __syncwarp();
    for (int i = c; i >= 0; --i) {
      const double xi = x[i] * rinv[i];
      __syncwarp();
      if (lane == 0) x[i] = xi;
      const T* ri = Ms + (int64_t)i * ld;
      for (int k = lane; k < i; k += 32) x[k] = fma(-(double)ri[k], xi, x[k]);
      __syncwarp();
    }
  }
}

// ------------------------------- register-resident Cholesky + inverse, l <= 128
// The same factorisation, shift retry and inverse as k_chol_inv, for
// factors of at most 128 columns, with the matrix in registers: thread
// (ta, tb) of a 16 x 16 grid holds the upper-triangle elements
// (ta + 16 p, tb + 16 q), p <= q < 8 (36 blocks; on p == q those with
// ta <= tb).  Step j of the right-looking factorisation: the owner of (j, j)
// forms R_jj and its reciprocal; the owners of row j scale it and publish
// it to shared memory; every thread updates its elements below and right of
// the pivot from the published row (independent FMAs on registers).  The
// inverse X = R^{-1} then overwrites R in the same registers, rows from the
// bottom: X_i,: <- X_i,: / R_ii (X_ii = 1 / R_ii), publish row i of X and
// column i of R (still R above the diagonal), and X_ab -= R_ai X_ib for
// a < i <= b (with X_ai starting from 0); the published vectors alternate
// between two buffers, so one barrier per step suffices.
__host__ __device__ constexpr int blk36(int p, int q) { return q * (q + 1) / 2 + p; }

template <typename U>
RSVD_DEV U to_u(double v) { return (U)v; }
template <>
RSVD_DEV float to_u<float>(double v) { return f64_to_f32_rn(v); }
RSVD_DEV double u_to_f64(double v) { return v; }
RSVD_DEV double u_to_f64(float v) { return f32_to_f64(v); }

// X = R^{-1} in place (registers x, layout as above); rinv (shared) holds
// 1 / R_ii in U precision on entry.
template <typename U>
RSVD_DEV void reg_tri_inv(U (&x)[36], const U* rinv, U (*rowx)[128], U (*colr)[128], int l, int ta, int tb) {
#pragma unroll
  for (int pi = 7; pi >= 0; --pi) {
    if (16 * pi >= l) continue;
    for (int ti = 15; ti >= 0; --ti) {
      const int i = 16 * pi + ti;
      if (i >= l) continue;
      const int buf = i & 1;
      const U ri = rinv[i];
      if (ta == ti) {                          // row i of X: scale, publish (b >= i)
#pragma unroll
        for (int q = pi; q < 8; ++q) {
          const int b = tb + 16 * q;
          if (b >= i && b < l) {
            U v = (b == i) ? ri : x[blk36(pi, q)] * ri;
            x[blk36(pi, q)] = v;
            rowx[buf][b] = v;
          }
        }
      }
      if (tb == ti) {                          // column i of R above the diagonal
#pragma unroll
        for (int p = 0; p <= pi; ++p) {
          const int a = ta + 16 * p;
          if (a < i) colr[buf][a] = x[blk36(p, pi)];
        }
      }
      __syncthreads();
      U cr[8];
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        const int a = ta + 16 * p;
        cr[p] = (p <= pi && a < i) ? colr[buf][a] : (U)0;
      }
#pragma unroll
      for (int q = pi; q < 8; ++q) {
        const int b = tb + 16 * q;
        if (b < i || b >= l) continue;
        const U xb = rowx[buf][b];
#pragma unroll
        for (int p = 0; p <= q; ++p) {
          const int a = ta + 16 * p;
          if (p <= pi && a < i && a <= b) {
            const U base = (b == i) ? (U)0 : x[blk36(p, q)];
            x[blk36(p, q)] = fma(-cr[p], xb, base);
          }
        }
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_chol_inv_reg(const Chan* __restrict__ ch, int f32_inverse,
                                                      int conditional) {
  const Chan& h = ch[blockIdx.x];
  if (conditional && !(h.res->flags & FLAG_SHIFTED)) return;
  const int l = h.l;
  const double* G = h.G;
  const int tid = threadIdx.x, ta = tid & 15, tb = tid >> 4;
  __shared__ T rowb[128];
  __shared__ T rinv_t[128];
  __shared__ __align__(16) unsigned char ibuf[2 * 2 * 128 * sizeof(double) + 128 * sizeof(double)];
  __shared__ int s_bad, fail;
  __shared__ double s_shift;
  if (tid < 32) {
    double tr = 0.0;
    for (int i = tid; i < l; i += 32) tr += G[i + (int64_t)i * l];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if (tid == 0) {
      fail = 0;
      s_shift = 11.0 * ((double)h.n * l + (double)l * (l + 1)) *
                (sizeof(T) == 8 ? 1.1102230246251565e-16 : 5.9604644775390625e-08) * tr;
    }
  }
  __syncthreads();
  T r[36];
  int bad = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int p = 0; p <= q; ++p) {
        const int a = ta + 16 * p, b = tb + 16 * q;
        T v = (T)0;
        if (a <= b && b < l) {
          double g = G[a + (int64_t)b * l];
          if (attempt == 1 && a == b) g += s_shift;
          v = to_u<T>(g);
        }
        r[blk36(p, q)] = v;
      }
    bad = 0;
#pragma unroll
    for (int pj = 0; pj < 8; ++pj) {
      if (16 * pj >= l || bad) continue;
      for (int tj = 0; tj < 16; ++tj) {
        const int j = 16 * pj + tj;
        if (j >= l) break;
        if (ta == tj && tb == tj) {            // the pivot, once
          const T d = r[blk36(pj, pj)];
          const int b0 = !(d > (T)0) || !isfinite(d);
          s_bad = b0;
          if (!b0) {
            const T rjj = sqrt(d);
            rinv_t[j] = (T)1 / rjj;
            r[blk36(pj, pj)] = rjj;
          }
        }
        __syncthreads();
        if (s_bad) { bad = 1; break; }         // uniform across the block
        if (ta == tj) {                        // row j: scale, publish
          const T inv = rinv_t[j];
#pragma unroll
          for (int q = pj; q < 8; ++q) {
            const int b = tb + 16 * q;
            if (b > j && b < l) {
              const T v = r[blk36(pj, q)] * inv;
              r[blk36(pj, q)] = v;
              rowb[b] = v;
            }
          }
        }
        __syncthreads();
        T ra[8], rbq[8];
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          const int a = ta + 16 * p, b = tb + 16 * p;
          ra[p] = (p >= pj && a > j && a < l) ? rowb[a] : (T)0;
          rbq[p] = (p >= pj && b > j && b < l) ? rowb[b] : (T)0;
        }
#pragma unroll
        for (int q = pj; q < 8; ++q)
#pragma unroll
          for (int p = pj; p <= q; ++p) {
            const int a = ta + 16 * p, b = tb + 16 * q;
            if (a > j && a <= b && b < l) r[blk36(p, q)] = fma(-ra[p], rbq[q], r[blk36(p, q)]);
          }
      }
    }
    __syncthreads();
    if (!bad) break;
    if (tid == 0) {
      if (attempt == 0) atomicOr(&h.res->flags, FLAG_SHIFTED);
      else { fail = 1; atomicOr(&h.res->flags, FLAG_CHOL_FAIL); }
    }
    __syncthreads();
    if (fail) return;
  }
  // R (upper, zero below) -> h.R
#pragma unroll
  for (int q = 0; q < 8; ++q)
#pragma unroll
    for (int p = 0; p <= q; ++p) {
      const int a = ta + 16 * p, b = tb + 16 * q;
      if (a <= b && b < l) h.R[a + (int64_t)b * l] = u_to_f64(r[blk36(p, q)]);
    }
  for (int b = tb; b < l; b += 16)
    for (int a = ta; a < l; a += 16)
      if (a > b) { h.R[a + (int64_t)b * l] = 0.0; h.Ri[a + (int64_t)b * l] = 0.0; }
  // R^{-1} -> h.Ri: FP32 on the mixed path (any invertible right factor keeps
  // the range; the next CholeskyQR round restores orthogonality), else T
  if (f32_inverse || sizeof(T) == 4) {
    float x[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) x[k] = (sizeof(T) == 4) ? (float)r[k] : to_u<float>((double)r[k]);
    float* rinv = (float*)(ibuf + 2 * 2 * 128 * sizeof(float));
    if (ta == tb) {
#pragma unroll
      for (int p = 0; p < 8; ++p)
        if (ta + 16 * p < l) rinv[ta + 16 * p] = 1.0f / x[blk36(p, p)];
    }
    __syncthreads();
    float (*rowx)[128] = (float (*)[128])ibuf;
    float (*colr)[128] = (float (*)[128])(ibuf + 2 * 128 * sizeof(float));
    reg_tri_inv<float>(x, rinv, rowx, colr, l, ta, tb);
    float* ri32 = h.Ri32;
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int p = 0; p <= q; ++p) {
        const int a = ta + 16 * p, b = tb + 16 * q;
        if (a <= b && b < l) {
          h.Ri[a + (int64_t)b * l] = f32_to_f64(x[blk36(p, q)]);
          if (ri32) ri32[a + (int64_t)b * l] = x[blk36(p, q)];
        }
      }
    if (ri32)
      for (int b = tb; b < l; b += 16)
        for (int a = ta; a < l; a += 16)
          if (a > b) ri32[a + (int64_t)b * l] = 0.0f;
  } else {
    double* rinv = (double*)(ibuf + 2 * 2 * 128 * sizeof(double));
    if (ta == tb) {
#pragma unroll
      for (int p = 0; p < 8; ++p)
        if (ta + 16 * p < l) rinv[ta + 16 * p] = 1.0 / (double)r[blk36(p, p)];
    }
    __syncthreads();
    double x[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) x[k] = (double)r[k];
    double (*rowx)[128] = (double (*)[128])ibuf;
    double (*colr)[128] = (double (*)[128])(ibuf + 2 * 128 * sizeof(double));
    reg_tri_inv<double>(x, rinv, rowx, colr, l, ta, tb);
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int p = 0; p <= q; ++p) {
        const int a = ta + 16 * p, b = tb + 16 * q;
        if (a <= b && b < l) h.Ri[a + (int64_t)b * l] = x[blk36(p, q)];
      }
  }
}

// The mixed path's factor in double-float arithmetic (pairs hi + lo of FP32
// numbers, about 48 significant bits; Dekker, 1971, and the TwoSum of Knuth;
// the trailing update keeps each pair in the unnormalised Sum2 form below
// until its row is the pivot row).  Same register layout, pivot order, shift and
// retry as k_chol_inv_reg, with every FP64 operation of the column steps
// replaced by FP32 instructions (this part issues FP64 arithmetic at a small
// fraction of its FP32 rate).  The Gram is first scaled by an exact power of
// two 2^(2k) that brings its largest diagonal entry into [1, 4), so that the
// lo parts stay normal FP32 numbers; R = R' 2^-k and R^{-1} = R'^{-1} 2^k.
// 48 bits match the accuracy of the tensor-core Gram it factors (six 8-bit
// slices), and the factor feeds an FP32 product and an FP32 Jacobi; the FP64
// path keeps k_chol_inv_reg<double>.  The inverse is the FP32 one of the
// mixed path, from R' rounded to FP32.
RSVD_DEV void df_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
RSVD_DEV void df_fast_two_sum(float a, float b, float& s, float& e) {   // |a| >= |b| or a = 0
  s = a + b;
  e = b - (s - a);
}
// (xh, xl) (yh, yl), normalised
RSVD_DEV void df_mul(float xh, float xl, float yh, float yl, float& rh, float& rl) {
  const float pr = xh * yh;
  float e = fmaf(xh, yh, -pr);
  e = fmaf(xh, yl, e);
  e = fmaf(xl, yh, e);
  df_fast_two_sum(pr, e, rh, rl);
}
// (ah, al) -= (xh, xl) (yh, yl), leaving the pair unnormalised: ah is the
// running FP32 sum and al collects every rounding error (the TwoSum error
// and the product's error terms), as in Sum2 / Dot2 of Ogita, Rump & Oishi
// (2005); the pair is renormalised once, when its row becomes the pivot row.
RSVD_DEV void df_fnms_lazy(float& ah, float& al, float xh, float xl, float yh, float yl) {
  const float pr = xh * yh;
  float e = fmaf(xh, yh, -pr);
  e = fmaf(xh, yl, e);
  e = fmaf(xl, yh, e);
  float sh, sl;
  df_two_sum(ah, -pr, sh, sl);
  ah = sh;
  al += sl - e;
}
RSVD_DEV void df_from_f64(double g, float& h, float& l) {
  h = f64_to_f32_rn(g);
  l = f64_to_f32_rn(g - f32_to_f64(h));
}

__global__ void __launch_bounds__(256, 1) k_chol_df(const Chan* __restrict__ ch, int conditional) {
  const Chan& h = ch[blockIdx.x];
  if (conditional && !(h.res->flags & FLAG_SHIFTED)) return;
  const int l = h.l;
  const double* G = h.G;
  const int tid = threadIdx.x, ta = tid & 15, tb = tid >> 4;
  __shared__ float rowh[128], rowl[128];
  __shared__ float rih[128], ril[128];
  __shared__ __align__(16) unsigned char ibuf[2 * 2 * 128 * sizeof(float) + 128 * sizeof(float)];
  __shared__ int s_bad, fail, s_k;
  __shared__ double s_shift;
  if (tid < 32) {
    double tr = 0.0, mx = 0.0;
    for (int i = tid; i < l; i += 32) {
      const double d = G[i + (int64_t)i * l];
      tr += d;
      mx = fmax(mx, d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      tr += __shfl_xor_sync(0xffffffffu, tr, o);
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (tid == 0) {
      fail = 0;
      // ilogb of the largest diagonal entry from its exponent field; zero,
      // subnormal or non-finite maxima keep the scale 1 (the factor fails)
      const int ex = (int)((__double_as_longlong(mx) >> 52) & 0x7FF);
      const int k = (ex == 0 || ex == 0x7FF) ? 0 : -((ex - 1023) >> 1);
      s_k = k;
      s_shift = ldexp(11.0 * ((double)h.n * l + (double)l * (l + 1)) * 3.552713678800501e-15 * tr, 2 * k);
    }
  }
  __syncthreads();
  const int k2 = 2 * s_k;
  float rh[36], rl[36];
  int bad = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int p = 0; p <= q; ++p) {
        const int a = ta + 16 * p, b = tb + 16 * q;
        float vh = 0.0f, vl = 0.0f;
        if (a <= b && b < l) {
          double g = ldexp(G[a + (int64_t)b * l], k2);
          if (attempt == 1 && a == b) g += s_shift;
          df_from_f64(g, vh, vl);
        }
        rh[blk36(p, q)] = vh;
        rl[blk36(p, q)] = vl;
      }
    bad = 0;
#pragma unroll
    for (int pj = 0; pj < 8; ++pj) {
      if (16 * pj >= l || bad) continue;
      for (int tj = 0; tj < 16; ++tj) {
        const int j = 16 * pj + tj;
        if (j >= l) break;
        if (ta == tj && tb == tj) {            // the pivot, once: R_jj = sqrt(d), 1 / R_jj in double-float
          float dh, dl;
          df_two_sum(rh[blk36(pj, pj)], rl[blk36(pj, pj)], dh, dl);
          const int b0 = !(dh > 0.0f) || !isfinite(dh);
          s_bad = b0;
          if (!b0) {
            const float sq = __fsqrt_rn(dh);   // one Newton step on sq^2 = d
            const float pr = sq * sq;
            const float pe = fmaf(sq, sq, -pr);
            const float c = (((dh - pr) - pe) + dl) * (0.5f / sq);
            float jh, jl;
            df_fast_two_sum(sq, c, jh, jl);
            const float iv = __frcp_rn(jh);    // one Newton step on R_jj x = 1
            const float er = fmaf(-jh, iv, 1.0f) - jl * iv;
            float ih, il;
            df_fast_two_sum(iv, er * iv, ih, il);
            rih[j] = ih;
            ril[j] = il;
            rh[blk36(pj, pj)] = jh;
            rl[blk36(pj, pj)] = jl;
          }
        }
        __syncthreads();
        if (s_bad) { bad = 1; break; }         // uniform across the block
        if (ta == tj) {                        // row j: scale, publish
          const float ih = rih[j], il = ril[j];
#pragma unroll
          for (int q = pj; q < 8; ++q) {
            const int b = tb + 16 * q;
            if (b > j && b < l) {
              float uh, ul, vh, vl;
              df_two_sum(rh[blk36(pj, q)], rl[blk36(pj, q)], uh, ul);
              df_mul(uh, ul, ih, il, vh, vl);
              rh[blk36(pj, q)] = vh;
              rl[blk36(pj, q)] = vl;
              rowh[b] = vh;
              rowl[b] = vl;
            }
          }
        }
        __syncthreads();
        float rah[8], ral[8], rbh[8], rbl[8];
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          const int a = ta + 16 * p, b = tb + 16 * p;
          const bool ua = p >= pj && a > j && a < l, ub = p >= pj && b > j && b < l;
          rah[p] = ua ? rowh[a] : 0.0f;
          ral[p] = ua ? rowl[a] : 0.0f;
          rbh[p] = ub ? rowh[b] : 0.0f;
          rbl[p] = ub ? rowl[b] : 0.0f;
        }
#pragma unroll
        for (int q = pj; q < 8; ++q)
#pragma unroll
          for (int p = pj; p <= q; ++p) {
            const int a = ta + 16 * p, b = tb + 16 * q;
            if (a > j && a <= b && b < l)
              df_fnms_lazy(rh[blk36(p, q)], rl[blk36(p, q)], rah[p], ral[p], rbh[q], rbl[q]);
          }
      }
    }
    __syncthreads();
    if (!bad) break;
    if (tid == 0) {
      if (attempt == 0) atomicOr(&h.res->flags, FLAG_SHIFTED);
      else { fail = 1; atomicOr(&h.res->flags, FLAG_CHOL_FAIL); }
    }
    __syncthreads();
    if (fail) return;
  }
  const int k = s_k;
  // R = (hi + lo) 2^-k (upper, zero below) -> h.R
#pragma unroll
  for (int q = 0; q < 8; ++q)
#pragma unroll
    for (int p = 0; p <= q; ++p) {
      const int a = ta + 16 * p, b = tb + 16 * q;
      if (a <= b && b < l)
        h.R[a + (int64_t)b * l] = ldexp(f32_to_f64(rh[blk36(p, q)]) + f32_to_f64(rl[blk36(p, q)]), -k);
    }
  for (int b = tb; b < l; b += 16)
    for (int a = ta; a < l; a += 16)
      if (a > b) { h.R[a + (int64_t)b * l] = 0.0; h.Ri[a + (int64_t)b * l] = 0.0; }
  // R^{-1} = R'^{-1} 2^k in FP32 from R' rounded to FP32 (its hi parts)
  float* rinv = (float*)(ibuf + 2 * 2 * 128 * sizeof(float));
  if (ta == tb) {
#pragma unroll
    for (int p = 0; p < 8; ++p)
      if (ta + 16 * p < l) rinv[ta + 16 * p] = 1.0f / rh[blk36(p, p)];
  }
  __syncthreads();
  float (*rowx)[128] = (float (*)[128])ibuf;
  float (*colr)[128] = (float (*)[128])(ibuf + 2 * 128 * sizeof(float));
  reg_tri_inv<float>(rh, rinv, rowx, colr, l, ta, tb);
  float* ri32 = h.Ri32;
#pragma unroll
  for (int q = 0; q < 8; ++q)
#pragma unroll
    for (int p = 0; p <= q; ++p) {
      const int a = ta + 16 * p, b = tb + 16 * q;
      if (a <= b && b < l) {
        const float x = ldexpf(rh[blk36(p, q)], k);
        h.Ri[a + (int64_t)b * l] = f32_to_f64(x);
        if (ri32) ri32[a + (int64_t)b * l] = x;
      }
    }
  if (ri32)
    for (int b = tb; b < l; b += 16)
      for (int a = ta; a < l; a += 16)
        if (a > b) ri32[a + (int64_t)b * l] = 0.0f;
}

void launch_chol_inv(const Chan* d_ch, int C, int accumulate, int max_l, int f32_inverse,
                     cudaStream_t st, int f32_chol, int conditional) {
  // the factor (stride l+1) and the l reciprocals of its diagonal; the FP32
  // inverse of large l also keeps 8 work vectors
  const size_t esz = f32_chol ? sizeof(float) : sizeof(double);
  size_t bytes = (size_t)max_l * (max_l + 1) * esz + (size_t)max_l * sizeof(double);
  const size_t b32 = (size_t)max_l * (max_l + 1) * sizeof(float) + 9 * (size_t)max_l * sizeof(float);
  if (b32 > bytes) bytes = b32;
  const int use_smem = bytes <= 200 * 1024;
  if (max_l <= 128 && !accumulate) {
    if (f32_chol) k_chol_inv_reg<float><<<C, 256, 0, st>>>(d_ch, 1, conditional);
    else if (f32_inverse) k_chol_df<<<C, 256, 0, st>>>(d_ch, conditional);     // the mixed path
    else k_chol_inv_reg<double><<<C, 256, 0, st>>>(d_ch, 0, conditional);
    note_launch();
    return;
  }
  if (f32_chol) {
    if (use_smem) {
      cudaFuncSetAttribute(k_chol_inv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      k_chol_inv<float><<<C, 256, bytes, st>>>(d_ch, accumulate, 1, 1, conditional);
    } else {
      k_chol_inv<float><<<C, 256, 0, st>>>(d_ch, accumulate, 0, 1, conditional);
    }
  } else {
    if (use_smem) {
      cudaFuncSetAttribute(k_chol_inv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      k_chol_inv<double><<<C, 256, bytes, st>>>(d_ch, accumulate, 1, f32_inverse, conditional);
    } else {
      k_chol_inv<double><<<C, 256, 0, st>>>(d_ch, accumulate, 0, f32_inverse, conditional);
    }
  }
  note_launch();
}

// ------------------------------------------------ one-sided Jacobi (Hestenes)
// Orthogonalise the columns of M = R^T by plane rotations on column pairs.
// For a pair with alpha = |m_i|^2, beta = |m_j|^2, gamma = m_i.m_j the
// rotation zeta = (beta - alpha)/(2 gamma), t = sign(zeta)/(|zeta| +
// sqrt(1 + zeta^2)), c = 1/sqrt(1+t^2), s = c t makes them orthogonal
// (Golub & Van Loan, 4th ed., Sec. 8.6.3).  Pairs are scheduled in parallel
// rounds by the round-robin ("circle") ordering of Brent & Luk (1985): in
// round r of m-1 rounds, index m-1 meets r and (r+i) meets (r-i) mod (m-1);
// every pair occurs once per sweep and the pairs of a round are disjoint, so
// one warp per pair runs without synchronisation inside the round.  Sweeps
// repeat until no pair exceeds |gamma| <= l eps sqrt(alpha beta) (or a cap).
// Result: M J = X Sigma with X orthonormal, so R^T = X Sigma J^T.
template <typename T> struct Vec2;
template <> struct Vec2<float> { typedef float4 V; static constexpr int N = 4; };
template <> struct Vec2<double> { typedef double2 V; static constexpr int N = 2; };

RSVD_DEV float vget(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
RSVD_DEV double vget(const double2& v, int i) { return i == 0 ? v.x : v.y; }

// Sweep count and flags; sigma_i = |M_i| sorted descending (ties by index),
// X = M_i / sigma_i, Z = J_i into the channel's buffers.
// M32 (and the channel has its FP32 scratch Ri32): store the sorted columns
// M_i unnormalised as FP32 (exact copies of the FP32 Jacobi columns) in h.M's
// buffer instead of X = M_i / sigma_i in FP64.
template <typename T, bool WANT_J, bool M32 = false>
RSVD_DEV void jacobi_finish(const Chan& h, const T* Mw, const T* Jw, int lp, int l, int sweep, int max_sweeps) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  if (threadIdx.x == 0) {
    h.res->sweeps = sweep + 1;
    if (sweep >= max_sweeps) atomicOr(&h.res->flags, FLAG_JACOBI_CAP);
  }
  __syncthreads();
  // column norms (unsorted) into scratch
  for (int cidx = warp; cidx < l; cidx += nwarp) {
    const T* cc = Mw + (int64_t)cidx * lp;
    double s = 0.0;
    for (int rr = lane; rr < l; rr += 32) s += (double)cc[rr] * (double)cc[rr];
    s = warp_sum(s);
    if (lane == 0) h.scr[cidx] = sqrt(s);
  }
  __syncthreads();
  // rank sort, descending, ties by index; write sigma, X = M_i / sigma_i, Z = J_i
  for (int cidx = warp; cidx < l; cidx += nwarp) {
    const double si = h.scr[cidx];
    int rank = 0;
    for (int o = lane; o < l; o += 32) {
      const double so = h.scr[o];
      rank += (so > si) || (so == si && o < cidx);
    }
    rank = warp_sum(rank);
    const T* cc = Mw + (int64_t)cidx * lp;
    const double inv = si > 0.0 ? 1.0 / si : 0.0;
    if (M32 && h.Ri32) {                    // the FP32 re-orthonormalisation follows (see reorth_x)
      float* m32 = (float*)h.M;
      for (int rr = lane; rr < l; rr += 32) m32[rr + (int64_t)rank * l] = (float)cc[rr];
    } else {
      for (int rr = lane; rr < l; rr += 32) h.M[rr + (int64_t)rank * l] = (double)cc[rr] * inv;
    }
    if (WANT_J) {
      const T* jc = Jw + (int64_t)cidx * lp;
      for (int rr = lane; rr < l; rr += 32) h.J[rr + (int64_t)rank * l] = (double)jc[rr];
    }
    if (lane == 0) h.sig[rank] = si;
  }
}

// Columns are stored with stride lp = round_up(l, 8 vectors), rows l..lp-1
// zero, so each 8-lane group moves 128 contiguous bytes per access
// (conflict-free) with 16-byte vector loads.
template <typename T, bool WANT_J>
__global__ void __launch_bounds__(512) k_jacobi(const Chan* __restrict__ ch, int use_smem,
                                                int max_sweeps) {
  typedef typename Vec2<T>::V V;
  constexpr int VE = Vec2<T>::N;
  extern __shared__ __align__(16) unsigned char sraw[];
  const Chan& h = ch[blockIdx.x];
  const int l = h.l;
  const int m = l + (l & 1);                       // even count; index l (if odd) is a zero column
  const int lp = (l + 8 * VE - 1) / (8 * VE) * (8 * VE);
  const int nv = lp / VE;                          // vectors per column
  T* Mw;
  T* Jw;
  if (use_smem) { Mw = (T*)sraw; Jw = Mw + (int64_t)l * lp; }
  else { Mw = (T*)h.G; Jw = (T*)h.Ri; }            // G and R^{-1} (sized l x (l+32)) are free here
  for (int e = threadIdx.x; e < lp * l; e += blockDim.x) {
    const int i = e % lp, j = e / lp;
    Mw[e] = (i < l) ? (T)h.R[j + (int64_t)i * l] : (T)0;      // M = R^T
    if (WANT_J) Jw[e] = (T)(i == j ? 1.0 : 0.0);
  }
  __syncthreads();
  const T eps = (sizeof(T) == 8) ? (T)1.1102230246251565e-16 : (T)5.9604645e-8;
  const T thr = (T)l * eps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const int grp = lane >> 3, gl = lane & 7;        // four 8-lane groups per warp, one pair each
  const int npairs = m / 2;
  const int per_pass = nwarp * 4;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    int rotated = 0;
    for (int r = 0; r < m - 1; ++r) {
      for (int base = 0; base < npairs; base += per_pass) {
        const int pi = base + warp * 4 + grp;
        int a = -1, b = -1;
        if (pi < npairs) {
          if (pi == 0) { a = r; b = m - 1; }
          else {
            a = r + pi; if (a >= m - 1) a -= m - 1;
            b = r - pi; if (b < 0) b += m - 1;
          }
          if (a > b) { const int t = a; a = b; b = t; }
          if (b >= l) a = b = -1;
        }
        T al = 0, be = 0, ga = 0;
        V* ca = (V*)(Mw + (int64_t)(a < 0 ? 0 : a) * lp);
        V* cb = (V*)(Mw + (int64_t)(b < 0 ? 0 : b) * lp);
        if (a >= 0)
          for (int v = gl; v < nv; v += 8) {
            const V x = ca[v], y = cb[v];
#pragma unroll
            for (int q = 0; q < VE; ++q) {
              const T xq = vget(x, q), yq = vget(y, q);
              al = fma(xq, xq, al); be = fma(yq, yq, be); ga = fma(xq, yq, ga);
            }
          }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {          // reduce inside the 8-lane group
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (a < 0 || ga == (T)0 || fabs(ga) <= thr * sqrt(al * be)) continue;
        T t, cs;
        if (sizeof(T) == 4) {
          const float zeta = __fdividef((float)(be - al), (float)(2 * ga));
          const float az = fabsf(zeta);
          float tf = az > 1e15f ? __fdividef(0.5f, az) : __fdividef(1.0f, az + sqrtf(fmaf(zeta, zeta, 1.0f)));
          tf = zeta >= 0.0f ? tf : -tf;
          t = (T)tf;
          cs = (T)rsqrtf(fmaf(tf, tf, 1.0f));
        } else {
          const T zeta = (be - al) / (2 * ga);
          if (fabs(zeta) > (T)1e15) t = (T)0.5 / zeta;
          else t = (zeta >= 0 ? (T)1 : (T)-1) / (fabs(zeta) + sqrt((T)1 + zeta * zeta));
          cs = (T)1 / sqrt((T)1 + t * t);
        }
        const T sn = cs * t;
        for (int v = gl; v < nv; v += 8) {
          V x = ca[v], y = cb[v];
          V nx, ny;
          T* px = (T*)&nx;
          T* py = (T*)&ny;
#pragma unroll
          for (int q = 0; q < VE; ++q) {
            const T xq = vget(x, q), yq = vget(y, q);
            px[q] = cs * xq - sn * yq;
            py[q] = sn * xq + cs * yq;
          }
          ca[v] = nx;
          cb[v] = ny;
        }
        if (WANT_J) {
          V* ja = (V*)(Jw + (int64_t)a * lp);
          V* jb = (V*)(Jw + (int64_t)b * lp);
          for (int v = gl; v < nv; v += 8) {
            V x = ja[v], y = jb[v];
            V nx, ny;
            T* px = (T*)&nx;
            T* py = (T*)&ny;
#pragma unroll
            for (int q = 0; q < VE; ++q) {
              const T xq = vget(x, q), yq = vget(y, q);
              px[q] = cs * xq - sn * yq;
              py[q] = sn * xq + cs * yq;
            }
            ja[v] = nx;
            jb[v] = ny;
          }
        }
        rotated = 1;
      }
      if (r < m - 2) __syncthreads();
    }
    if (!__syncthreads_or(rotated)) break;     // also the barrier after the last round
  }
  jacobi_finish<T, WANT_J>(h, Mw, Jw, lp, l, sweep, max_sweeps);
}

// The same one-sided Jacobi for the mixed path's factors of at most 128
// columns (FP32, left vectors only, shared memory; the sorted columns leave
// unnormalised in FP32 for the re-orthonormalisation): column stride 32 NV
// floats fixed at compile time, one 8-lane group per pair (64 groups cover
// every pair of a round), and each lane keeps its NV float4 of both columns
// in registers between the dot products and the rotation.  Same pair
// schedule, summation order, rotation formulas and stopping rule as
// k_jacobi<float, false>, so the same results (M is held scaled by an exact
// power of two, which changes no rounding unless the unscaled squares would
// overflow).
template <int NV>
__global__ void __launch_bounds__(512) k_jacobi_f32s(const Chan* __restrict__ ch, int max_sweeps) {
  extern __shared__ __align__(16) unsigned char sraw[];
  constexpr int lp = 32 * NV;
  const Chan& h = ch[blockIdx.x];
  const int l = h.l;
  const int m = l + (l & 1);
  float* Mw = (float*)sraw;
  __shared__ float smx[16];
  float mx = 0.0f;
  for (int e = threadIdx.x; e < lp * l; e += blockDim.x) {
    const int i = e % lp, j = e / lp;
    const float v = (i < l) ? (float)h.R[j + (int64_t)i * l] : 0.0f;      // M = R^T
    Mw[e] = v;
    mx = fmaxf(mx, fabsf(v));
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) smx[warp] = mx;
  __syncthreads();
  mx = 0.0f;
#pragma unroll
  for (int w = 0; w < 16; ++w) mx = fmaxf(mx, smx[w]);
  // M 2^-e with its largest entry in [1/2, 1), so that the squared norms and
  // their products below cannot overflow (scale 1 for a zero or non-finite
  // M); an exact power of two, undone before the finish
  const int ex = (int)((__float_as_uint(mx) >> 23) & 0xFFu);
  const int es = (ex == 0 || ex == 0xFF) ? 0 : ex - 126;
  if (es != 0)
    for (int e = threadIdx.x; e < lp * l; e += blockDim.x) Mw[e] = ldexpf(Mw[e], -es);
  __syncthreads();
  const float thr = (float)l * 5.9604645e-8f;
  const int grp = lane >> 3, gl = lane & 7;
  const int pi = warp * 4 + grp;                   // this group's pair slot
  const int npairs = m / 2;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    int rotated = 0;
    for (int r = 0; r < m - 1; ++r) {
      int a = -1, b = -1;
      if (pi < npairs) {
        if (pi == 0) { a = r; b = m - 1; }
        else {
          a = r + pi; if (a >= m - 1) a -= m - 1;
          b = r - pi; if (b < 0) b += m - 1;
        }
        if (a > b) { const int t = a; a = b; b = t; }
        if (b >= l) a = b = -1;
      }
      float4 x[NV], y[NV];
      float al = 0.0f, be = 0.0f, ga = 0.0f;
      float4* ca = (float4*)(Mw + (a < 0 ? 0 : a) * lp);
      float4* cb = (float4*)(Mw + (b < 0 ? 0 : b) * lp);
      if (a >= 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          x[v] = ca[gl + 8 * v];
          y[v] = cb[gl + 8 * v];
          al = fmaf(x[v].x, x[v].x, al); be = fmaf(y[v].x, y[v].x, be); ga = fmaf(x[v].x, y[v].x, ga);
          al = fmaf(x[v].y, x[v].y, al); be = fmaf(y[v].y, y[v].y, be); ga = fmaf(x[v].y, y[v].y, ga);
          al = fmaf(x[v].z, x[v].z, al); be = fmaf(y[v].z, y[v].z, be); ga = fmaf(x[v].z, y[v].z, ga);
          al = fmaf(x[v].w, x[v].w, al); be = fmaf(y[v].w, y[v].w, be); ga = fmaf(x[v].w, y[v].w, ga);
        }
      }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {            // reduce inside the 8-lane group
        al += __shfl_xor_sync(0xffffffffu, al, o);
        be += __shfl_xor_sync(0xffffffffu, be, o);
        ga += __shfl_xor_sync(0xffffffffu, ga, o);
      }
      if (a >= 0 && ga != 0.0f && !(fabsf(ga) <= thr * sqrtf(al * be))) {
        const float zeta = __fdividef(be - al, 2.0f * ga);
        const float az = fabsf(zeta);
        float tf = az > 1e15f ? __fdividef(0.5f, az) : __fdividef(1.0f, az + sqrtf(fmaf(zeta, zeta, 1.0f)));
        tf = zeta >= 0.0f ? tf : -tf;
        const float cs = rsqrtf(fmaf(tf, tf, 1.0f));
        const float sn = cs * tf;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          float4 nx, ny;
          nx.x = cs * x[v].x - sn * y[v].x; ny.x = sn * x[v].x + cs * y[v].x;
          nx.y = cs * x[v].y - sn * y[v].y; ny.y = sn * x[v].y + cs * y[v].y;
          nx.z = cs * x[v].z - sn * y[v].z; ny.z = sn * x[v].z + cs * y[v].z;
          nx.w = cs * x[v].w - sn * y[v].w; ny.w = sn * x[v].w + cs * y[v].w;
          ca[gl + 8 * v] = nx;
          cb[gl + 8 * v] = ny;
        }
        rotated = 1;
      }
      if (r < m - 2) __syncthreads();
    }
    if (!__syncthreads_or(rotated)) break;         // also the barrier after the last round
  }
  if (es != 0) {
    for (int e = threadIdx.x; e < lp * l; e += blockDim.x) Mw[e] = ldexpf(Mw[e], es);
    __syncthreads();
  }
  jacobi_finish<float, false, true>(h, Mw, (const float*)nullptr, lp, l, sweep, max_sweeps);
}

// Symmetric storage: for symmetric V the triplets pair as v_i = sign(lambda_i)
// u_i, so V ~ U_k diag(sign_i sigma_i) U_k^T needs U_k and the signs only;
// sign_i = sign(u_i . v_i) (one warp per column, fixed-order FP64 sum).
__global__ void __launch_bounds__(256) k_sym_signs(const double* __restrict__ U, int64_t ldu,
                                                   const double* __restrict__ V, int64_t ldv, int n, int k,
                                                   double* __restrict__ signs) {
  const int col = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (col >= k) return;
  const double* u = U + (int64_t)col * ldu;
  const double* v = V + (int64_t)col * ldv;
  double s = 0.0;
  for (int r = lane; r < n; r += 32) s = fma(u[r], v[r], s);
  s = warp_sum(s);
  if (lane == 0) signs[col] = s >= 0.0 ? 1.0 : -1.0;
}

void launch_sym_signs(const double* U, int64_t ldu, const double* V, int64_t ldv, int n, int k, double* signs,
                      cudaStream_t st) {
  if (k <= 0) return;
  k_sym_signs<<<(k + 7) / 8, 256, 0, st>>>(U, ldu, V, ldv, n, k, signs);
  note_launch();
}

// FP64 -> FP32 copies of small per-channel operands (the lift's X~, the
// probe coefficients C) for the FP32 tile products, one grid row per channel.
__global__ void __launch_bounds__(256) k_cvt_f32(const CvtDesc* __restrict__ d) {
  const CvtDesc c = d[blockIdx.y];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < c.count; e += (int64_t)gridDim.x * blockDim.x)
    c.dst[e] = f64_to_f32_rn(c.src[e]);
}

void launch_cvt_f32(const CvtDesc* d_desc, int C, int64_t max_count, cudaStream_t st) {
  if (C <= 0 || max_count <= 0) return;
  const int bx = (int)std::max<int64_t>(1, std::min<int64_t>(64, (max_count + 255) / 256));
  k_cvt_f32<<<dim3(bx, C), 256, 0, st>>>(d_desc);
  note_launch();
}

// Re-orthonormalisation of the FP32 Jacobi vectors X = M D (M the FP32
// columns, D = diag(1 / sigma), sigma_i = |M_i|; l <= 128):
//   G = D (M^T M) D  (M^T M from the compensated Gram),
//   X~ = X R^{-1} = M D + M (D (R^{-1} - I))  with R^T R = G,
// the second term small (R ~ I), so it is formed in FP32 and the first in FP64.
RSVD_DEV void reorth_inv(const Chan& h, double* inv) {
  for (int i = threadIdx.x; i < h.l; i += blockDim.x) {
    const double si = h.sig[i];
    inv[i] = si > 0.0 ? 1.0 / si : 0.0;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) k_reorth_scale(const Chan* __restrict__ ch) {
  __shared__ double inv[128];
  const Chan& h = ch[blockIdx.y];
  reorth_inv(h, inv);
  const int l = h.l;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < l * l; e += gridDim.x * blockDim.x)
    h.G[e] *= inv[e % l] * inv[e / l];
}

__global__ void __launch_bounds__(256) k_reorth_prep(const Chan* __restrict__ ch) {
  __shared__ double inv[128];
  const Chan& h = ch[blockIdx.y];
  reorth_inv(h, inv);
  const int l = h.l;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < l * l; e += gridDim.x * blockDim.x) {
    const int i = e % l, j = e / l;
    h.Ri32[e] = f64_to_f32_rn(inv[i] * (h.Ri[e] - (i == j ? 1.0 : 0.0)));
  }
}

__global__ void __launch_bounds__(256) k_reorth_add(const Chan* __restrict__ ch) {
  __shared__ double inv[128];
  const Chan& h = ch[blockIdx.y];
  reorth_inv(h, inv);
  const int l = h.l;
  const float* m32 = (const float*)h.M;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < l * l; e += gridDim.x * blockDim.x)
    h.J[e] = fma((double)m32[e], inv[e / l], h.J[e]);
}

void launch_reorth(int stage, const Chan* d_ch, int C, int max_l, cudaStream_t st) {
  if (C <= 0) return;
  const dim3 grid(std::max(1, std::min(16, (max_l * max_l + 255) / 256)), C);
  if (stage == 0) k_reorth_scale<<<grid, 256, 0, st>>>(d_ch);
  else if (stage == 1) k_reorth_prep<<<grid, 256, 0, st>>>(d_ch);
  else k_reorth_add<<<grid, 256, 0, st>>>(d_ch);
  note_launch();
}

void launch_jacobi(const Chan* d_ch, int C, int fp32, int max_l, cudaStream_t st) {
  // mixed path (fp32): only the left vectors X are used; FP64 path needs J too
  const size_t esz = fp32 ? sizeof(float) : sizeof(double);
  const int ve = fp32 ? 4 : 2;
  const size_t lp = (size_t)((max_l + 8 * ve - 1) / (8 * ve) * (8 * ve));
  const size_t bytes = (fp32 ? 1 : 2) * (size_t)max_l * lp * esz;
  const int use_smem = bytes <= 200 * 1024;
  const int sweeps = jacobi_max_sweeps();
  if (fp32 && max_l <= 128) {
    const int nv = (max_l + 31) / 32;
    int b2 = max_l * 32 * nv * (int)sizeof(float);
    // one wave of channels: take most of the shared memory, so that no other
    // kernel's block (the probe block runs beside this one on a second
    // stream) shares the SM with this latency-bound one
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        C <= nsm && b2 < 200 * 1024)
      b2 = 200 * 1024;
    void (*kf)(const Chan*, int) = nv == 1 ? k_jacobi_f32s<1> : nv == 2 ? k_jacobi_f32s<2>
                                 : nv == 3 ? k_jacobi_f32s<3> : k_jacobi_f32s<4>;
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, b2);
    kf<<<C, 512, b2, st>>>(d_ch, sweeps);
    note_launch();
    return;
  }
  if (fp32) {
    if (use_smem) {
      cudaFuncSetAttribute(k_jacobi<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      k_jacobi<float, false><<<C, 512, bytes, st>>>(d_ch, 1, sweeps);
    } else {
      k_jacobi<float, false><<<C, 512, 0, st>>>(d_ch, 0, sweeps);
    }
  } else {
    if (use_smem) {
      cudaFuncSetAttribute(k_jacobi<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      k_jacobi<double, true><<<C, 512, bytes, st>>>(d_ch, 1, sweeps);
    } else {
      k_jacobi<double, true><<<C, 512, 0, st>>>(d_ch, 0, sweeps);
    }
  }
  note_launch();
}

// ------------------------------------------------------------ rank selection
// FP64 identity: for orthonormal U_k = Q X_k and V_k Sigma_k = V^T U_k,
// ||V - U_k Sigma_k V_k^T||_F^2 = ||V||_F^2 - sum_{i<=k} sigma_i^2.
// Probe form (mixed path): with G the probe block (s Gaussian columns),
// C = Q^T V G, D = X^T C, ||(I - U_k U_k^T) V G||^2 = ||V G - Q C||^2 +
// sum_{i>k} |D_i|^2, and E||(I-P)V G||_F^2 = s ||(I-P) V||_F^2.
// Probe energies of the s columns for the current k, held one per lane:
// mean and upper confidence bound over the lanes (all 32 lanes call).
RSVD_DEV void probe_stats(double e, int s, double& mean, double& ucb) {
  const int lane = threadIdx.x & 31;
  double v = lane < s ? e : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  mean = v / s;
  double d = lane < s ? (e - mean) * (e - mean) : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  const double var = s > 1 ? d / (s - 1) : 0.0;
  ucb = mean + PROBE_Z * sqrt(var / s);
}

// One 256-thread block per channel.  Probe layout (mixed path): est_part[j] =
// ||R g_j||^2 with R = V G - Q C the probe residual, est_part[s + i s + j] =
// D_ij^2 for D = X^T C; e_j(k) = est_part[j] + sum_{i >= k} est_part[s + i s + j].
// For l <= 128 the lanes of warp 0 form e_j(k) for every k (the same
// additions, in the same order, as a walk down from k0), the eight warps
// evaluate the bound for all k at once, and thread 0 replays the walk on
// the stored values; larger l walks on warp 0.  The chosen rank and
// estimate are the same either way.
__global__ void __launch_bounds__(256) k_select(const Chan* __restrict__ ch, int policy, double tol_plan,
                                                int use_probe) {
  __shared__ double E[129][33];
  __shared__ double Ms[129], Us[129];
  __shared__ int s_k;
  const Chan& h = ch[blockIdx.x];
  const double tol = h.tol > 0.0 ? h.tol : tol_plan;
  const int l = h.l;
  ChanResult* res = h.res;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double fro2 = res->fro2;
  const int kcap = min(h.k_cap, l);
  const double thr = tol * tol * fro2;
  int k = -1;
  double est2 = 0.0;
  bool unmet = false;
  if (use_probe) {
    const int s = h.nprobe;
    const double* ep = h.est_part;
    const int kfix = min(h.k_fixed, kcap);
    const int k0 = policy == RSVD_RANK_FIXED ? kfix : kcap;
    const double floor2 = precision_floor2(res->wres2, l, fro2);
    if (l <= 128) {
      const int kmin = policy == RSVD_RANK_FIXED ? k0 : 1;
      // the D_ij^2 terms into shared memory (coalesced), then each lane's
      // running sums replace them in place, walking down from l - 1
      for (int e = tid; e < l * s; e += blockDim.x) E[e / s][e % s] = ep[s + e];
      __syncthreads();
      if (warp == 0) {
        double e = 0.0;
        if (lane < s) {
          e = ep[lane];
          for (int i = l - 1; i >= k0; --i) e += E[i][lane];
          E[k0][lane] = e;
          for (int kk = k0 - 1; kk >= kmin; --kk) {
            e += E[kk][lane];
            E[kk][lane] = e;
          }
        }
      }
      __syncthreads();
      for (int kk = kmin + warp; kk <= k0; kk += 8) {
        double mean, ucb;
        probe_stats(lane < s ? E[kk][lane] : 0.0, s, mean, ucb);
        if (lane == 0) {
          Ms[kk] = mean + floor2;
          Us[kk] = ucb + floor2;
        }
      }
      __syncthreads();
      if (tid == 0) {
        k = k0;
        est2 = Ms[k0];
        if (policy != RSVD_RANK_FIXED) {
          if (Us[k0] > thr) unmet = true;
          else
            for (int kk = k0 - 1; kk >= 1; --kk) {
              if (Us[kk] > thr) break;
              k = kk;
              est2 = Ms[kk];
            }
        }
      }
    } else if (warp == 0) {
      double e = 0.0;
      if (lane < s) {
        e = ep[lane];
        for (int i = l - 1; i >= k0; --i) e += ep[s + (int64_t)i * s + lane];
      }
      double mean, ucb;
      probe_stats(e, s, mean, ucb);
      mean += floor2; ucb += floor2;
      k = k0;
      est2 = mean;
      if (policy != RSVD_RANK_FIXED) {
        if (ucb > thr) unmet = true;
        else {
          // walk k downward while the bound stays under the threshold
          for (int kk = k0 - 1; kk >= 1; --kk) {
            if (lane < s) e += ep[s + (int64_t)kk * s + lane];
            probe_stats(e, s, mean, ucb);
            mean += floor2; ucb += floor2;
            if (ucb > thr) break;
            k = kk;
            est2 = mean;
          }
        }
      }
    }
  }
  if (tid == 0) {
    int status = RSVD_OK;
    if (res->flags & FLAG_NONFINITE) status = RSVD_ERR_NONFINITE;
    else if (res->flags & FLAG_CHOL_FAIL) status = RSVD_ERR_NOT_CONVERGED;
    if (!use_probe) {
      if (policy == RSVD_RANK_FIXED) {
        k = min(h.k_fixed, kcap);
        double s2 = 0.0;
        for (int i = 0; i < k; ++i) s2 += h.sig[i] * h.sig[i];
        est2 = fmax(fro2 - s2, 0.0);
      } else {
        double s2 = 0.0;
        for (int i = 0; i < kcap; ++i) {
          s2 += h.sig[i] * h.sig[i];
          if (fro2 - s2 <= thr) { k = i + 1; est2 = fmax(fro2 - s2, 0.0); break; }
        }
        if (k < 0) { k = kcap; est2 = fmax(fro2 - s2, 0.0); }
        unmet = est2 > thr;
      }
    }
    if (policy != RSVD_RANK_FIXED && fro2 > 0.0 && unmet && status == RSVD_OK) status = RSVD_ERR_TOL_NOT_MET;
    if (k < 0) k = 0;
    s_k = k;
    res->k_out = k;
    res->l_used = l;
    res->err_est = fro2 > 0.0 ? sqrt(est2 / fro2) : 0.0;
    if (status == RSVD_OK && (res->flags & FLAG_JACOBI_CAP)) status = RSVD_ERR_NOT_CONVERGED;
    if (status == RSVD_OK && (res->flags & FLAG_SHIFTED)) status = RSVD_WARN_SHIFTED_CQR;
    res->status = status;
  }
  __syncthreads();
  const int kk = s_k;
  for (int i = tid; i < kk; i += blockDim.x) {
    h.S[i] = h.sig[i];
    h.scr[i] = h.sig[i] > 0.0 ? 1.0 / h.sig[i] : 0.0;   // column scale of R_k = W X_k Sigma_k^{-1}
  }
}

void launch_select(const Chan* d_ch, int C, int policy, double tol, int use_probe,
                   cudaStream_t st) {
  k_select<<<C, 256, 0, st>>>(d_ch, policy, tol, use_probe);
  note_launch();
}

// ------------------------------------------------------------ probe features
// From the probe's singular values t (descending, h.sig[0..15]):
// [log(t_j / t_1), j = 2..16 | log t_1 | 0.5 log(sum t^2 / 16) | log n | log tol]
__global__ void k_features(const Chan* __restrict__ ch, double tol_plan, float* __restrict__ feat) {
  const Chan& h = ch[blockIdx.x];
  if (threadIdx.x != 0) return;
  const double tol = h.tol > 0.0 ? h.tol : tol_plan;
  double t[16], s2 = 0.0;
  for (int j = 0; j < 16; ++j) {
    t[j] = j < h.l ? h.sig[j] : 0.0;
    s2 += t[j] * t[j];
    t[j] = fmax(t[j], 1e-300);
  }
  float* f = feat + (int64_t)blockIdx.x * 19;
  for (int j = 1; j < 16; ++j) f[j - 1] = (float)log(t[j] / t[0]);
  f[15] = (float)log(t[0]);
  f[16] = (float)(0.5 * log(fmax(s2, 1e-300) / 16.0));
  f[17] = (float)log((double)h.n);
  f[18] = (float)log(tol);
}

void launch_features(const Chan* d_ch, int C, double tol, float* feat, cudaStream_t st) {
  k_features<<<C, 32, 0, st>>>(d_ch, tol, feat);
  note_launch();
}

// ------------------------------------------------------- block sum of squares
__global__ void __launch_bounds__(256) k_sumsq(const SumsqDesc* __restrict__ sd) {
  __shared__ double sh[32];
  const SumsqDesc* d = sd + blockIdx.x;
  const int rows = d->rows, cols = d->cols;
  double s = 0.0;
  for (int j = 0; j < cols; ++j) {
    if (d->esz == 8) {
      const double* col = (const double*)d->p + (int64_t)j * d->ld;
      for (int r = threadIdx.x; r < rows; r += blockDim.x) s = fma(col[r], col[r], s);
    } else {
      const float* col = (const float*)d->p + (int64_t)j * d->ld;
      float sf = 0.0f;
      for (int r = threadIdx.x; r < rows; r += blockDim.x) sf = fmaf(col[r], col[r], sf);
      s += f32_to_f64(sf);
    }
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *d->out = s;
}

__global__ void __launch_bounds__(256) k_colsumsq(const SumsqDesc* __restrict__ sd) {
  __shared__ double sh[32];
  const SumsqDesc* d = sd + blockIdx.x;
  const int j = blockIdx.y;
  if (j >= d->cols) return;
  double s = 0.0;
  if (d->esz == 8) {
    const double* col = (const double*)d->p + (int64_t)j * d->ld;
    for (int r = threadIdx.x; r < d->rows; r += blockDim.x) s = fma(col[r], col[r], s);
  } else {
    const float* col = (const float*)d->p + (int64_t)j * d->ld;
    for (int r = threadIdx.x; r < d->rows; r += blockDim.x) {
      const double v = f32_to_f64(col[r]);
      s = fma(v, v, s);
    }
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) d->out[j] = s;
}

// Q32 <- T32 for the channels whose flags carry FLAG_SHIFTED (the output of
// the conditional third CholeskyQR round lands in T32).
__global__ void __launch_bounds__(256) k_copy_t_to_q(const Chan* __restrict__ ch) {
  const Chan& h = ch[blockIdx.y];
  if (!(h.res->flags & FLAG_SHIFTED)) return;
  const int64_t total = (int64_t)h.l * h.ldt;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    h.Q32[e] = h.T32[e];
}

__global__ void __launch_bounds__(256) k_copy64_if(const CopyDesc* __restrict__ cd) {
  const CopyDesc d = cd[blockIdx.y];
  if (!(*d.flags & FLAG_SHIFTED)) return;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < d.count; e += (int64_t)gridDim.x * blockDim.x)
    d.dst[e] = d.src[e];
}
void launch_copy64_if_shifted(const CopyDesc* d_cd, int C, cudaStream_t st) {
  if (C < 1) return;
  k_copy64_if<<<dim3(64, C), 256, 0, st>>>(d_cd);
  note_launch();
}

void launch_copy_t_to_q_if_shifted(const Chan* d_ch, int C, cudaStream_t st) {
  if (C < 1) return;
  k_copy_t_to_q<<<dim3(64, C), 256, 0, st>>>(d_ch);
  note_launch();
}

void launch_colsumsq(const SumsqDesc* d_sd, int C, int max_cols, cudaStream_t st) {
  if (C < 1 || max_cols < 1) return;
  k_colsumsq<<<dim3(C, max_cols), 256, 0, st>>>(d_sd);
  note_launch();
}

void launch_sumsq(const SumsqDesc* d_sd, int C, cudaStream_t st) {
  if (C <= 0) return;
  k_sumsq<<<C, 256, 0, st>>>(d_sd);
  note_launch();
}

// ------------------------------------------------------------------ sign fix
// Flip (u_i, v_i) so that the largest-magnitude entry of u_i is positive
// (ties: lowest row).  Magnitudes are compared as the integer bit patterns of
// |u| (monotonic for finite values) and signs flipped by the sign bit, so the
// scan and the flip stay off this part's narrow FP64 pipe.
__global__ void __launch_bounds__(256) k_signfix(const Chan* __restrict__ ch) {
  __shared__ unsigned long long sv[256];
  __shared__ int si[256];
  const Chan& h = ch[blockIdx.x];
  const int col = blockIdx.y;
  if (col >= h.res->k_out || h.U == nullptr) return;
  unsigned long long* u = (unsigned long long*)(h.U + (int64_t)col * h.ldu);
  const unsigned long long mag = 0x7FFFFFFFFFFFFFFFull, sgn = 0x8000000000000000ull;
  unsigned long long best = 0;
  int bi = 0x7fffffff;
  for (int r = threadIdx.x; r < h.n; r += blockDim.x) {
    const unsigned long long a = u[r] & mag;
    if (bi == 0x7fffffff || a > best) { best = a; bi = r; }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const unsigned long long ob = sv[threadIdx.x + s];
      const int oi = si[threadIdx.x + s];
      if (oi != 0x7fffffff &&
          (si[threadIdx.x] == 0x7fffffff || ob > sv[threadIdx.x] || (ob == sv[threadIdx.x] && oi < si[threadIdx.x]))) {
        sv[threadIdx.x] = ob;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const bool neg = si[0] != 0x7fffffff && (u[si[0]] & sgn) && (u[si[0]] & mag);
  __syncthreads();
  if (neg) {
    for (int r = threadIdx.x; r < h.n; r += blockDim.x) u[r] ^= sgn;
    if (h.V) {
      unsigned long long* v = (unsigned long long*)(h.V + (int64_t)col * h.ldv);
      for (int r = threadIdx.x; r < h.n; r += blockDim.x) v[r] ^= sgn;
    }
  }
}

void launch_signfix(const Chan* d_ch, int C, int max_k, cudaStream_t st) {
  if (max_k <= 0) return;
  k_signfix<<<dim3(C, max_k), 256, 0, st>>>(d_ch);
  note_launch();
}

}  // namespace rsvd
