// Exact residual ||V - U diag(S) W^T||_F and ||V||_F, accumulated in FP64
// over every entry.  This is the check behind the relative-Frobenius
// tolerance (the paper's validation of a rank-R_SVD form against the full
// matrix, "Randomized matrix decompositions" paragraph); it is not part of a
// decomposition.
//
// The n x n matrix is cut into 64 x 64 tiles; each CTA walks a fixed set of
// tiles (grid-stride) and writes one partial pair {residual^2, ||V||^2}, so
// the partial count is bounded and the sum order is fixed.  A tile is a
// 64 x 64 x K FP64 product of two staged 16-wide K slices:
//   stored V:   res = V_tile - (U S) W^T, K = k;
//   tile rule:  V_tile = H_rows H_cols^T + eta (regenerated in FP64, K = M),
//               then res = V_tile - (U S) W^T, K = k  --  every entry of the
//               rule is rebuilt from its definition, nothing is read back.
// Stored V is read column-major, V[r + c lda]; lanes run along r, so each
// half-warp reads 128 contiguous bytes.
#include <algorithm>

#include "kernels.h"

namespace rsvd {

struct ResidDesc {
  const double* A; int64_t lda;
  const double* U; int64_t ldu;
  const double* V; int64_t ldv;
  const double* S;
  int n, k;
  double* part;          // 2 doubles per CTA: residual^2, ||A||^2
  // tile rule (A == nullptr): H (n x ldh, row j contiguous over m) and noise
  const double* H; int64_t ldh; int M;
  uint32_t key; double amp3;
};

static constexpr int RES_BLOCKS_MAX = 152 * 8;

template <bool RULE>
__global__ void __launch_bounds__(256) k_resid(ResidDesc d) {
  __shared__ double Us[16][64 + 1];
  __shared__ double Vs[16][64 + 1];
  __shared__ double sh[2][8];
  const int nt = (d.n + 63) / 64;
  const int64_t tiles = (int64_t)nt * nt;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double r2 = 0.0, a2 = 0.0;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int ti = (int)(tile / nt), tj = (int)(tile % nt);
    const int r0 = ti * 64, c0 = tj * 64;
    double acc[4][4];   // row r0 + tx + 16 i, column c0 + ty + 16 j
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    if constexpr (RULE) {
      // smooth part H_rows H_cols^T
      for (int t0 = 0; t0 < d.M; t0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
          const int tt = e & 15, rr = e >> 4;        // 16 consecutive m of one row: contiguous
          const int t = t0 + tt;
          const int r = r0 + rr, c = c0 + rr;
          Us[tt][rr] = (t < d.M && r < d.n) ? d.H[(int64_t)r * d.ldh + t] : 0.0;
          Vs[tt][rr] = (t < d.M && c < d.n) ? d.H[(int64_t)c * d.ldh + t] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int tt = 0; tt < 16; ++tt)
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(Us[tt][tx + 16 * i], Vs[tt][ty + 16 * j], acc[i][j]);
        __syncthreads();
      }
      // + noise: the entry itself, and its energy
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = r0 + tx + 16 * i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = c0 + ty + 16 * j;
          if (r < d.n && c < d.n) {
            const uint32_t lo = (uint32_t)min(r, c), hi = (uint32_t)max(r, c);
            uint32_t h = lowbias32(lo * 0x9E3779B1u + d.key);
            h = lowbias32(h ^ (hi * 0x85EBCA77u));
            const int num = 2 * (int)(h >> 8) + 1 - (1 << 24);
            const double a = acc[i][j] + d.amp3 * ((double)num * 5.9604644775390625e-8);
            acc[i][j] = a;
            a2 = fma(a, a, a2);
          } else {
            acc[i][j] = 0.0;
          }
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = r0 + tx + 16 * i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = c0 + ty + 16 * j;
          const double a = (r < d.n && c < d.n) ? d.A[r + (int64_t)c * d.lda] : 0.0;
          acc[i][j] = a;
          a2 = fma(a, a, a2);
        }
      }
    }
    // - (U S) W^T
    for (int t0 = 0; t0 < d.k; t0 += 16) {
      for (int e = threadIdx.x; e < 16 * 64; e += 256) {
        const int rr = e & 63, tt = e >> 6;            // 64 consecutive rows of one column: contiguous
        const int t = t0 + tt;
        const int r = r0 + rr, c = c0 + rr;
        Us[tt][rr] = (t < d.k && r < d.n) ? d.U[r + (int64_t)t * d.ldu] * d.S[t] : 0.0;
        Vs[tt][rr] = (t < d.k && c < d.n) ? d.V[c + (int64_t)t * d.ldv] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int tt = 0; tt < 16; ++tt)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(-Us[tt][tx + 16 * i], Vs[tt][ty + 16 * j], acc[i][j]);
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) r2 = fma(acc[i][j], acc[i][j], r2);   // zero outside the matrix
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sh[0][w] = r2; sh[1][w] = a2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int q = 0; q < 8; ++q) { s0 += sh[0][q]; s1 += sh[1][q]; }
    d.part[2 * blockIdx.x] = s0;
    d.part[2 * blockIdx.x + 1] = s1;
  }
}

int resid_blocks(int64_t n) {
  const int64_t nt = (n + 63) / 64;
  return (int)std::min<int64_t>(nt * nt, RES_BLOCKS_MAX);
}

void launch_resid(const double* A, int64_t lda, const double* U, int64_t ldu, const double* V, int64_t ldv,
                  const double* S, int n, int k, double* part, cudaStream_t st) {
  ResidDesc d{A, lda, U, ldu, V, ldv, S, n, k, part, nullptr, 0, 0, 0u, 0.0};
  k_resid<false><<<resid_blocks(n), 256, 0, st>>>(d);
  note_launch();
}

void launch_resid_rule(const double* H, int64_t ldh, int M, uint32_t key, double amp3, const double* U,
                       int64_t ldu, const double* V, int64_t ldv, const double* S, int n, int k, double* part,
                       cudaStream_t st) {
  ResidDesc d{nullptr, 0, U, ldu, V, ldv, S, n, k, part, H, ldh, M, key, amp3};
  k_resid<true><<<resid_blocks(n), 256, 0, st>>>(d);
  note_launch();
}

}  // namespace rsvd
