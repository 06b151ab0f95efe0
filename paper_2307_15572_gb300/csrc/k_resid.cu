// Exact residual ||V - U diag(S) W^T||_F and ||V||_F, accumulated in FP64
// over every entry (64 x 64 tiles, one partial pair per tile, summed on the
// host in a fixed order).  This is the check behind the relative-Frobenius
// tolerance; it is not part of a decomposition.
#include <vector>

#include "kernels.h"

namespace rsvd {

struct ResidDesc {
  const double* A; int64_t lda;
  const double* U; int64_t ldu;
  const double* V; int64_t ldv;
  const double* S;
  int n, k;
  double* part;     // 2 doubles per tile: residual^2, ||A||^2
};

__global__ void __launch_bounds__(256) k_resid(ResidDesc d) {
  __shared__ double Us[16][64 + 1];
  __shared__ double Vs[16][64 + 1];
  __shared__ double sh[2][8];
  const int nt = (d.n + 63) / 64;
  const int ti = blockIdx.x / nt, tj = blockIdx.x % nt;
  const int r0 = ti * 64, c0 = tj * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int t0 = 0; t0 < d.k; t0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int rr = e & 63, tt = e >> 6;
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
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(Us[tt][ty * 4 + i], Vs[tt][tx * 4 + j], acc[i][j]);
    __syncthreads();
  }
  double r2 = 0.0, a2 = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty * 4 + i;
    if (r >= d.n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx * 4 + j;
      if (c >= d.n) continue;
      const double a = d.A[(int64_t)r * d.lda + c];
      const double dd = a - acc[i][j];
      r2 = fma(dd, dd, r2);
      a2 = fma(a, a, a2);
    }
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

int resid_tiles(int n) { const int nt = (n + 63) / 64; return nt * nt; }

void launch_resid(const double* A, int64_t lda, const double* U, int64_t ldu, const double* V, int64_t ldv,
                  const double* S, int n, int k, double* part, cudaStream_t st) {
  ResidDesc d{A, lda, U, ldu, V, ldv, S, n, k, part};
  k_resid<<<resid_tiles(n), 256, 0, st>>>(d);
  note_launch();
}

}  // namespace rsvd
