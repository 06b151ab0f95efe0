// Tile rule (matrix-free channels): the factor panel the tensor core turns
// into rule entries, and the reductions of the entry energies.
//
// A_ij = sum_m w_m g_m(x_i) g_m(x_j) + eta_ij with x_i = 8 i / (n - 1) and
// g_m(x) = exp(-(x - c_m)^2 / (2 s_m^2)).  With H_jm = sqrt(w_m) g_m(x_j)
// (w_m >= 0) the smooth part of a row panel is H_panel H^T: every pass
// generates every entry it reads (n^2 M multiply-adds on the tensor core),
// nothing of A is kept between panels or passes.
#include <algorithm>
#include <cmath>

#include "kernels.h"

namespace rsvd {

// H as two FP16 words of its FP32 value times hscale (rows j contiguous over
// m, leading dim ldh >= M; columns M..ldh-1 are zero).  The exponentials are
// FP64.  hscale puts the largest factor entry at 2^14 (FP16 overflows past
// 65504), so entries down to ~2^-24 / hscale keep their relative precision
// and smaller ones carry at most 2^-25 / hscale absolute error: ~2^-39 of
// the largest entry, negligible in every product.  hi + lo keeps 22 bits.
__global__ void __launch_bounds__(256) k_rule_prep(RuleDesc d) {
  const int64_t total = (int64_t)d.n * d.ldh;
  const double step = d.n > 1 ? 8.0 / (double)(d.n - 1) : 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / d.ldh), m = (int)(e % d.ldh);
    float h = 0.0f;
    if (m < d.M) {
      const double t = step * j - d.c[m];
      const double g = exp(-(t * t) / (2.0 * d.s[m] * d.s[m]));
      h = f64_to_f32_rn(sqrt(d.w[m]) * g * d.hscale);
    }
    const __half hi = __float2half_rn(h);
    d.H[0][e] = hi;
    d.H[1][e] = __float2half_rn(h - __half2float(hi));     // the remainder is exact in FP32
  }
}

double rule_hscale(const double* w, int M) {
  double mx = 0.0;
  for (int m = 0; m < M; ++m) mx = std::max(mx, w[m]);
  if (!(mx > 0.0)) return 1.0;
  int e = 14 - (int)std::ceil(std::log2(std::sqrt(mx)));
  e = std::max(-60, std::min(60, e));
  return std::ldexp(1.0, e);
}

void launch_rule_prep(const RuleDesc& d, cudaStream_t st) {
  const int64_t total = (int64_t)d.n * d.ldh;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  k_rule_prep<<<blocks, 256, 0, st>>>(d);
  note_launch();
}

RSVD_DEV double rsum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;
}

// FP64 path: H in FP64 (rows j contiguous over m, leading dim ldh >= M;
// columns M..ldh-1 zero).
__global__ void __launch_bounds__(256) k_rule_prep64(RuleDesc64 d) {
  const int64_t total = (int64_t)d.n * d.ldh;
  const double step = d.n > 1 ? 8.0 / (double)(d.n - 1) : 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / d.ldh), m = (int)(e % d.ldh);
    double h = 0.0;
    if (m < d.M) {
      const double t = step * j - d.c[m];
      h = sqrt(d.w[m]) * exp(-(t * t) / (2.0 * d.s[m] * d.s[m]));
    }
    d.H[e] = h;
  }
}

void launch_rule_prep64(const RuleDesc64& d, cudaStream_t st) {
  const int64_t total = (int64_t)d.n * d.ldh;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  k_rule_prep64<<<blocks, 256, 0, st>>>(d);
  note_launch();
}

// Add the hash noise to a generated FP64 row panel (column-major, rows x n,
// leading dim ldp; row i is matrix row r0 + i) and, if part is given, write
// each block's {sum v^2, 0} to part[2 block].  eta = amp3 (num 2^-24) with
// num = 2 (h >> 8) + 1 - 2^24 exact, amp3 = eta scale * sqrt(3).
__global__ void __launch_bounds__(256) k_rule_noise64(double* __restrict__ P, int64_t ldp, int rows, int n, int r0,
                                                      uint32_t key, double amp3, double* __restrict__ part) {
  __shared__ double sh[32];
  const int64_t total = (int64_t)rows * n;
  double s2 = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % rows), j = (int)(e / rows);
    const int gi = r0 + i;
    const uint32_t lo = (uint32_t)min(gi, j), hi = (uint32_t)max(gi, j);
    uint32_t h = lowbias32(lo * 0x9E3779B1u + key);
    h = lowbias32(h ^ (hi * 0x85EBCA77u));
    const int num = 2 * (int)(h >> 8) + 1 - (1 << 24);
    double* q = P + i + (int64_t)j * ldp;
    const double v = *q + amp3 * ((double)num * 5.9604644775390625e-8);
    *q = v;
    s2 = fma(v, v, s2);
  }
  if (part) {
    const double t = rsum(s2, sh);
    if (threadIdx.x == 0) {
      part[2 * (int64_t)blockIdx.x] = t;
      part[2 * (int64_t)blockIdx.x + 1] = 0.0;
    }
  }
}

void launch_rule_noise64(double* P, int64_t ldp, int rows, int n, int r0, uint32_t key, double amp3, double* part,
                         cudaStream_t st) {
  k_rule_noise64<<<kRuleNoiseBlocks, 256, 0, st>>>(P, ldp, rows, n, r0, key, amp3, part);
  note_launch();
}

// out[0..1] = column sums of part (nparts x 2), fixed order.
__global__ void __launch_bounds__(256) k_rule_part_sum(const double* __restrict__ part, int nparts,
                                                        double* __restrict__ out) {
  __shared__ double sh[32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    a += part[2 * (int64_t)i];
    b += part[2 * (int64_t)i + 1];
  }
  a = rsum(a, sh);
  b = rsum(b, sh);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
  }
}

void launch_rule_part_sum(const double* part, int nparts, double* out, cudaStream_t st) {
  k_rule_part_sum<<<1, 256, 0, st>>>(part, nparts, out);
  note_launch();
}

// res->fro2, res->wres2 from the per-panel sums (npanels x 2), in order.
__global__ void k_rule_finish(const double* __restrict__ sums, int npanels, ChanResult* res) {
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int p = 0; p < npanels; ++p) {
    a += sums[2 * p];
    b += sums[2 * p + 1];
  }
  res->fro2 = a;
  res->wres2 = b;
}

void launch_rule_finish(const double* sums, int npanels, ChanResult* res, cudaStream_t st) {
  k_rule_finish<<<1, 32, 0, st>>>(sums, npanels, res);
  note_launch();
}

}  // namespace rsvd
