// Mixed-path helper kernels.
//
//   * V (FP64) -> BF16 words V_0 + V_1 (+ V_2), each word the round-to-nearest
//     BF16 of what the previous words left over, fused with ||V||_F^2 and a
//     NaN/Inf check (one streaming pass: 8 bytes read, 2 per word written);
//   * the random projection matrix P (and the probe block) as BF16 words in
//     the K-major layout the tensor-core pass reads;
//   * the probe residual of the error estimate:
//     ||V G - Q (Q^T V G)||_F^2 and |(X^T C)_i|^2 per singular index.
#include "kernels.h"

namespace rsvd {

template <typename T>
RSVD_DEV T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

RSVD_DEV double bsum(double v, double* sh) {
  v = wsum(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    r = wsum(r);
  }
  __syncthreads();
  if (threadIdx.x == 0) sh[0] = r;
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

// FP64 -> FP32 with round-to-nearest-even done on the integer pipe (the FP64
// units are a small fraction of this part's throughput).  Normal results are
// assembled from the bit fields; zeros, subnormal or overflowing results and
// non-finite inputs take the conversion instruction.
RSVD_DEV float f64_to_f32_rn(double a) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(a);
  const unsigned int e = (unsigned int)(b >> 52) & 0x7FFu;
  const int fe = (int)e - 1023 + 127;
  if (fe <= 0 || fe >= 255) return __double2float_rn(a);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const unsigned int keep = (unsigned int)(m >> 29);
  const unsigned int rest = (unsigned int)(m & 0x1FFFFFFFull);
  const unsigned int up = (rest > 0x10000000u) || (rest == 0x10000000u && (keep & 1u));
  const unsigned int r = ((unsigned int)fe << 23) + keep + up;     // carry into the exponent is RN's overflow
  return __uint_as_float((unsigned int)(b >> 32 & 0x80000000u) | r);
}

// 8 rows per tile; fro_part gets one partial per tile.  Each thread handles
// pairs of adjacent columns so the BF16 words go out as 4-byte stores.
// ||V||^2 is accumulated from the FP32 values (relative error ~1e-7, far
// below what the relative tolerance needs) and summed in FP64 per tile.
__global__ void __launch_bounds__(256) k_convert(const Chan* __restrict__ ch,
                                                 const int* __restrict__ off, int C, int nsl) {
  __shared__ double sh[32];
  const int t = blockIdx.x;
  const int c = find_chan(off, C, t);
  const Chan& h = ch[c];
  const int b = t - off[c];
  const int r0 = b * 8, r1 = min(h.n, r0 + 8);
  float s = 0.0f;
  bool bad = false;
  const int npair = (h.n + 1) >> 1;
  for (int r = r0; r < r1; ++r) {
    const double* row = h.A + (int64_t)r * h.lda;
    for (int p = threadIdx.x; p < npair; p += blockDim.x) {
      const int j = 2 * p;
      const double a0 = row[j];
      const double a1 = (j + 1 < h.n) ? row[j + 1] : 0.0;
      bad |= !isfinite(a0) || !isfinite(a1);
      float f0 = f64_to_f32_rn(a0), f1 = f64_to_f32_rn(a1);
      s = fmaf(f0, f0, s);
      s = fmaf(f1, f1, s);
      for (int w = 0; w < nsl; ++w) {
        const __nv_bfloat16 q0 = __float2bfloat16_rn(f0), q1 = __float2bfloat16_rn(f1);
        *(__nv_bfloat162*)(h.Ab[w] + (int64_t)r * h.ldb + j) = __halves2bfloat162(q0, q1);
        f0 -= __bfloat162float(q0);     // exact: the remainder fits in FP32
        f1 -= __bfloat162float(q1);
      }
    }
  }
  const double sd = bsum((double)s, sh);
  if (bad) atomicOr(&h.res->flags, FLAG_NONFINITE);
  if (threadIdx.x == 0) h.fro_part[b] = sd;
}

void launch_convert_slices(const Chan* d_ch, const int* d_off, int C, int tiles, int nsl,
                           cudaStream_t st) {
  if (tiles > 0) { k_convert<<<tiles, 256, 0, st>>>(d_ch, d_off, C, nsl); note_launch(); }
}

// Columns [j0, j1) of the X words: j < l are sketch columns (global column
// col0 + j, TAG_OMEGA), j >= l probe columns (column j - l, TAG_RESID).
// Word 0 holds the BF16 value, which is exact, so higher words are zero.
__global__ void __launch_bounds__(256) k_omega_bf16(const Chan* __restrict__ ch,
                                                    const int* __restrict__ off, int C,
                                                    uint64_t seed, int col0, int j0, int j1,
                                                    uint64_t pseed, int nsl) {
  const int t = blockIdx.x;
  const int c = find_chan(off, C, t);
  const Chan& h = ch[c];
  const int r0 = (t - off[c]) * 64;
  const int rows = min(64, h.n - r0);
  const int jend = min(j1, h.lw);
  for (int e = threadIdx.x; e < 64 * (jend - j0); e += blockDim.x) {
    const int rr = e & 63, j = j0 + (e >> 6);
    if (rr >= rows) continue;
    const int i = r0 + rr;
    float g;
    if (j < h.l) g = gauss_f32(seed, (uint32_t)i, (uint32_t)(col0 + j), TAG_OMEGA);
    else g = gauss_f32(pseed, (uint32_t)i, (uint32_t)(j - h.l), TAG_RESID);
    const int64_t o = (int64_t)j * h.ldb + i;
    h.Xb[0][o] = __float2bfloat16_rn(g);
    for (int w = 1; w < nsl; ++w) h.Xb[w][o] = __float2bfloat16_rn(0.0f);
  }
}

void launch_omega_bf16(const Chan* d_ch, const int* d_off, int C, int tiles, uint64_t seed,
                       int col0, int j0, int j1, uint64_t pseed, int nsl, cudaStream_t st) {
  if (tiles > 0) { k_omega_bf16<<<tiles, 256, 0, st>>>(d_ch, d_off, C, seed, col0, j0, j1, pseed, nsl); note_launch(); }
}

// ||V G - Q C||^2 partial per 64-row tile (V G = Y32[:, l:l+s], C = C64).
__global__ void __launch_bounds__(256) k_probe_resid(const Chan* __restrict__ ch,
                                                     const int* __restrict__ off, int C) {
  extern __shared__ float Cs[];   // l x s
  __shared__ double sh[32];
  const int t = blockIdx.x;
  const int c = find_chan(off, C, t);
  const Chan& h = ch[c];
  const int l = h.l, s = h.nprobe;
  for (int e = threadIdx.x; e < l * s; e += blockDim.x) Cs[e] = (float)h.C64[e];
  __syncthreads();
  const int r0 = (t - off[c]) * 64;
  const int r = r0 + (threadIdx.x & 63);
  const int tg = threadIdx.x >> 6;   // 4 groups of probes
  double sq = 0.0;
  if (r < h.n) {
    for (int p = tg; p < s; p += 4) {
      float acc = 0.0f;
      for (int a = 0; a < l; ++a) acc = fmaf(h.Q32[r + (int64_t)a * h.ldt], Cs[a + p * l], acc);
      const float v = h.Y32[r + (int64_t)(l + p) * h.ldt] - acc;
      sq += (double)v * (double)v;
    }
  }
  sq = bsum(sq, sh);
  if (threadIdx.x == 0) h.fro_part[t - off[c]] = sq;
}

// est_part[0] = sum of the partials; est_part[1+i] = |(X^T C)_i|^2.
__global__ void __launch_bounds__(256) k_probe_finish(const Chan* __restrict__ ch) {
  __shared__ double sh[32];
  const Chan& h = ch[blockIdx.x];
  const int l = h.l, s = h.nprobe;
  const int nb = (h.n + 63) / 64;
  double v = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v += h.fro_part[i];
  v = bsum(v, sh);
  if (threadIdx.x == 0) h.est_part[0] = v;
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    double acc2 = 0.0;
    for (int p = 0; p < s; ++p) {
      double d = 0.0;
      for (int a = 0; a < l; ++a) d = fma(h.M[a + (int64_t)i * l], h.C64[a + (int64_t)p * l], d);
      acc2 = fma(d, d, acc2);
    }
    h.est_part[1 + i] = acc2;
  }
}

void launch_probe_resid(const Chan* d_ch, const int* d_off, int C, int tiles, int max_l, int s,
                        cudaStream_t st) {
  if (tiles <= 0) return;
  const size_t bytes = (size_t)max_l * s * sizeof(float);
  if (bytes > 48 * 1024)
    cudaFuncSetAttribute(k_probe_resid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  k_probe_resid<<<tiles, 256, bytes, st>>>(d_ch, d_off, C);
  note_launch();
}

void launch_probe_finish(const Chan* d_ch, int C, cudaStream_t st) {
  k_probe_finish<<<C, 256, 0, st>>>(d_ch);
  note_launch();
}

// Zero column blocks of tall matrices (before k-split accumulation).
__global__ void k_zero(const ZeroDesc* __restrict__ zd, const int* __restrict__ off, int C) {
  const int t = blockIdx.x;
  const int c = find_chan(off, C, t);
  const ZeroDesc z = zd[c];
  const int r0 = (t - off[c]) * 64;
  for (int e = threadIdx.x; e < 64 * z.cols; e += blockDim.x) {
    const int rr = e & 63, j = e >> 6;
    const int r = r0 + rr;
    if (r < z.rows) {
      if (z.esz == 8) ((double*)z.p)[r + (int64_t)j * z.ld] = 0.0;
      else ((float*)z.p)[r + (int64_t)j * z.ld] = 0.0f;
    }
  }
}

void launch_zero(const ZeroDesc* d_zd, const int* d_off, int C, int tiles, cudaStream_t st) {
  if (tiles > 0) { k_zero<<<tiles, 256, 0, st>>>(d_zd, d_off, C); note_launch(); }
}

}  // namespace rsvd
