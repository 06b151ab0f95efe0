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

// 8 rows per tile; fro_part gets one partial per tile.  Each thread owns
// pairs of adjacent columns (two 8-byte loads of the raw FP64 bits, four
// pairs 512 columns apart in flight) and writes each BF16 word pair as one
// 4-byte store; the FP64 -> FP32 rounding and the word split use 32-bit
// integer and FP32 instructions only (no FP64 instruction per element: FP64
// is a small fraction of this part's issue rate).  ||V||^2 is accumulated
// from the FP32 values (relative error ~1e-7) and summed in FP64 per tile;
// so is the energy of the remainder the words leave out (wres_part), which
// the probe error estimate cannot see and the rank rule adds back.
RSVD_DEV void convert_body(const Chan* __restrict__ ch, const int* __restrict__ off, int C, int nsl, int t) {
  __shared__ double sh[32];
  const int c = find_chan(off, C, t);
  const Chan& h = ch[c];
  const int b = t - off[c];
  const int r0 = b * 8, r1 = min(h.n, r0 + 8);
  const int n = h.n;
  const int npair = (n + 1) >> 1;
  float s = 0.0f, w = 0.0f;
  bool bad = false;
  for (int r = r0; r < r1; ++r) {
    const int2* row = (const int2*)(h.A + (int64_t)r * h.lda);
    __nv_bfloat162* o0 = (__nv_bfloat162*)(h.Ab[0] + (int64_t)r * h.ldb);
    __nv_bfloat162* o1 = (__nv_bfloat162*)(h.Ab[1] + (int64_t)r * h.ldb);
    __nv_bfloat162* o2 = (__nv_bfloat162*)(h.Ab[2] + (int64_t)r * h.ldb);
    for (int p0 = 0; p0 < npair; p0 += 1024) {
      int2 v[4][2];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int p = p0 + threadIdx.x + 256 * u;
        const int j = 2 * p;
        v[u][0] = (p < npair) ? __ldcs(row + j) : make_int2(0, 0);
        v[u][1] = (p < npair && j + 1 < n) ? __ldcs(row + j + 1) : make_int2(0, 0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int p = p0 + threadIdx.x + 256 * u;
        if (p >= npair) continue;
        float2 f;
        f.x = f64w_to_f32_rn((unsigned int)v[u][0].y, (unsigned int)v[u][0].x, bad);
        f.y = f64w_to_f32_rn((unsigned int)v[u][1].y, (unsigned int)v[u][1].x, bad);
        s = fmaf(f.x, f.x, s);
        s = fmaf(f.y, f.y, s);
        __nv_bfloat162 q = __float22bfloat162_rn(f);
        o0[p] = q;
        float2 g = __bfloat1622float2(q);
        f.x -= g.x;                        // exact: the remainder fits in FP32
        f.y -= g.y;
        if (nsl > 1) {
          q = __float22bfloat162_rn(f);
          o1[p] = q;
          g = __bfloat1622float2(q);
          f.x -= g.x;
          f.y -= g.y;
          if (nsl > 2) {
            q = __float22bfloat162_rn(f);
            o2[p] = q;
            g = __bfloat1622float2(q);
            f.x -= g.x;
            f.y -= g.y;
          }
        }
        w = fmaf(f.x, f.x, w);             // what the words leave out
        w = fmaf(f.y, f.y, w);
      }
    }
  }
  const double sd = bsum(f32_to_f64(s), sh);
  const double wd = bsum(f32_to_f64(w), sh);
  if (bad) atomicOr(&h.res->flags, FLAG_NONFINITE);
  if (threadIdx.x == 0) {
    h.fro_part[b] = sd;
    if (h.wres_part) h.wres_part[b] = wd;
  }
}

__global__ void __launch_bounds__(256) k_convert(const Chan* __restrict__ ch, const int* __restrict__ off, int C,
                                                 int nsl) {
  convert_body(ch, off, C, nsl, blockIdx.x);
}

void launch_convert_slices(const Chan* d_ch, const int* d_off, int C, int tiles, int nsl,
                           cudaStream_t st) {
  if (tiles > 0) { k_convert<<<tiles, 256, 0, st>>>(d_ch, d_off, C, nsl); note_launch(); }
}

// Columns [j0, j1) of the X words: j < l are sketch columns (global column
// col0 + j, TAG_OMEGA), j >= l probe columns (column j - l, TAG_RESID).
// Word 0 holds the BF16 value, which is exact, so higher words are zero.
RSVD_DEV void omega_body(const Chan* __restrict__ ch, const int* __restrict__ off, int C, uint64_t seed, int col0,
                         int j0, int j1, uint64_t pseed, int nsl, uint32_t tag, int t) {
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
    if (j < h.l) g = gauss_f32(seed, (uint32_t)i, (uint32_t)(col0 + h.col0 + j), tag);
    else g = gauss_f32(pseed, (uint32_t)i, (uint32_t)(j - h.l), TAG_RESID);
    const int64_t o = (int64_t)j * h.ldb + i;
    h.Xb[0][o] = __float2bfloat16_rn(g);
    for (int w = 1; w < nsl; ++w) h.Xb[w][o] = __float2bfloat16_rn(0.0f);
  }
}

__global__ void __launch_bounds__(256) k_omega_bf16(const Chan* __restrict__ ch, const int* __restrict__ off, int C,
                                                    uint64_t seed, int col0, int j0, int j1, uint64_t pseed, int nsl,
                                                    uint32_t tag) {
  omega_body(ch, off, C, seed, col0, j0, j1, pseed, nsl, tag, blockIdx.x);
}

// The conversion (HBM-bound) and the sketch matrix (Philox + Box-Muller,
// ALU-bound) in one grid: their blocks are interleaved evenly, so the SMs
// generate P while the conversion waits on memory.  Block b is P block
// floor(b t64 / total) if that count steps at b, else conversion block
// b - floor((b + 1) t64 / total).
__global__ void __launch_bounds__(256) k_convert_omega(const Chan* __restrict__ ch, const int* __restrict__ off8,
                                                       int t8, const int* __restrict__ off64, int t64, int C, int nsl,
                                                       uint64_t seed, uint64_t pseed, int onsl) {
  const int64_t total = (int64_t)t8 + t64;
  const int64_t b = blockIdx.x;
  const int64_t lo = b * t64 / total, hi = (b + 1) * t64 / total;
  if (hi > lo) omega_body(ch, off64, C, seed, 0, 0, 1 << 30, pseed, onsl, TAG_OMEGA, (int)lo);
  else convert_body(ch, off8, C, nsl, (int)(b - hi));
}

void launch_convert_omega(const Chan* d_ch, const int* d_off8, int t8, const int* d_off64, int t64, int C, int nsl,
                          uint64_t seed, uint64_t pseed, int onsl, cudaStream_t st) {
  if (t8 + t64 <= 0) return;
  k_convert_omega<<<t8 + t64, 256, 0, st>>>(d_ch, d_off8, t8, d_off64, t64, C, nsl, seed, pseed, onsl);
  note_launch();
}

void launch_omega_bf16(const Chan* d_ch, const int* d_off, int C, int tiles, uint64_t seed,
                       int col0, int j0, int j1, uint64_t pseed, int nsl, cudaStream_t st, uint32_t tag) {
  if (tiles > 0) { k_omega_bf16<<<tiles, 256, 0, st>>>(d_ch, d_off, C, seed, col0, j0, j1, pseed, nsl, tag); note_launch(); }
}

// est_part[s + i s + j] = D_ij^2 for D = X^T C (X the small SVD's left
// vectors in M, C = Q^T V G), one warp per row i, lane j < s; the residual
// energies est_part[0..s) come from the column sums of V G - Q C.
__global__ void __launch_bounds__(256) k_probe_finish(const Chan* __restrict__ ch) {
  // C (l x s, l <= 128) staged in shared memory with the probe index
  // fastest (a warp reads one row of it, conflict-free); block y takes 32
  // rows i of X, warp w rows i0 + 4w .. i0 + 4w + 3, lane = probe column j;
  // four independent FMA chains per dot product
  __shared__ double Cs[128][33];
  const Chan& h = ch[blockIdx.x];
  const int l = h.l, s = h.nprobe;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (l > 128) {                                   // wide factors: one dot product per thread
    const int i = blockIdx.y * 32 + (threadIdx.x >> 5);
    for (int ii = i; ii < min(l, blockIdx.y * 32 + 32); ii += 8) {
      if (lane >= s) break;
      double d = 0.0;
      for (int a = 0; a < l; ++a) d = fma(h.M[a + (int64_t)ii * l], h.C64[a + (int64_t)lane * l], d);
      h.est_part[s + (int64_t)ii * s + lane] = d * d;
    }
    return;
  }
  for (int e = threadIdx.x; e < l * 32; e += blockDim.x) {
    const int a = e % l, j = e / l;
    Cs[a][j] = j < s ? h.C64[a + (int64_t)j * l] : 0.0;
  }
  __syncthreads();
  if (lane >= s) return;
#pragma unroll 1
  for (int r = 0; r < 4; ++r) {
    const int i = blockIdx.y * 32 + 4 * warp + r;
    if (i >= l) break;
    const double* m = h.M + (int64_t)i * l;
    double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
    int a = 0;
    for (; a + 4 <= l; a += 4) {
      d0 = fma(__ldg(m + a), Cs[a][lane], d0);
      d1 = fma(__ldg(m + a + 1), Cs[a + 1][lane], d1);
      d2 = fma(__ldg(m + a + 2), Cs[a + 2][lane], d2);
      d3 = fma(__ldg(m + a + 3), Cs[a + 3][lane], d3);
    }
    for (; a < l; ++a) d0 = fma(__ldg(m + a), Cs[a][lane], d0);
    const double d = (d0 + d1) + (d2 + d3);
    h.est_part[s + (int64_t)i * s + lane] = d * d;
  }
}

void launch_probe_finish(const Chan* d_ch, int C, int max_l, cudaStream_t st) {
  k_probe_finish<<<dim3(C, (max_l + 31) / 32), 256, 0, st>>>(d_ch);
  note_launch();
}

// ------------------------------------------------------------ probe block
// The probe block of the mixed path's error estimate (s <= 32 columns, far
// narrower than the 128-wide tiles of the general products): C = Q^T Z
// (l x s) and the residual R = Z - Q C in place of Z, FP32 FMA (ample for
// an estimate).

RSVD_DEV int probe_chan(const ProbeDesc* __restrict__ pd, int C, int b) {
  int lo = 0, hi = C - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pd[mid].tile0 <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One block per (row split, 128-column chunk of Q): thread (i, jh) sums
// Q[:, c0 + i] . Z[:, 16 jh + jj] over the split's rows, 32 rows at a time
// staged in shared memory (Q by coalesced loads down its columns; Z's 32 x 32
// block through L1), the 16 Z values of a row read as four 16-byte vectors;
// the next 32 rows load into registers while the current ones are summed.
__global__ void __launch_bounds__(256, 2) k_probe_tn(const ProbeDesc* __restrict__ pd, int C) {
  __shared__ float Qs[32][129];
  __shared__ __align__(16) float Zs[32][32];
  const ProbeDesc* g = pd + probe_chan(pd, C, blockIdx.x);
  const int local = blockIdx.x - g->tile0;
  const int lch = (g->l + 127) >> 7;
  const int split = local / lch, c0 = (local % lch) * 128;
  const int n = g->n, l = g->l, s = g->s;
  const int rb = split * g->split_rows, re = min(n, rb + g->split_rows);
  const float* Q = g->Q;
  const float* Z = g->Z;
  const int64_t ldq = g->ldq, ldz = g->ldz;
  const int tid = threadIdx.x, i = tid & 127, jh = tid >> 7;
  float qn[16], zn[4];
  auto fetch = [&](int r0) {
#pragma unroll
    for (int p = 0; p < 16; ++p) {
      const int e = tid + 256 * p, rr = e & 31, cc = e >> 5;
      const int gr = r0 + rr, gc = c0 + cc;
      qn[p] = (gr < re && gc < l) ? __ldg(Q + gr + (int64_t)gc * ldq) : 0.0f;
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int e = tid + 256 * p, jj = e & 31, rr = e >> 5;
      const int gr = r0 + rr;
      zn[p] = (gr < re && jj < s) ? __ldg(Z + gr + (int64_t)jj * ldz) : 0.0f;
    }
  };
  float acc[16];
#pragma unroll
  for (int jj = 0; jj < 16; ++jj) acc[jj] = 0.0f;
  if (rb < re) fetch(rb);
  for (int r0 = rb; r0 < re; r0 += 32) {
#pragma unroll
    for (int p = 0; p < 16; ++p) {
      const int e = tid + 256 * p;
      Qs[e & 31][e >> 5] = qn[p];
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int e = tid + 256 * p;
      Zs[e >> 5][e & 31] = zn[p];
    }
    __syncthreads();
    if (r0 + 32 < re) fetch(r0 + 32);
#pragma unroll 4
    for (int rr = 0; rr < 32; ++rr) {
      const float q = Qs[rr][i];
      const float4* zr = reinterpret_cast<const float4*>(&Zs[rr][16 * jh]);
#pragma unroll
      for (int v4 = 0; v4 < 4; ++v4) {
        const float4 z = zr[v4];
        acc[4 * v4] = fmaf(q, z.x, acc[4 * v4]);
        acc[4 * v4 + 1] = fmaf(q, z.y, acc[4 * v4 + 1]);
        acc[4 * v4 + 2] = fmaf(q, z.z, acc[4 * v4 + 2]);
        acc[4 * v4 + 3] = fmaf(q, z.w, acc[4 * v4 + 3]);
      }
    }
    __syncthreads();
  }
  if (c0 + i < l) {
    double* part = g->part + (int64_t)split * l * s;
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      const int j = 16 * jh + jj;
      if (j < s) part[(c0 + i) + (int64_t)j * l] = f32_to_f64(acc[jj]);
    }
  }
}

// C = sum of the split partials (FP64, in split order), and its FP32
// rounding padded to 32 columns per row of C (C32[k * 32 + j], zero for
// j >= s) for the residual kernel.
__global__ void k_probe_tn_reduce(const ProbeDesc* __restrict__ pd) {
  const ProbeDesc* g = pd + blockIdx.y;
  const int l = g->l, s = g->s, ls = l * s, splits = g->splits;
  const double* part = g->part;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < l * 32; e += gridDim.x * blockDim.x) {
    const int k = e >> 5, j = e & 31;
    float c32 = 0.0f;
    if (j < s) {
      const int64_t o = k + (int64_t)j * l;
      double v = 0.0;
#pragma unroll 8
      for (int p = 0; p < splits; ++p) v += __ldg(part + (int64_t)p * ls + o);
      g->C[o] = v;
      c32 = f64_to_f32_rn(v);
    }
    g->C32[e] = c32;
  }
}

// A 128-row block, one row per thread, 16 columns at a time: R = Z - Q C
// with C (rounded to FP32) in shared memory, read as 16-byte vectors, and Q
// down its columns (coalesced), 16 k at a time so that 16 loads per thread
// are in flight.
__global__ void __launch_bounds__(128) k_probe_nn_sub(const ProbeDesc* __restrict__ pd, int C) {
  __shared__ __align__(16) float Cs[256][32];
  const ProbeDesc* g = pd + probe_chan(pd, C, blockIdx.x);
  const int l = g->l, s = g->s, n = g->n;
  {
    const float4* src = reinterpret_cast<const float4*>(g->C32);
    float4* dst = reinterpret_cast<float4*>(&Cs[0][0]);
#pragma unroll 4
    for (int e = threadIdx.x; e < 256 * 8; e += blockDim.x)
      dst[e] = e < l * 8 ? __ldg(src + e) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
  __syncthreads();
  const int r = (blockIdx.x - g->tile0) * 128 + threadIdx.x;
  if (r >= n) return;
  const float* q = g->Q + r;
  const int64_t ldq = g->ldq;
  for (int jb = 0; jb < s; jb += 16) {
    float acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0.0f;
    for (int k0 = 0; k0 < l; k0 += 16) {
      float qk[16];
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) qk[kk] = k0 + kk < l ? __ldg(q + (int64_t)(k0 + kk) * ldq) : 0.0f;
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        const float4* cr = reinterpret_cast<const float4*>(&Cs[k0 + kk][jb]);
#pragma unroll
        for (int v4 = 0; v4 < 4; ++v4) {
          const float4 c = cr[v4];
          acc[4 * v4] = fmaf(qk[kk], c.x, acc[4 * v4]);
          acc[4 * v4 + 1] = fmaf(qk[kk], c.y, acc[4 * v4 + 1]);
          acc[4 * v4 + 2] = fmaf(qk[kk], c.z, acc[4 * v4 + 2]);
          acc[4 * v4 + 3] = fmaf(qk[kk], c.w, acc[4 * v4 + 3]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (jb + j < s) g->Z[r + (int64_t)(jb + j) * g->ldz] -= acc[j];
  }
}

void launch_probe_block(const ProbeDesc* d_tn, const ProbeDesc* d_nn, int C, int tn_blocks, int nn_blocks,
                        cudaStream_t st) {
  if (C <= 0) return;
  k_probe_tn<<<tn_blocks, 256, 0, st>>>(d_tn, C);
  k_probe_tn_reduce<<<dim3(16, C), 256, 0, st>>>(d_tn);
  k_probe_nn_sub<<<nn_blocks, 128, 0, st>>>(d_nn, C);
  note_launch(3);
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
