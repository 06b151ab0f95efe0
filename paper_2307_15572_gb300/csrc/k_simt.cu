// SIMT tile kernels of the pipeline (CUDA cores).
//
//   * Z = V X for the all-FP64 path (Fig. 1 step 1 and the projection
//     Y^T = V Q of step 1', V symmetric), FP64 FMA;
//   * Gram matrices Y^T Y of CholeskyQR (Fukaya et al., 2014), either in
//     FP64 or, for FP32 data, with the compensated dot product "Dot2" of
//     Ogita, Rump & Oishi (SIAM J. Sci. Comput. 26, 2005: TwoProduct by FMA,
//     TwoSum by Knuth's six-flop form), which returns a result as accurate
//     as one computed in twice the working precision -- an FP64-grade Gram
//     from FP32 operands at FP32 throughput;
//   * Q = Y R^{-1} (CholeskyQR's triangular solve through the explicit
//     inverse) and the lift L = Q L_Y of Fig. 1 step 3.
//
// One templated 64 x 64 x 16 tile kernel serves all of them: C (m x n,
// column-major) = op(A) (m x k) * B (k x n, column-major).  Operand A is read
// either "row" style, A(i,kk) = A[i*lda + kk] (the dense symmetric V, or
// Y^T for a Gram), or "col" style, A(i,kk) = A[i + kk*lda] (tall Q or Y).
// Channels of a batch are tiled together: tile t belongs to channel c with
// off[c] <= t < off[c+1].
#include "kernels.h"

namespace rsvd {

enum { AROW = 0, ACOL = 1 };
enum { ACC_F64 = 0, ACC_F32 = 1, ACC_DOT2 = 2 };

template <int ACC> struct AccT { typedef float T; };
template <> struct AccT<ACC_F64> { typedef double T; };

RSVD_DEV void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}

template <typename TA, typename TB, typename TC, int AL, int ACC>
__global__ void __launch_bounds__(256)
k_tile_mm(const MMDesc* __restrict__ md, const int* __restrict__ off, int C) {
  typedef typename AccT<ACC>::T T;
  __shared__ T As[16][64 + 4];
  __shared__ T Bs[16][64 + 4];
  const int t = blockIdx.x;
  const int c = find_chan(off, C, t);
  const MMDesc d = md[c];
  int local = t - off[c];
  const int per_split = d.mt * d.nt;
  const int split = local / per_split;
  local -= split * per_split;
  const int mi = local / d.nt, ni = local % d.nt;
  if (d.sym && ni < mi) return;                  // Gram: upper tile triangle only
  const int m0 = mi * 64, n0 = ni * 64;
  const int ncols = d.ncols_dev ? min(d.n, *d.ncols_dev) : d.n;
  if (n0 >= ncols) return;
  const int kb = split * d.kchunk;
  const int ke = min(d.k, kb + d.kchunk);
  const TA* __restrict__ A = (const TA*)d.A;
  const TB* __restrict__ B = (const TB*)d.B;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

  T acc[4][4], cmp[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { acc[i][j] = 0; cmp[i][j] = 0; }

  for (int k0 = kb; k0 < ke; k0 += 16) {
    // A tile: 64 (m) x 16 (k) -> As[k][m]
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int e = tid + p * 256;
      int mm, kk;
      if (AL == AROW) { mm = e >> 4; kk = e & 15; }   // contiguous along k
      else { mm = e & 63; kk = e >> 6; }              // contiguous along m
      const int gm = m0 + mm, gk = k0 + kk;
      T v = 0;
      if (gm < d.m && gk < ke)
        v = (T)(AL == AROW ? A[(int64_t)gm * d.lda + gk] : A[gm + (int64_t)gk * d.lda]);
      As[kk][mm] = v;
    }
    // B tile: 16 (k) x 64 (n), column-major source -> Bs[k][n]
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int e = tid + p * 256;
      const int kk = e & 15, nn = e >> 4;
      const int gk = k0 + kk, gn = n0 + nn;
      T v = 0;
      if (gn < ncols && gk < ke) v = (T)B[gk + (int64_t)gn * d.ldb];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (ACC == ACC_DOT2) {
            const float p = (float)a[i] * (float)b[j];
            const float pe = fmaf((float)a[i], (float)b[j], -p);
            float s, se;
            two_sum((float)acc[i][j], p, s, se);
            acc[i][j] = s;
            cmp[i][j] += se + pe;
          } else {
            acc[i][j] = fma(a[i], b[j], acc[i][j]);
          }
        }
    }
    __syncthreads();
  }

  TC* __restrict__ Cp = (TC*)d.Cm + (d.mode == MM_PARTIAL ? (int64_t)split * d.pstride : 0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= d.m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= ncols) continue;
      double v = (double)acc[i][j] + (ACC == ACC_DOT2 ? (double)cmp[i][j] : 0.0);
      if (d.colscale) v *= d.colscale[gn];
      TC* dst = Cp + gm + (int64_t)gn * d.ldc;
      if (d.mode == MM_ATOMIC) atomicAdd(dst, (TC)v);
      else *dst = (TC)v;
      if (d.nsl > 0) {                   // BF16 word slices of the FP32 result
        float r = (float)v;
        for (int s = 0; s < d.nsl; ++s) {
          const __nv_bfloat16 h = __float2bfloat16_rn(r);
          d.sl[s][gm + (int64_t)gn * d.ldsl] = h;
          r -= __bfloat162float(h);
        }
      }
    }
  }
}

// Sum the split partials of a Gram / inner product in a fixed order; for a
// symmetric Gram only the upper tiles were written, so mirror them.
__global__ void k_reduce_partials(const MMDesc* __restrict__ md, double* const* __restrict__ outp,
                                  int C) {
  const int c = blockIdx.y;
  const MMDesc d = md[c];
  double* out = outp[c];
  const int total = d.m * d.n;
  const int ks = d.ks;
  const double* P = (const double*)d.Cm;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    int i = e % d.m, j = e / d.m;
    int si = i, sj = j;
    if (d.sym && (i / 64) > (j / 64)) { si = j; sj = i; }
    double s = 0.0;
    for (int p = 0; p < ks; ++p) s += P[(int64_t)p * d.pstride + si + (int64_t)sj * d.ldc];
    out[i + (int64_t)j * d.m] = s;
  }
  (void)C;
}

void launch_tile_mm(MMKind kind, const MMDesc* d_md, const int* d_off, int C, int tiles,
                    cudaStream_t st) {
  if (tiles <= 0) return;
  switch (kind) {
    case MMK_DENSE_F64: k_tile_mm<double, double, double, AROW, ACC_F64><<<tiles, 256, 0, st>>>(d_md, d_off, C); break;
    case MMK_GRAM_F64:  k_tile_mm<double, double, double, AROW, ACC_F64><<<tiles, 256, 0, st>>>(d_md, d_off, C); break;
    case MMK_NN_F64:    k_tile_mm<double, double, double, ACOL, ACC_F64><<<tiles, 256, 0, st>>>(d_md, d_off, C); break;
    case MMK_GRAM_DOT2: k_tile_mm<float, float, double, AROW, ACC_DOT2><<<tiles, 256, 0, st>>>(d_md, d_off, C); break;
    case MMK_NN_F32_F64B: k_tile_mm<float, double, float, ACOL, ACC_F32><<<tiles, 256, 0, st>>>(d_md, d_off, C); break;
    case MMK_NN_F32_OUT64: k_tile_mm<float, double, double, ACOL, ACC_F32><<<tiles, 256, 0, st>>>(d_md, d_off, C); break;
  }
}

void launch_reduce_partials(const MMDesc* d_md, double* const* d_out, int C, int max_elems,
                            cudaStream_t st) {
  if (C <= 0) return;
  dim3 grid((max_elems + 255) / 256 < 64 ? (max_elems + 255) / 256 : 64, C);
  if (grid.x == 0) grid.x = 1;
  k_reduce_partials<<<grid, 256, 0, st>>>(d_md, d_out, C);
}

}  // namespace rsvd
