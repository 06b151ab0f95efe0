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
  // descriptor fields into registers (a struct copy would live on the stack)
  const MMDesc* __restrict__ dp = md + c;
  const int dm = dp->m, dn = dp->n, dk = dp->k, mt = dp->mt, nt = dp->nt, kchunk = dp->kchunk;
  const int mode = dp->mode, sym = dp->sym, nsl = dp->nsl;
  const int64_t lda = dp->lda, ldb = dp->ldb, ldc = dp->ldc, pstride = dp->pstride, ldsl = dp->ldsl;
  const double* __restrict__ colscale = dp->colscale;
  __nv_bfloat16* sl0 = dp->sl[0];
  __nv_bfloat16* sl1 = dp->sl[1];
  __nv_bfloat16* sl2 = dp->sl[2];
  int local = t - off[c];
  const int per_split = mt * nt;
  const int split = local / per_split;
  local -= split * per_split;
  const int mi = local / nt, ni = local % nt;
  if (sym && ni < mi) return;                    // Gram: upper tile triangle only
  const int m0 = mi * 64, n0 = ni * 64;
  const int ncols = dp->ncols_dev ? min(dn, *dp->ncols_dev) : dn;
  if (n0 >= ncols) return;
  const int kb = split * kchunk;
  const int ke = min(dk, kb + kchunk);
  const TA* __restrict__ A = (const TA*)dp->A;
  const TB* __restrict__ B = (const TB*)dp->B;
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
      if (gm < dm && gk < ke)
        v = (T)(AL == AROW ? A[(int64_t)gm * lda + gk] : A[gm + (int64_t)gk * lda]);
      As[kk][mm] = v;
    }
    // B tile: 16 (k) x 64 (n), column-major source -> Bs[k][n]
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int e = tid + p * 256;
      const int kk = e & 15, nn = e >> 4;
      const int gk = k0 + kk, gn = n0 + nn;
      T v = 0;
      if (gn < ncols && gk < ke) v = (T)B[gk + (int64_t)gn * ldb];
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

  TC* __restrict__ Cp = (TC*)dp->Cm + (mode == MM_PARTIAL ? (int64_t)split * pstride : 0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= dm) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= ncols) continue;
      double v = (double)acc[i][j] + (ACC == ACC_DOT2 ? (double)cmp[i][j] : 0.0);
      if (colscale) v *= colscale[gn];
      TC* dst = Cp + gm + (int64_t)gn * ldc;
      if (mode == MM_ATOMIC) atomicAdd(dst, (TC)v);
      else *dst = (TC)v;
      if (nsl > 0) {                     // BF16 word slices of the FP32 result
        const int64_t o = gm + (int64_t)gn * ldsl;
        float r = (float)v;
        __nv_bfloat16 h = __float2bfloat16_rn(r);
        sl0[o] = h;
        if (nsl > 1) {
          r -= __bfloat162float(h);
          h = __float2bfloat16_rn(r);
          sl1[o] = h;
          if (nsl > 2) {
            r -= __bfloat162float(h);
            sl2[o] = __float2bfloat16_rn(r);
          }
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
    case MMK_DENSE_F64: k_tile_mm<double, double, double, AROW, ACC_F64><<<tiles, 256, 0, st>>>(d_md, d_off, C); note_launch(); break;
    case MMK_GRAM_F64:  k_tile_mm<double, double, double, AROW, ACC_F64><<<tiles, 256, 0, st>>>(d_md, d_off, C); note_launch(); break;
    case MMK_NN_F64:    k_tile_mm<double, double, double, ACOL, ACC_F64><<<tiles, 256, 0, st>>>(d_md, d_off, C); note_launch(); break;
    case MMK_GRAM_DOT2: k_tile_mm<float, float, double, AROW, ACC_DOT2><<<tiles, 256, 0, st>>>(d_md, d_off, C); note_launch(); break;
    case MMK_NN_F32_F64B: k_tile_mm<float, double, float, ACOL, ACC_F32><<<tiles, 256, 0, st>>>(d_md, d_off, C); note_launch(); break;
    case MMK_NN_F32_OUT64: k_tile_mm<float, double, double, ACOL, ACC_F32><<<tiles, 256, 0, st>>>(d_md, d_off, C); note_launch(); break;
    case MMK_GRAM_F32: k_tile_mm<float, float, double, AROW, ACC_F32><<<tiles, 256, 0, st>>>(d_md, d_off, C); note_launch(); break;
  }
}

void launch_reduce_partials(const MMDesc* d_md, double* const* d_out, int C, int max_elems,
                            cudaStream_t st) {
  if (C <= 0) return;
  dim3 grid((max_elems + 255) / 256 < 64 ? (max_elems + 255) / 256 : 64, C);
  if (grid.x == 0) grid.x = 1;
  k_reduce_partials<<<grid, 256, 0, st>>>(d_md, d_out, C);
  note_launch();
}

}  // namespace rsvd
