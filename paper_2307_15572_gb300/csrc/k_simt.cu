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

RSVD_DEV void store_out(float* d, float v, bool atomic) { if (atomic) atomicAdd(d, v); else *d = v; }
RSVD_DEV void store_out(double* d, float v, bool atomic) {
  const double w = f32_to_f64(v);
  if (atomic) atomicAdd(d, w); else *d = w;
}

RSVD_DEV unsigned int pack_bf2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (unsigned int)__bfloat16_as_ushort(lo) | ((unsigned int)__bfloat16_as_ushort(hi) << 16);
}

RSVD_DEV float to_f32(float x) { return x; }
RSVD_DEV float to_f32(double x) { return f64_to_f32_rn(x); }   // integer-pipe rounding

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
  if (dp->cond && !(*dp->cond & FLAG_SHIFTED)) return;
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
  // each warp owns a 4 x 8 patch of the 16 x 16 grid of 4 x 4 output blocks
  // (rows ty, columns tx): reads of B are conflict-free, and in a Gram's
  // diagonal tile two warps lie wholly below the diagonal and skip their
  // arithmetic (the reduction mirrors the upper triangle)
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int ty = 4 * (w >> 1) + (lane >> 3), tx = 8 * (w & 1) + (lane & 7);
  const bool lower = sym && mi == ni && ty > tx;

  T acc[4][4], cmp[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { acc[i][j] = 0; cmp[i][j] = 0; }

  if constexpr (ACC == ACC_DOT2) {
    // The compensated Gram: the next 16-wide k slice is loaded into registers
    // while the current one is consumed from the other shared-memory buffer,
    // so the global loads overlap the arithmetic and one barrier separates
    // the slices (the generic loop below waits on both).
    __shared__ T As2[2][16][64 + 4];
    __shared__ T Bs2[2][16][64 + 4];
    T ra[4], rb[4];
    auto load = [&](int k0) {
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int e = tid + p * 256;
        int mm, kk;
        if (AL == AROW) { mm = e >> 4; kk = e & 15; }
        else { mm = e & 63; kk = e >> 6; }
        const int gm = m0 + mm, gk = k0 + kk;
        ra[p] = (gm < dm && gk < ke) ? (T)(AL == AROW ? A[(int64_t)gm * lda + gk] : A[gm + (int64_t)gk * lda]) : (T)0;
        const int kb2 = e & 15, nn = e >> 4;
        const int gk2 = k0 + kb2, gn = n0 + nn;
        rb[p] = (gn < ncols && gk2 < ke) ? (T)B[gk2 + (int64_t)gn * ldb] : (T)0;
      }
    };
    auto store = [&](int buf) {
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int e = tid + p * 256;
        int mm, kk;
        if (AL == AROW) { mm = e >> 4; kk = e & 15; }
        else { mm = e & 63; kk = e >> 6; }
        As2[buf][kk][mm] = ra[p];
        Bs2[buf][e & 15][e >> 4] = rb[p];
      }
    };
    if (kb < ke) {
      load(kb);
      store(0);
      __syncthreads();
    }
    int buf = 0;
    for (int k0 = kb; k0 < ke; k0 += 16, buf ^= 1) {
      const bool more = k0 + 16 < ke;
      if (more) load(k0 + 16);
      if (!lower) {
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
          float a[4], b[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = (float)As2[buf][kk][ty * 4 + i];
#pragma unroll
          for (int j = 0; j < 4; ++j) b[j] = (float)Bs2[buf][kk][tx * 4 + j];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const float p = a[i] * b[j];
              const float pe = fmaf(a[i], b[j], -p);
              float sv, se;
              two_sum((float)acc[i][j], p, sv, se);
              acc[i][j] = sv;
              cmp[i][j] += se + pe;
            }
        }
      }
      if (more) store(buf ^ 1);
      __syncthreads();
    }
  } else
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
    if (!lower) {
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
    }
    __syncthreads();
  }

  TC* __restrict__ Cp = (TC*)dp->Cm + (mode == MM_PARTIAL ? (int64_t)split * pstride : 0);
  if (lower) return;                             // never read (mirrored from the upper triangle)
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
      else if (mode == MM_SUB) *dst = *dst - (TC)v;
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

// Epilogue of the 128 x 128 tiles: the thread's 8 x 8 block (rows tx*4+q and
// 64+tx*4+q, columns ty*4+j and 64+ty*4+j) to the output -- store, atomic add
// (k split), subtract, or split partial -- with the optional column scale and
// BF16 word slices of the result.
template <typename TC>
RSVD_DEV void mm128_store(const MMDesc* __restrict__ dp, const float (&acc)[8][8], int split, int m0, int n0,
                          int ncols, int tx, int ty) {
  const int dm = dp->m, mode = dp->mode, nsl = dp->nsl;
  const int64_t ldc = dp->ldc, pstride = dp->pstride, ldsl = dp->ldsl;
  const double* __restrict__ colscale = dp->colscale;
  TC* __restrict__ Cp = (TC*)dp->Cm + (mode == MM_PARTIAL ? (int64_t)split * pstride : 0);
  __nv_bfloat16* sl0 = dp->sl[0];
  __nv_bfloat16* sl1 = dp->sl[1];
  __nv_bfloat16* sl2 = dp->sl[2];
  // each thread owns rows {r4, r4+1, r4+2, r4+3} (two such groups) of 8
  // columns: full groups go out as one vector store per column
  const bool vec_ok = (mode == MM_STORE) && (sizeof(TC) == 4) && ((ldc & 3) == 0) &&
                      ((((uintptr_t)Cp) & 15) == 0);
#pragma unroll
  for (int ig = 0; ig < 2; ++ig) {
    const int r4 = m0 + ig * 64 + tx * 4;
    if (r4 >= dm) continue;
    const bool full = r4 + 3 < dm;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gn = n0 + (j < 4 ? ty * 4 + j : 64 + ty * 4 + j - 4);
      if (gn >= ncols) continue;
      float v[4];
      const float cs = colscale ? f64_to_f32_rn(colscale[gn]) : 1.0f;
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = acc[ig * 4 + q][j] * cs;
      TC* dst = Cp + r4 + (int64_t)gn * ldc;
      if (mode == MM_SUB) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (r4 + q < dm) dst[q] = dst[q] - (TC)v[q];
      } else if (full && vec_ok) {
        *(float4*)dst = make_float4(v[0], v[1], v[2], v[3]);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (r4 + q < dm) store_out(dst + q, v[q], mode == MM_ATOMIC);
      }
      if (nsl > 0) {
        const int64_t o = r4 + (int64_t)gn * ldsl;
        __nv_bfloat16 w0[4], w1[4], w2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float r = v[q];
          w0[q] = __float2bfloat16_rn(r);
          r -= __bfloat162float(w0[q]);
          w1[q] = __float2bfloat16_rn(r);
          r -= __bfloat162float(w1[q]);
          w2[q] = __float2bfloat16_rn(r);
        }
        if (full && ((ldsl & 3) == 0)) {
          *(uint2*)(sl0 + o) = make_uint2(pack_bf2(w0[0], w0[1]), pack_bf2(w0[2], w0[3]));
          if (nsl > 1) *(uint2*)(sl1 + o) = make_uint2(pack_bf2(w1[0], w1[1]), pack_bf2(w1[2], w1[3]));
          if (nsl > 2) *(uint2*)(sl2 + o) = make_uint2(pack_bf2(w2[0], w2[1]), pack_bf2(w2[2], w2[3]));
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (r4 + q >= dm) continue;
            sl0[o + q] = w0[q];
            if (nsl > 1) sl1[o + q] = w1[q];
            if (nsl > 2) sl2[o + q] = w2[q];
          }
        }
      }
    }
  }
}

// FP32-compute tiles (Grams of FP32 data, triangular solve, lift): 128 x 128
// output tile, k steps of 8, 256 threads with an 8 x 8 register block each
// (two 4 x 4 quadrants, so shared-memory reads are float4 and conflict-free),
// next k step prefetched into registers while the current one is used.
template <typename TA, typename TB, typename TC, int AL, int ACC>
__global__ void __launch_bounds__(256, ACC == ACC_DOT2 ? 1 : 2)
k_tile_mm128(const MMDesc* __restrict__ md, const int* __restrict__ off, int C) {
  // rows padded by 4 floats: the staging stores (8 consecutive threads on 8
  // different k rows) hit 8 distinct banks, and rows stay 16-byte aligned
  __shared__ __align__(16) float As[2][8][132];
  __shared__ __align__(16) float Bs[2][8][132];
  const int t = blockIdx.x;
  const int c = find_chan(off, C, t);
  const MMDesc* __restrict__ dp = md + c;
  if (dp->cond && !(*dp->cond & FLAG_SHIFTED)) return;
  const int dm = dp->m, dn = dp->n, dk = dp->k, mt = dp->mt, nt = dp->nt, kchunk = dp->kchunk;
  const int sym = dp->sym;
  const int64_t lda = dp->lda, ldb = dp->ldb;
  int local = t - off[c];
  const int per_split = mt * nt;
  const int split = local / per_split;
  local -= split * per_split;
  const int mi = local / nt, ni = local % nt;
  if (sym && ni < mi) return;
  const int m0 = mi * 128, n0 = ni * 128;
  const int ncols = dp->ncols_dev ? min(dn, *dp->ncols_dev) : dn;
  if (n0 >= ncols) return;
  const int kb = split * kchunk;
  const int ke = min(dk, kb + kchunk);
  const TA* __restrict__ A = (const TA*)dp->A;
  const TB* __restrict__ B = (const TB*)dp->B;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

  float acc[8][8], cmp[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) { acc[i][j] = 0.0f; cmp[i][j] = 0.0f; }

  // staging: 4 A and 4 B elements per thread per k step
  float ra[4], rb[4];
  auto gload = [&](int k0) {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int e = tid + p * 256;
      int mm, kk;
      if (AL == AROW) { kk = e & 7; mm = e >> 3; } else { mm = e & 127; kk = e >> 7; }
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.0f;
      if (gm < dm && gk < ke) v = to_f32(AL == AROW ? A[(int64_t)gm * lda + gk] : A[gm + (int64_t)gk * lda]);
      ra[p] = v;
      const int kb2 = e & 7, nn = e >> 3;
      const int gn = n0 + nn, gk2 = k0 + kb2;
      float w = 0.0f;
      if (gn < ncols && gk2 < ke) w = to_f32(B[gk2 + (int64_t)gn * ldb]);
      rb[p] = w;
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int e = tid + p * 256;
      int mm, kk;
      if (AL == AROW) { kk = e & 7; mm = e >> 3; } else { mm = e & 127; kk = e >> 7; }
      As[buf][kk][mm] = ra[p];
      Bs[buf][e & 7][e >> 3] = rb[p];
    }
  };
  int buf = 0;
  if (kb < ke) { gload(kb); sstore(0); }
  __syncthreads();
  for (int k0 = kb; k0 < ke; k0 += 8) {
    const bool more = k0 + 8 < ke;
    if (more) gload(k0 + 8);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      // rows follow tx (4 consecutive rows per thread -> vector stores of the
      // column-major result), columns follow ty
      const float4 a0 = *(const float4*)&As[buf][kk][tx * 4];
      const float4 a1 = *(const float4*)&As[buf][kk][64 + tx * 4];
      const float4 b0 = *(const float4*)&Bs[buf][kk][ty * 4];
      const float4 b1 = *(const float4*)&Bs[buf][kk][64 + ty * 4];
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (ACC == ACC_DOT2) {
            const float p = a[i] * b[j];
            const float pe = fmaf(a[i], b[j], -p);
            float s, se;
            two_sum(acc[i][j], p, s, se);
            acc[i][j] = s;
            cmp[i][j] += se + pe;
          } else {
            acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
          }
        }
    }
    if (more) {
      sstore(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }

  mm128_store<TC>(dp, acc, split, m0, n0, ncols, tx, ty);
}

// The same 128 x 128 FP32 tiles with both operands FP32 in global memory,
// fed by cp.async into a 4-stage shared-memory ring: the loads of k step
// s + 3 are in flight while step s is computed, so the global latency (the
// tile's k extent is often only l = 128, 16 steps) is hidden instead of
// exposed once per step as with register staging.  Tall column-major A
// (ACOL) moves in 16-byte copies where the leading dimension and base allow,
// row-style A (a Gram's Y^T) and B in 4-byte copies; out-of-range elements
// are zero-filled by the copy itself.
RSVD_DEV void cp_async4(void* sdst, const void* gsrc, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
               "l"(gsrc), "r"(bytes) : "memory");
}
RSVD_DEV void cp_async16(void* sdst, const void* gsrc, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
               "l"(gsrc), "r"(bytes) : "memory");
}
RSVD_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
RSVD_DEV void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <typename TC, int AL>
__global__ void __launch_bounds__(256, 2)
k_tile_mm128_cp(const MMDesc* __restrict__ md, const int* __restrict__ off, int C) {
  constexpr int S = 4;
  __shared__ __align__(16) float As[S][8][132];
  __shared__ __align__(16) float Bs[S][8][132];
  const int t = blockIdx.x;
  const int c = find_chan(off, C, t);
  const MMDesc* __restrict__ dp = md + c;
  if (dp->cond && !(*dp->cond & FLAG_SHIFTED)) return;
  const int dm = dp->m, dn = dp->n, dk = dp->k, mt = dp->mt, nt = dp->nt, kchunk = dp->kchunk;
  const int sym = dp->sym;
  const int64_t lda = dp->lda, ldb = dp->ldb;
  int local = t - off[c];
  const int per_split = mt * nt;
  const int split = local / per_split;
  local -= split * per_split;
  const int mi = local / nt, ni = local % nt;
  if (sym && ni < mi) return;
  const int m0 = mi * 128, n0 = ni * 128;
  const int ncols = dp->ncols_dev ? min(dn, *dp->ncols_dev) : dn;
  if (n0 >= ncols) return;
  const int kb = split * kchunk;
  const int ke = min(dk, kb + kchunk);
  const float* __restrict__ A = (const float*)dp->A;
  const float* __restrict__ B = (const float*)dp->B;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const bool a16 = AL == ACOL && (lda & 3) == 0 && (((uintptr_t)A) & 15) == 0;
  const int nk = ke > kb ? (ke - kb + 7) / 8 : 0;

  auto issue = [&](int step) {
    const int buf = step % S, k0 = kb + 8 * step;
    if (AL == ACOL && a16) {
      const int kk = tid >> 5, mm = 4 * (tid & 31);
      const int gm = m0 + mm, gk = k0 + kk;
      int bytes = 0;
      if (gk < ke && gm < dm) bytes = 4 * min(4, dm - gm);
      cp_async16(&As[buf][kk][mm], bytes ? (const void*)(A + gm + (int64_t)gk * lda) : (const void*)A, bytes);
    } else {
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int e = tid + p * 256;
        int mm, kk;
        if (AL == AROW) { kk = e & 7; mm = e >> 3; } else { mm = e & 127; kk = e >> 7; }
        const int gm = m0 + mm, gk = k0 + kk;
        const bool in = gm < dm && gk < ke;
        const float* src = in ? (AL == AROW ? A + (int64_t)gm * lda + gk : A + gm + (int64_t)gk * lda) : A;
        cp_async4(&As[buf][kk][mm], src, in ? 4 : 0);
      }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int e = tid + p * 256;
      const int kk = e & 7, nn = e >> 3;
      const int gk = k0 + kk, gn = n0 + nn;
      const bool in = gn < ncols && gk < ke;
      cp_async4(&Bs[buf][kk][nn], in ? (const void*)(B + gk + (int64_t)gn * ldb) : (const void*)B, in ? 4 : 0);
    }
  };

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
#pragma unroll
  for (int s0 = 0; s0 < S - 1; ++s0) {
    if (s0 < nk) issue(s0);
    cp_async_commit();
  }
  for (int step = 0; step < nk; ++step) {
    cp_async_wait<S - 2>();
    __syncthreads();                       // step's tiles landed; step - 1's buffer is free
    if (step + S - 1 < nk) issue(step + S - 1);
    cp_async_commit();
    const int buf = step % S;
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const float4 a0 = *(const float4*)&As[buf][kk][tx * 4];
      const float4 a1 = *(const float4*)&As[buf][kk][64 + tx * 4];
      const float4 b0 = *(const float4*)&Bs[buf][kk][ty * 4];
      const float4 b1 = *(const float4*)&Bs[buf][kk][64 + ty * 4];
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
  }
  cp_async_wait<0>();
  mm128_store<TC>(dp, acc, split, m0, n0, ncols, tx, ty);
}

// Sum the split partials of a Gram / inner product in a fixed order; for a
// symmetric Gram only the upper tiles were written, so mirror them.
__global__ void k_reduce_partials(const MMDesc* __restrict__ md, double* const* __restrict__ outp,
                                  int C) {
  const int c = blockIdx.y;
  const MMDesc d = md[c];
  if (d.cond && !(*d.cond & FLAG_SHIFTED)) return;
  double* out = outp[c];
  const int total = d.m * d.n;
  const int ks = d.ks;
  const double* P = (const double*)d.Cm;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    int i = e % d.m, j = e / d.m;
    int si = i, sj = j;
    if (d.sym && i > j) { si = j; sj = i; }      // only the upper triangle is computed
    double s = 0.0;
    for (int p = 0; p < ks; ++p) s += P[(int64_t)p * d.pstride + si + (int64_t)sj * d.ldc];
    out[i + (int64_t)j * d.m] = s;
  }
  (void)C;
}

int tile_of(MMKind kind) {
  switch (kind) {
    case MMK_NN_F32_F64B: case MMK_NN_F32_OUT64: case MMK_GRAM_F32: case MMK_NN_F32:
    case MMK_NN_F32_OUT64_B32: return 128;
    default: return 64;
  }
}

void launch_tile_mm(MMKind kind, const MMDesc* d_md, const int* d_off, int C, int tiles,
                    cudaStream_t st) {
  if (tiles <= 0) return;
  switch (kind) {
    case MMK_DENSE_F64: k_tile_mm<double, double, double, AROW, ACC_F64><<<tiles, 256, 0, st>>>(d_md, d_off, C); break;
    case MMK_GRAM_F64:  k_tile_mm<double, double, double, AROW, ACC_F64><<<tiles, 256, 0, st>>>(d_md, d_off, C); break;
    case MMK_NN_F64:    k_tile_mm<double, double, double, ACOL, ACC_F64><<<tiles, 256, 0, st>>>(d_md, d_off, C); break;
    case MMK_GRAM_DOT2: k_tile_mm<float, float, double, AROW, ACC_DOT2><<<tiles, 256, 0, st>>>(d_md, d_off, C); break;
    case MMK_NN_F32_F64B: k_tile_mm128<float, double, float, ACOL, ACC_F32><<<tiles, 256, 0, st>>>(d_md, d_off, C); break;
    case MMK_NN_F32_OUT64: k_tile_mm128<float, double, double, ACOL, ACC_F32><<<tiles, 256, 0, st>>>(d_md, d_off, C); break;
    case MMK_GRAM_F32: k_tile_mm128_cp<double, AROW><<<tiles, 256, 0, st>>>(d_md, d_off, C); break;
    case MMK_NN_F32: k_tile_mm128_cp<float, ACOL><<<tiles, 256, 0, st>>>(d_md, d_off, C); break;
    case MMK_NN_F32_OUT64_B32: k_tile_mm128_cp<double, ACOL><<<tiles, 256, 0, st>>>(d_md, d_off, C); break;
  }
  note_launch();
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
