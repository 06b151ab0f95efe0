// Tall-times-small products C = A B on the tensor cores: A an n x K FP32
// panel (K <= 128, column-major), B a K x N matrix (N <= 128, FP32 or FP64,
// column-major, optionally with its columns scaled), C FP32 (with optional
// BF16 words of the result) or FP64.  These are CholeskyQR's Q = Y R^{-1}
// (Fukaya et al., 2014) and the lifts U = Q X, V = W X Sigma^{-1} of
// Fig. 1 step 3 on the mixed path.
//
// The same error-free splitting as the tensor-core Gram (Ozaki, Ogita, Oishi
// & Rump, 2012).  Each row of a 128-row tile of A is scaled by a power of two
// 2^-e_r and cut into three 8-bit fixed-point BF16 slices; each column of B
// likewise (scale 2^-f_j), once per call by k_nn_tc_prep, into a
// shared-memory image that the product kernel copies in with one bulk copy
// per channel.  The slice products of levels 2 to 4 are summed exactly over
// K <= 128 in three TMEM accumulators (level 2: 128 * 2^16 units, 3:
// 128 * 2 * 2^15, 4: 128 * 5 * 2^13, all below 2^24); the three products
// of levels 5 and 6 (each term below 2^-25 of the row-maximum x
// column-maximum scale, like the rounding of the operands) are dropped.  C is
// the product of A and B, each rounded to 24 fractional bits of its row
// (column) maximum, up to those dropped terms, then rounded to FP32 (or
// widened to FP64 from that FP32 value): the accuracy of an FP32 product.
//
// k_nn_tc: persistent, one 256-thread CTA per SM, 96 KiB of A slices and
// 96 KiB of B image, 512 TMEM columns.  Per tile every thread loads 64
// entries of one row of A (a warp reads 32 consecutive rows of a column:
// coalesced), the row maxima give the exponents, the slices go to shared
// memory in the 128B-swizzled K-major layout, the next tile's entries are
// loaded into registers while one thread issues the six slice-pair products
// (M = N = 128, K = 16, up to eight k steps) and eight warps (TMEM lane
// quarter x column half) add the levels, scale by 2^(e_r + f_j) and store
// column by column (coalesced).
#include "kernels.h"
#include "tc_ptx.cuh"

namespace rsvd {

namespace {
constexpr int NT_SLICES = 3;
constexpr int NT_SLICE_BYTES = 2 * 16384;                 // 128 rows x 128 k of BF16
constexpr int NT_IMG_BYTES = NT_SLICES * NT_SLICE_BYTES;  // 96 KiB per operand
constexpr int NT_THREADS = 256;
constexpr int NT_MISC = 2048;                             // barriers, TMEM slot, maxima, exponents
constexpr int NT_SMEM = 2 * NT_IMG_BYTES + 1024 + NT_MISC;
}  // namespace

int nn_tc_img_bytes() { return NT_IMG_BYTES; }

// ------------------------------------------------------------ B images
// Grid (channel, 4): block y takes 32 output columns j (rows of the B
// image); thread = column j, half h of the k range.  B' = B diag(colscale)
// rounded to FP32.
__global__ void __launch_bounds__(64) k_nn_tc_prep(const NnTcDesc* __restrict__ nd) {
  const NnTcDesc* g = nd + blockIdx.x;
  if (g->cond && !(*g->cond & FLAG_SHIFTED)) return;
  __shared__ float smax[2][32];
  const int tid = threadIdx.x, jl = tid & 31, h = tid >> 5;
  const int j = blockIdx.y * 32 + jl;
  const int K = g->K, N = g->N;
  float v[64];
  float mx = 0.0f;
  if (j < N) {
    const double cs = g->colscale ? g->colscale[j] : 1.0;
#pragma unroll
    for (int k = 0; k < 64; ++k) {
      const int kk = 64 * h + k;
      float x = 0.0f;
      if (kk < K) {
        if (g->b64) {
          const double b = ((const double*)g->B)[kk + (int64_t)j * g->ldb];
          x = f64_to_f32_rn(g->colscale ? b * cs : b);
        } else {
          const float b = ((const float*)g->B)[kk + (int64_t)j * g->ldb];
          x = g->colscale ? f64_to_f32_rn((double)b * cs) : b;
        }
      }
      v[k] = x;
      mx = fmaxf(mx, fabsf(x));
    }
  } else {
#pragma unroll
    for (int k = 0; k < 64; ++k) v[k] = 0.0f;
  }
  smax[h][jl] = mx;
  __syncthreads();
  const int f = slice_exp(fmaxf(smax[0][jl], smax[1][jl]));
  if (h == 0) g->fexp[j] = f;
  unsigned char* img = (unsigned char*)g->bimg;     // the shared-memory image, in global memory
  slice_row64<NT_SLICES>(v, pow2f_exp(-f), j, h, [&](int s, uint32_t off, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    *reinterpret_cast<uint4*>(img + (size_t)s * NT_SLICE_BYTES + off) = make_uint4(a, b, c, d);
  });
}

RSVD_DEV int nt_chan(const NnTcDesc* __restrict__ nd, int C, int t) {
  int lo = 0, hi = C - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (nd[mid].tile0 <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Slice pairs (A slice, B slice, accumulator = level - 2) in issue order.
__constant__ unsigned char c_nt_pairs[6][3] = {{0, 0, 0}, {0, 1, 1}, {1, 0, 1}, {0, 2, 2}, {1, 1, 2}, {2, 0, 2}};

// First tile at or after t (stepping by `step`) whose channel is not skipped.
RSVD_DEV int nt_live(const NnTcDesc* __restrict__ nd, int C, int t, int tiles, int step) {
  for (; t < tiles; t += step) {
    const NnTcDesc* g = nd + nt_chan(nd, C, t);
    if (!g->cond || (*g->cond & FLAG_SHIFTED)) break;
  }
  return t;
}

// Row r0 + r of tile t, columns 64h .. 64h + 63 (zero outside n x K): a warp
// reads 32 consecutive rows of a column per load.
RSVD_DEV void nt_load(const NnTcDesc* __restrict__ nd, int C, int t, int r, int h, float (&v)[64]) {
  const NnTcDesc* g = nd + nt_chan(nd, C, t);
  const int row = (t - g->tile0) * 128 + r;
  const int n = g->n, K = g->K;
  const int64_t lda = g->lda;
  const float* src = g->A + row + (int64_t)(64 * h) * lda;
  const bool live = row < n;
#pragma unroll
  for (int k = 0; k < 64; ++k) v[k] = (live && 64 * h + k < K) ? __ldg(src + (int64_t)k * lda) : 0.0f;
}

struct NtOut {
  float* C32;
  double* C64;
  int64_t ldc;
  __nv_bfloat16* sl[3];
  int64_t ldsl;
};

// Epilogue of one thread: tile row `grow` (TMEM lane), 64 columns from
// 64 chalf, 16 per round trip.  MODE 0: FP32, 1: FP32 and NSL BF16 words,
// 2: FP64 (from the FP32 value, exactly scaled).
template <int MODE, int NSL>
RSVD_DEV void nt_epilogue(uint32_t ta, int chalf, int ncols, int grow, bool live, int er, const int* scol,
                          const NtOut& o) {
  const float se = pow2f_exp(er);
#pragma unroll 1
  for (int u = 0; u < 4; ++u) {
    const int j0 = chalf * 64 + u * 16;
    if (j0 >= ncols) break;                           // warp-uniform
    uint32_t a2[16], a3[16], a4[16];
    tmem_ld16_nw(ta + (uint32_t)j0, a2);
    tmem_ld16_nw(ta + 128 + (uint32_t)j0, a3);
    tmem_ld16_nw(ta + 256 + (uint32_t)j0, a4);
    tmem_wait_ld();
    if (!live) continue;
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      const int j = j0 + jj;
      // small levels first; every level sum is exact, the two adds round once each
      const float s = (__uint_as_float(a4[jj]) + __uint_as_float(a3[jj])) + __uint_as_float(a2[jj]);
      const int fj = scol[j];
      if (j < ncols) {
        if (MODE == 2) {
          o.C64[grow + (int64_t)j * o.ldc] = scale_pow2_f64(f32_to_f64(s * se), fj);
        } else {
          const float val = (s * se) * pow2f_exp(fj);
          o.C32[grow + (int64_t)j * o.ldc] = val;
          if (MODE == 1) {
            const int64_t oo = grow + (int64_t)j * o.ldsl;
            float rem = val;
#pragma unroll
            for (int w = 0; w < NSL; ++w) {
              const __nv_bfloat16 q = __float2bfloat16_rn(rem);
              o.sl[w][oo] = q;
              rem -= __bfloat162float(q);
            }
          }
        }
      }
    }
  }
}

__global__ void __launch_bounds__(NT_THREADS, 1)
k_nn_tc(const NnTcDesc* __restrict__ nd, int C, int tiles, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* misc = base + 2 * NT_IMG_BYTES;
  uint64_t* bar_b = (uint64_t*)misc;                  // B image landed
  uint64_t* bar_m = bar_b + 1;                        // MMAs done
  uint32_t* tmem_slot = (uint32_t*)(bar_m + 1);
  float* smax = (float*)(misc + 64);                  // [2][128] row maxima of A
  int* srow = (int*)(misc + 64 + 1024);               // [128] row exponents
  int* scol = srow + 128;                             // [128] column exponents of B
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    mbar_init(bar_b, 1);
    mbar_init(bar_m, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sa_base = smem_addr(base), sb_base = sa_base + NT_IMG_BYTES;
  const int r = tid & 127, h = tid >> 7;              // loading: row r, k = 64h .. 64h + 63
  const int qd = warp & 3, chalf = warp >> 2;         // epilogue: TMEM lanes 32 qd.., columns 64 chalf..
  int it = 0, nb = 0;                                 // MMA rounds, B loads of this CTA
  const NnTcDesc* cur = nullptr;
  bool healthy = true;
  float v[64];
  int t = nt_live(nd, C, blockIdx.x, tiles, gridDim.x);
  if (t < tiles) nt_load(nd, C, t, r, h, v);
  while (t < tiles) {
    const NnTcDesc* g = nd + nt_chan(nd, C, t);
    const int r0 = (t - g->tile0) * 128;
    const bool newb = g != cur;
    if (newb) {
      if (tid == 0) {
        mbar_arrive_expect_tx(bar_b, (uint32_t)NT_IMG_BYTES);
        bulk_g2s(base + NT_IMG_BYTES, g->bimg, (uint32_t)NT_IMG_BYTES, bar_b);
      }
      if (tid < 128) scol[tid] = g->fexp[tid];
      cur = g;
    }

    // ---- the row maximum and the slices of the loaded entries
    float mx = 0.0f;
#pragma unroll
    for (int k = 0; k < 64; ++k) mx = fmaxf(mx, fabsf(v[k]));
    smax[h * 128 + r] = mx;
    __syncthreads();
    const int e = slice_exp(fmaxf(smax[r], smax[128 + r]));
    if (h == 0) srow[r] = e;
    slice_row64<NT_SLICES>(v, pow2f_exp(-e), r, h, [&](int s, uint32_t off, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
      st_shared_v4(sa_base + (uint32_t)(s * NT_SLICE_BYTES) + off, a, b, c, d);
    });
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    // the next tile's entries load while this one is multiplied and stored
    const int tn = nt_live(nd, C, t + gridDim.x, tiles, gridDim.x);
    if (tn < tiles) nt_load(nd, C, tn, r, h, v);

    // ---- the slice-pair products
    if (tid == 0) {
      bool ok = true;
      if (newb) {
        ok = mbar_wait(bar_b, (uint32_t)(nb & 1));
        ++nb;
        if (!ok) set_err(err, DERR_TIMEOUT_TMA);
      }
      tc_fence_after();
      if (ok) {
        const uint32_t idesc = idesc_bf16(128);
        const int nks = (g->K + 15) >> 4;
        int last = -1;
#pragma unroll 1
        for (int p = 0; p < 6; ++p) {
          const int sa = c_nt_pairs[p][0], sb = c_nt_pairs[p][1], acc = c_nt_pairs[p][2];
          const bool first = acc != last;
          last = acc;
#pragma unroll 1
          for (int kk = 0; kk < nks; ++kk) {
            const uint32_t ko = (uint32_t)((kk >> 2) * 16384 + (kk & 3) * 32);
            const uint64_t ad = sdesc_sw128(sa_base + (uint32_t)(sa * NT_SLICE_BYTES) + ko);
            const uint64_t bd = sdesc_sw128(sb_base + (uint32_t)(sb * NT_SLICE_BYTES) + ko);
            mma_bf16(tmem + (uint32_t)(acc * 128), ad, bd, idesc, (first && kk == 0) ? 0u : 1u);
          }
        }
      }
      mma_commit(bar_m);          // also after a failed wait: completes when prior MMAs do
    }

    // ---- epilogue (the error word is read before the wait, so that its
    // load overlaps the products)
    const int errv = *(volatile int*)err;
    int ok = 1;
    if (lane == 0) ok = mbar_wait(bar_m, (uint32_t)(it & 1)) ? 1 : 0;
    ++it;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) {
      if (lane == 0) set_err(err, DERR_TIMEOUT_EPI);
      healthy = false;
    }
    if (healthy) healthy = errv == 0;
    tc_fence_after();
    if (healthy) {
      const int i = qd * 32 + lane;                   // tile row
      const int grow = r0 + i;
      const bool live = grow < g->n;
      const int ncols = g->ncols_dev ? min(g->N, *g->ncols_dev) : g->N;
      NtOut o;
      o.C32 = g->C32; o.C64 = g->C64; o.ldc = g->ldc;
      o.sl[0] = g->sl[0]; o.sl[1] = g->sl[1]; o.sl[2] = g->sl[2]; o.ldsl = g->ldsl;
      const int nsl = g->nsl;
      const uint32_t ta = tmem + ((uint32_t)(qd * 32) << 16);
      const int er = srow[i];
      if (o.C64) nt_epilogue<2, 0>(ta, chalf, ncols, grow, live, er, scol, o);
      else if (nsl == 0) nt_epilogue<0, 0>(ta, chalf, ncols, grow, live, er, scol, o);
      else if (nsl == 1) nt_epilogue<1, 1>(ta, chalf, ncols, grow, live, er, scol, o);
      else if (nsl == 2) nt_epilogue<1, 2>(ta, chalf, ncols, grow, live, er, scol, o);
      else nt_epilogue<1, 3>(ta, chalf, ncols, grow, live, er, scol, o);
    }
    tc_fence_before();
    if (__syncthreads_or(healthy ? 0 : 1)) break;    // also frees the slices and TMEM for the next tile
    t = tn;
  }
  if (!healthy && tid == 0 && it > 0) mbar_wait(bar_m, (uint32_t)((it - 1) & 1));
  if (tid == 0 && nb > 0) mbar_wait(bar_b, (uint32_t)((nb - 1) & 1));   // no bulk copy left in flight
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

int launch_nn_tc(const NnTcDesc* d_nd, int C, int tiles, int* d_err, cudaStream_t st) {
  if (tiles <= 0 || C <= 0) return 0;
  k_nn_tc_prep<<<dim3(C, 4), 64, 0, st>>>(d_nd);
  note_launch();
  const cudaError_t e = cudaFuncSetAttribute(k_nn_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, NT_SMEM);
  if (e != cudaSuccess) return (int)e;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      nsm < 1)
    nsm = 148;
  const int grid = tiles < nsm ? tiles : nsm;
  k_nn_tc<<<grid, NT_THREADS, NT_SMEM, st>>>(d_nd, C, tiles, d_err);
  note_launch();
  return (int)cudaGetLastError();
}

}  // namespace rsvd
