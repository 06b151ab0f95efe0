// Gram matrices G = Y^T Y of tall FP32 panels (n x l, l <= 128) on the
// tensor cores, to FP64-grade accuracy: the Grams of CholeskyQR (Fukaya,
// Nakatsukasa, Yanagisawa & Yamamoto, 2014) on the mixed path, where Y has a
// condition number up to ~1e5 and an FP32 Gram would lose the Cholesky.
//
// Error-free splitting in the manner of Ozaki, Ogita, Oishi & Rump (Numer.
// Algorithms 59, 2012).  Each 128-row tile of Y is scaled per column by a
// power of two, x = y 2^-e with |x| < 1, and cut into six fixed-point slices
//     x = a_1 + ... + a_6 (+ r),   a_k = rint(r_(k-1) 2^(8k)) 2^(-8k),
// each an integer of at most nine bits times a power of two: exact in BF16.
// Then x_i x_j = sum over slice pairs a_(i,s) a_(j,t), grouped by level
// s + t.  Over one tile every product of levels 2, 3 and 4 is a multiple of
// its level's unit and every partial sum stays below 2^24 units (level 2:
// 128 * 2^16, level 3: 128 * 2 * 2^15, level 4: 128 * 5 * 2^13), so the
// tensor core sums those levels exactly whatever the rounding of its FP32
// accumulation.  Levels 5-7 (below 2^-23 of the total) share a fourth,
// rounded accumulator; higher levels (below 2^-47) are dropped, and each
// entry's remainder r is at most 2^-49 of its tile-column maximum.
//
// k_gram_tc (persistent, one 256-thread CTA per SM, 192 KiB of slices, all
// 512 TMEM columns): per tile every thread loads 64 rows of one column, the
// column maxima give the exponents, the slices go to shared memory in the
// 128B-swizzled K-major layout (M = columns of Y, K = rows of the tile), one
// thread issues the 21 slice-pair MMAs (M = N = 128, K = 16, eight k steps)
// into the four accumulators (an FP32-grade form takes three slices and the
// six exact products of levels 2-4), and the epilogue (eight warps: TMEM lane
// quarter x column half) adds the three exact levels and the rest into a
// double-float pair (hi, lo) per entry -- exact but for the rest -- and
// stores the upper triangle with the tile's column exponents.
// k_gram_tc_reduce: per entry, the tiles' pairs brought to a common power of
// two (exact scaling), summed in double-float (Knuth's TwoSum), converted to
// FP64 and scaled; the upper triangle is mirrored.
#include "kernels.h"
#include "tc_ptx.cuh"

namespace rsvd {

namespace {
constexpr int GT_ROWS = 128;                         // rows of Y per tile: the MMA's k extent
constexpr int GT_SLICES = 6;
constexpr int GT_HALF_BYTES = 128 * 64 * 2;          // 128 columns x 64 rows of BF16: one swizzle column
constexpr int GT_SLICE_BYTES = 2 * GT_HALF_BYTES;    // 32 KiB
constexpr int GT_THREADS = 256;
constexpr int GT_MISC = 2048;                        // mbarrier, TMEM slot, column maxima
constexpr int GT_SMEM = GT_SLICES * GT_SLICE_BYTES + 1024 + GT_MISC;
constexpr int GT_PART = 2 * 128 * 128;               // floats per tile: hi plane, lo plane
}  // namespace

RSVD_DEV int gt_chan(const GramTcDesc* __restrict__ gd, int C, int t) {
  int lo = 0, hi = C - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (gd[mid].tile0 <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Rows 64h .. 64h + 63 of tile t, column m (zero outside n x l): 16-byte
// loads along the column.
RSVD_DEV void gt_load(const GramTcDesc* __restrict__ gd, int C, int t, int m, int h, float (&v)[64]) {
  const GramTcDesc* g = gd + gt_chan(gd, C, t);
  const int r0 = (t - g->tile0) * GT_ROWS + 64 * h;
  const int rows = g->n - r0;
  if (m < g->l && rows >= 64) {
    const float4* src = reinterpret_cast<const float4*>(g->Y + (int64_t)m * g->ldy + r0);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float4 f = __ldg(src + q);
      v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
    }
  } else {
    const float* src = g->Y + (int64_t)m * g->ldy + r0;
    const bool col = m < g->l;
#pragma unroll
    for (int k = 0; k < 64; ++k) v[k] = (col && k < rows) ? __ldg(src + k) : 0.0f;
  }
}

// Slice pairs (s, t) in issue order and their accumulator (0: level 2,
// 1: level 3, 2: level 4, 3: levels 5-7, smallest first).
__constant__ unsigned char c_gt_pairs[21][3] = {
    {0, 0, 0}, {0, 1, 1}, {1, 0, 1}, {0, 2, 2}, {1, 1, 2}, {2, 0, 2},
    {0, 5, 3}, {1, 4, 3}, {2, 3, 3}, {3, 2, 3}, {4, 1, 3}, {5, 0, 3},
    {0, 4, 3}, {1, 3, 3}, {2, 2, 3}, {3, 1, 3}, {4, 0, 3},
    {0, 3, 3}, {1, 2, 3}, {2, 1, 3}, {3, 0, 3}};

// NS = 6: 21 products, FP64-grade; NS = 3: the 6 products of levels 2-4
// (all exact), the Gram of the operand rounded to 24 fractional bits of its
// tile-column maxima: FP32-grade.
template <int NS>
__global__ void __launch_bounds__(GT_THREADS, 1)
k_gram_tc(const GramTcDesc* __restrict__ gd, int C, int tiles, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bar = (uint64_t*)(base + GT_SLICES * GT_SLICE_BYTES);
  uint32_t* tmem_slot = (uint32_t*)(bar + 1);
  float* smax = (float*)(base + GT_SLICES * GT_SLICE_BYTES + 64);   // [2][128]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sbase = smem_addr(base);
  const int m = tid & 127, h = tid >> 7;             // slicing: column m, rows 64h .. 64h + 63
  const int qd = warp & 3, chalf = warp >> 2;        // epilogue: TMEM lanes 32 qd.., columns 64 chalf..
  int it = 0;
  bool healthy = true;
  float v[64];
  if (blockIdx.x < tiles) gt_load(gd, C, blockIdx.x, m, h, v);
  for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++it) {
    const GramTcDesc* g = gd + gt_chan(gd, C, t);
    const int local = t - g->tile0;
    const int l = g->l;

    // ---- the column maximum of the loaded entries
    float mx = 0.0f;
#pragma unroll
    for (int k = 0; k < 64; ++k) mx = fmaxf(mx, fabsf(v[k]));
    smax[h * 128 + m] = mx;
    __syncthreads();
    // a non-finite maximum takes the ceiling exponent (and propagates through
    // the slices)
    const int e = slice_exp(fmaxf(smax[m], smax[128 + m]));
    if (h == 0) g->exps[local * 128 + m] = e;
    slice_row64<NS>(v, pow2f_exp(-e), m, h, [&](int s, uint32_t off, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
      st_shared_v4(sbase + (uint32_t)(s * GT_SLICE_BYTES) + off, a, b, c, d);
    });
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    // the next tile's entries load while this one is multiplied and stored
    if (t + (int)gridDim.x < tiles) gt_load(gd, C, t + gridDim.x, m, h, v);

    // ---- the 21 slice-pair products into the four accumulators
    if (tid == 0) {
      tc_fence_after();
      const uint32_t idesc = idesc_bf16(128);
      int last = -1;
#pragma unroll 1
      for (int p = 0; p < (NS == 6 ? 21 : 6); ++p) {
        const int sa = c_gt_pairs[p][0], sb = c_gt_pairs[p][1], acc = c_gt_pairs[p][2];
        const bool first = acc != last;
        last = acc;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const uint32_t ko = (uint32_t)((kk >> 2) * GT_HALF_BYTES + (kk & 3) * 32);
          const uint64_t ad = sdesc_sw128(sbase + (uint32_t)(sa * GT_SLICE_BYTES) + ko);
          const uint64_t bd = sdesc_sw128(sbase + (uint32_t)(sb * GT_SLICE_BYTES) + ko);
          mma_bf16(tmem + (uint32_t)(acc * 128), ad, bd, idesc, (first && kk == 0) ? 0u : 1u);
        }
      }
      mma_commit(bar);
    }

    // ---- epilogue: (hi, lo) of each upper-triangle entry
    int ok = 1;
    if (lane == 0) ok = mbar_wait(bar, (uint32_t)(it & 1)) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) {
      if (lane == 0) set_err(err, DERR_TIMEOUT_EPI);
      healthy = false;
    }
    tc_fence_after();
    if (healthy) {
      const int i = qd * 32 + lane;                    // entry row = column i of Y
      float* Ph = g->part + (int64_t)local * GT_PART;
      float* Pl = Ph + 128 * 128;
#pragma unroll 1
      for (int u = 0; u < 4; ++u) {
        const int j0 = chalf * 64 + u * 16;
        if (j0 >= l || j0 + 15 < qd * 32) continue;   // warp-uniform: no entry of the warp is needed
        uint32_t a2[16], a3[16], a4[16], ar[16];
        const uint32_t ta = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)j0;
        tmem_ld16_nw(ta, a2);
        tmem_ld16_nw(ta + 128, a3);
        tmem_ld16_nw(ta + 256, a4);
        if (NS == 6) tmem_ld16_nw(ta + 384, ar);
        tmem_wait_ld();
        if (i < l) {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int j = j0 + jj;
            if (j < i || j >= l) continue;
            const float v2 = __uint_as_float(a2[jj]), v3 = __uint_as_float(a3[jj]);
            const float v4 = __uint_as_float(a4[jj]), vr = NS == 6 ? __uint_as_float(ar[jj]) : 0.0f;
            float s1 = v2 + v3, bb = s1 - v2;
            const float e1 = (v2 - (s1 - bb)) + (v3 - bb);
            const float s2 = s1 + v4;
            bb = s2 - s1;
            const float e2 = (s1 - (s2 - bb)) + (v4 - bb);
            const float lo = (e1 + e2) + vr;          // e1 + e2 is exact
            const float hi = s2 + lo;
            Ph[i + j * 128] = hi;
            Pl[i + j * 128] = lo - (hi - s2);
          }
        }
      }
    }
    tc_fence_before();
    if (__syncthreads_or(healthy ? 0 : 1)) break;     // also frees the slices and TMEM for the next tile
  }
  if (!healthy && tid == 0 && it > 0) {
    // give MMAs still in flight a bounded chance to finish before TMEM goes
    mbar_wait(bar, (uint32_t)(it & 1));
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// Double-float accumulation (s_hi, s_lo) += (b_hi, b_lo): TwoSum of the
// leading parts, then the trailing parts and a renormalisation.
RSVD_DEV void gt_df_add(float& sh, float& sl, float bh, float bl) {
  const float s = sh + bh, bb = s - sh;
  float e = (sh - (s - bb)) + (bh - bb);
  e += sl + bl;
  sh = s + e;
  sl = e - (sh - s);
}

__global__ void __launch_bounds__(256)
k_gram_tc_reduce(const GramTcDesc* __restrict__ gd, int C) {
  const GramTcDesc* g = gd + blockIdx.y;
  const int l = g->l, T = g->ntiles;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < l * l; e += gridDim.x * blockDim.x) {
    const int i = e % l, j = e / l;
    if (i > j) continue;
    float sh = 0.0f, sl = 0.0f;
    int F = -1000;                                    // exponent of the running sum's unit
    for (int t = 0; t < T; ++t) {
      const float* P = g->part + (int64_t)t * GT_PART + i + j * 128;
      const int* ex = g->exps + t * 128;
      const int f = __ldg(ex + i) + __ldg(ex + j);
      const float bh = __ldg(P), bl = __ldg(P + 128 * 128);
      if (f > F) {                                    // a larger unit: rescale the sum (exactly)
        const float r = pow2f_exp(F - f);
        sh *= r;
        sl *= r;
        F = f;
      }
      const float w = pow2f_exp(f - F);
      gt_df_add(sh, sl, bh * w, bl * w);
    }
    const double u = __longlong_as_double((long long)(1023 + F) << 52);   // 2^F, |F| <= 252
    const double v = ((double)sh + (double)sl) * u;
    g->G[i + (int64_t)j * l] = v;
    g->G[j + (int64_t)i * l] = v;
  }
  (void)C;
}

int launch_gram_tc(const GramTcDesc* d_gd, int C, int tiles, int fp32_grade, int* d_err, cudaStream_t st) {
  if (tiles <= 0 || C <= 0) return 0;
  // both forms take the six-slice shared memory: one CTA per SM, so that no
  // second CTA waits on the TMEM allocation
  const cudaError_t e = cudaFuncSetAttribute(fp32_grade ? k_gram_tc<3> : k_gram_tc<6>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, GT_SMEM);
  if (e != cudaSuccess) return (int)e;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      nsm < 1)
    nsm = 148;
  const int grid = tiles < nsm ? tiles : nsm;
  if (fp32_grade) k_gram_tc<3><<<grid, GT_THREADS, GT_SMEM, st>>>(d_gd, C, tiles, d_err);
  else k_gram_tc<6><<<grid, GT_THREADS, GT_SMEM, st>>>(d_gd, C, tiles, d_err);
  note_launch();
  k_gram_tc_reduce<<<dim3(64, C), 256, 0, st>>>(d_gd, C);
  note_launch();
  return (int)cudaGetLastError();
}

int gram_tc_part_floats(int n) { return ((n + GT_ROWS - 1) / GT_ROWS) * GT_PART; }

}  // namespace rsvd
