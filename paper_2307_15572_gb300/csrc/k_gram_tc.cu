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
// into the four accumulators, and the epilogue (eight warps: TMEM lane
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

// 2^k as FP32 for k <= 127 (0 below the normal range).
RSVD_DEV float gt_pow2f(int k) { return k < -126 ? 0.0f : __uint_as_float((uint32_t)(127 + k) << 23); }

RSVD_DEV uint32_t gt_pack(float lo, float hi) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);   // both exact: at most nine significant bits
  return *reinterpret_cast<const uint32_t*>(&p);
}

RSVD_DEV void gt_st16(uint32_t saddr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(saddr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// Slice pairs (s, t) in issue order and their accumulator (0: level 2,
// 1: level 3, 2: level 4, 3: levels 5-7, smallest first).
__constant__ unsigned char c_gt_pairs[21][3] = {
    {0, 0, 0}, {0, 1, 1}, {1, 0, 1}, {0, 2, 2}, {1, 1, 2}, {2, 0, 2},
    {0, 5, 3}, {1, 4, 3}, {2, 3, 3}, {3, 2, 3}, {4, 1, 3}, {5, 0, 3},
    {0, 4, 3}, {1, 3, 3}, {2, 2, 3}, {3, 1, 3}, {4, 0, 3},
    {0, 3, 3}, {1, 2, 3}, {2, 1, 3}, {3, 0, 3}};

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
  for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++it) {
    const GramTcDesc* g = gd + gt_chan(gd, C, t);
    const int local = t - g->tile0;
    const int r0 = local * GT_ROWS;
    const int n = g->n, l = g->l;

    // ---- the thread's 64 entries and the column maximum
    float v[64];
    float mx = 0.0f;
    if (m < l) {
      const float* src = g->Y + (int64_t)m * g->ldy + r0 + 64 * h;
      const int rows = n - (r0 + 64 * h);
      if (rows >= 64) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const float4 f = __ldg(reinterpret_cast<const float4*>(src) + q);
          v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 64; ++k) v[k] = k < rows ? __ldg(src + k) : 0.0f;
      }
#pragma unroll
      for (int k = 0; k < 64; ++k) mx = fmaxf(mx, fabsf(v[k]));
    } else {
#pragma unroll
      for (int k = 0; k < 64; ++k) v[k] = 0.0f;
    }
    smax[h * 128 + m] = mx;
    __syncthreads();
    // cm < 2^e for normal cm; zero and subnormal maxima take the floor -126,
    // a non-finite one the ceiling (and propagates through the slices)
    const float cm = fmaxf(smax[m], smax[128 + m]);
    int e = (int)((__float_as_uint(cm) >> 23) & 0xFFu) - 126;
    e = max(-126, min(126, e));
    if (h == 0) g->exps[local * 128 + m] = e;
    const float sc = gt_pow2f(-e);

    // ---- six slices, 8 rows (one 16-byte chunk per slice) at a time
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      uint32_t w[GT_SLICES][4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        float x0 = v[8 * q + 2 * p] * sc, x1 = v[8 * q + 2 * p + 1] * sc;
#pragma unroll
        for (int s = 0; s < GT_SLICES; ++s) {
          const float up = __uint_as_float((uint32_t)(127 + 8 * (s + 1)) << 23);
          const float dn = __uint_as_float((uint32_t)(127 - 8 * (s + 1)) << 23);
          const float d0 = rintf(x0 * up) * dn, d1 = rintf(x1 * up) * dn;
          x0 -= d0;                                    // exact: the bits below 2^(-8(s+1))
          x1 -= d1;
          w[s][p] = gt_pack(d0, d1);
        }
      }
      const uint32_t off = (uint32_t)(h * GT_HALF_BYTES + m * 128 + ((q ^ (m & 7)) << 4));
#pragma unroll
      for (int s = 0; s < GT_SLICES; ++s)
        gt_st16(sbase + (uint32_t)(s * GT_SLICE_BYTES) + off, w[s][0], w[s][1], w[s][2], w[s][3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();

    // ---- the 21 slice-pair products into the four accumulators
    if (tid == 0) {
      tc_fence_after();
      const uint32_t idesc = idesc_bf16(128);
      int last = -1;
#pragma unroll 1
      for (int p = 0; p < 21; ++p) {
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
        tmem_ld16_nw(ta + 384, ar);
        tmem_wait_ld();
        if (i < l) {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int j = j0 + jj;
            if (j < i || j >= l) continue;
            const float v2 = __uint_as_float(a2[jj]), v3 = __uint_as_float(a3[jj]);
            const float v4 = __uint_as_float(a4[jj]), vr = __uint_as_float(ar[jj]);
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
        const float r = gt_pow2f(F - f);
        sh *= r;
        sl *= r;
        F = f;
      }
      const float w = gt_pow2f(f - F);
      gt_df_add(sh, sl, bh * w, bl * w);
    }
    const double u = __longlong_as_double((long long)(1023 + F) << 52);   // 2^F, |F| <= 252
    const double v = ((double)sh + (double)sl) * u;
    g->G[i + (int64_t)j * l] = v;
    g->G[j + (int64_t)i * l] = v;
  }
  (void)C;
}

int launch_gram_tc(const GramTcDesc* d_gd, int C, int tiles, int* d_err, cudaStream_t st) {
  if (tiles <= 0 || C <= 0) return 0;
  const cudaError_t e = cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, GT_SMEM);
  if (e != cudaSuccess) return (int)e;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      nsm < 1)
    nsm = 148;
  const int grid = tiles < nsm ? tiles : nsm;
  k_gram_tc<<<grid, GT_THREADS, GT_SMEM, st>>>(d_gd, C, tiles, d_err);
  note_launch();
  k_gram_tc_reduce<<<dim3(64, C), 256, 0, st>>>(d_gd, C);
  note_launch();
  return (int)cudaGetLastError();
}

int gram_tc_part_floats(int n) { return ((n + GT_ROWS - 1) / GT_ROWS) * GT_PART; }

}  // namespace rsvd
