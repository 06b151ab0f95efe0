// Tensor-core passes over V for the mixed path: Y = V X on sm_103a.  The
// same kernel also generates the entries of a tile rule (TC_RULE): with H the
// n x M matrix of sqrt(w_m) g_m(x_j) in FP16 words, a panel of rule rows is
// H H_panel^T, to which the epilogue adds the hash noise before splitting the
// entries into the words the next pass reads.
//
// This is the contraction of Fig. 1 step 1 (Z = V P) and of the projection
// (Y^T = V Q, V symmetric) when V is held as a sum of BF16 words,
// V ~ V_0 + V_1 (+ V_2), and X likewise: Y = sum over word pairs (a, b) with
// a + b < max(SA, SX) of V_a X_b, accumulated in FP32.  Two words carry ~16
// significant bits of each FP64 entry, three ~24.
//
// Structure (persistent CTAs, one per SM, each taking 128-row tiles of Y with
// all of their columns in turn):
//   * warp 0, one thread: TMA producer.  For each 64-wide k step it waits for
//     the stage to be free, arms the stage's mbarrier with the byte count and
//     issues 2-D tiled bulk copies (128B swizzle) of the V word tiles
//     (128 x 64) and X word tiles (BN x 64);
//   * warp 1, one thread: MMA issuer.  Waits for the stage, issues
//     tcgen05.mma.cta_group::1.kind::f16 (M = 128, N = BN, K = 16) for each
//     word pair and 16-wide k slice into one TMEM accumulator, then
//     tcgen05.commit to the stage's "empty" barrier; a final commit signals
//     the epilogue;
//   * all four warps: epilogue.  tcgen05.ld (32 lanes x 32 bit, 16 columns at
//     a time) from the warp's TMEM lane quarter, coalesced column-major
//     stores (or red.global.add when k is split across CTAs).
// Every mbarrier wait is bounded (~2 s of clock64); on expiry the thread
// records an error code, stops issuing work, and the CTA still drains its
// own copies and frees TMEM before returning.
#include <cudaTypedefs.h>
#include <stdio.h>
#include <stdlib.h>

#include "tc_gemm.h"
#include "tc_ptx.cuh"

namespace rsvd {

static constexpr int BM = 128;
static constexpr int BK = 64;
static constexpr int A_TILE_BYTES = BM * BK * 2;   // 16 KiB
static constexpr int SMEM_BUDGET = 220 * 1024;

int tc_stage_bytes(int sa, int sx, int bn) { return sa * A_TILE_BYTES + sx * bn * BK * 2; }

int tc_stages(int sa, int sx, int bn) {
  const int sb = tc_stage_bytes(sa, sx, bn);
  int st = (SMEM_BUDGET - 1024 - 256) / sb;
  if (st > 8) st = 8;
  return st;
}

// PTX helpers (mbarriers, TMA, TMEM, tcgen05.mma): tc_ptx.cuh
// ------------------------------------------------------------------ kernel
// The tensor core rounds its FP32 accumulation toward zero, so one TMEM
// accumulator summed over all n/16 MMA steps would carry a bias growing
// linearly with n (~n/16 * 2^-24 relative: 5e-5 at n = 12,000).  The k loop
// is therefore cut into chunks of CHUNK_KT 64-wide steps; each chunk is
// accumulated from zero in one of two TMEM buffers and the four epilogue
// warps add it into FP32 registers (round to nearest) while the next chunk
// runs in the other buffer.  The bias is then bounded by one chunk's worth
// (4 * CHUNK_KT truncations, ~2e-6), and the register sum is unbiased.
// A channel may ask for shorter chunks (chunk_kt): the tile-rule generator,
// whose k extent is only M, takes one 64-wide step per chunk.
static constexpr int CHUNK_KT = 8;
// Register accumulator width of the epilogue: 160 columns for most launches;
// the wide instantiation (176) serves the passes whose column count splits
// better into two tiles of up to 176 than into three of up to 160 (the tile
// rule's 330 columns), at the cost of 16 more registers per thread.
static constexpr int BN_NARROW = TC_BN_NARROW;
static constexpr int BN_MAX = TC_BN_MAX;
static constexpr int NTHREADS = 192;          // warps 0-3 epilogue, 4 producer, 5 MMA
static constexpr int NTHREADS_RULE = 320;     // generation: warps 0-3 and 6-9 epilogue (two groups)

// Work item -> channel, k split, output tile.
struct TcItem {
  const TcChan* ch;
  int m0, n0, kb, nk;
  int local;                 // item index within its channel
};

RSVD_DEV void tc_item(const TcChan* __restrict__ chs, int C, int item, int bn, TcItem& I) {
  int lo = 0, hi = C - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (chs[mid].item0 <= item) lo = mid; else hi = mid - 1;
  }
  const TcChan* ch = chs + lo;
  int local = item - ch->item0;
  I.ch = ch;
  I.local = local;
  const int per_split = ch->mt * ch->nt;
  const int split = local / per_split;
  local -= split * per_split;
  const int mi = local / ch->nt, ni = local % ch->nt;
  I.m0 = mi * BM;
  I.n0 = ni * bn;
  const int kt_total = (ch->n + BK - 1) / BK;
  I.kb = split * ch->kt_per_split;
  I.nk = max(0, min(kt_total, I.kb + ch->kt_per_split) - I.kb);
}

// Final processing of 16 generated columns of one tile row (one lane = one
// row j of the generated block = matrix column j; column col = matrix row
// r0 + col): noise, words, energy, remainder.  The inner hash of the noise is
// mix(min(i, j) * C1 + key): the row's is computed once per tile (hrow), the
// 16 columns' by 16 lanes and broadcast.  All lanes take part (shuffles).
// The 16 entries are made first, with no branch between them, so their hash
// chains interleave; then the words of the live ones are stored (`live`
// masks rows past the end, nj the columns past the end).  Constants:
// amp_s = sqrt(3) eta 2^-24 (the noise numerator is an odd integer below
// 2^24), hinv2 = hscale^-2 (a power of two: the scaling is exact).
template <int NW, bool WY>
RSVD_DEV void rule_group(const uint32_t (&r)[16], int row, bool live, int col0, int ncols, int r0, uint32_t hrow,
                         uint32_t key, float amp_s, float hinv2, __nv_bfloat16* W0, __nv_bfloat16* W1,
                         __nv_bfloat16* W2, int64_t ldw, float* Y, int64_t ldy, float& s2, float& r2, int lane) {
  const int i0 = r0 + col0;
  const uint32_t hcol = lowbias32((uint32_t)(i0 + (lane & 15)) * 0x9E3779B1u + key);
  const uint32_t rowc = (uint32_t)row * 0x85EBCA77u;
  float v[16];
#pragma unroll
  for (int jj = 0; jj < 16; ++jj) {
    const uint32_t hc = __shfl_sync(0xffffffffu, hcol, jj);
    const int i = i0 + jj;
    const uint32_t h = lowbias32(row <= i ? (hrow ^ ((uint32_t)i * 0x85EBCA77u)) : (hc ^ rowc));
    const float eta = (float)(2 * (int)(h >> 8) + 1 - (1 << 24)) * amp_s;
    v[jj] = fmaf(__uint_as_float(r[jj]), hinv2, eta);
  }
  if (!live) return;
  const int nj = ncols - col0;                         // uniform across the warp
#pragma unroll
  for (int jj = 0; jj < 16; ++jj) {
    if (jj >= nj) break;
    const float x = v[jj];
    s2 = fmaf(x, x, s2);
    const int64_t o = row + (int64_t)(col0 + jj) * ldw;
    if (NW > 0) {
      __nv_bfloat16 q = __float2bfloat16_rn(x);
      W0[o] = q;
      float rem = x - __bfloat162float(q);             // exact
      if (NW > 1) {
        q = __float2bfloat16_rn(rem);
        W1[o] = q;
        rem -= __bfloat162float(q);
      }
      if (NW > 2) {
        q = __float2bfloat16_rn(rem);
        W2[o] = q;
        rem -= __bfloat162float(q);
      }
      r2 = fmaf(rem, rem, r2);
    }
    if (WY) Y[row + (int64_t)(col0 + jj) * ldy] = x;
  }
}

// Persistent: each CTA takes items blockIdx.x, blockIdx.x + gridDim.x, ...
// The k-step counter (stage ring) and the chunk counter (TMEM ping-pong)
// run on across items, so the producer loads item i+1 and the MMA warp
// computes it while the epilogue warps still store item i.
template <int SA, int SX, bool RULE, int BNM = BN_NARROW>
__global__ void __launch_bounds__(RULE ? NTHREADS_RULE : NTHREADS, 1)
k_tc_gemm(const TcChan* __restrict__ chs, int C, int items, int bn, int stages, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int SB = SA * A_TILE_BYTES + SX * bn * BK * 2;
  uint64_t* full = (uint64_t*)(base + (size_t)stages * SB);
  uint64_t* empty = full + stages;
  uint64_t* acc_full = empty + stages;     // [2] MMA -> epilogue
  uint64_t* acc_empty = acc_full + 2;      // [2] epilogue -> MMA (128 arrivals)
  uint32_t* tmem_slot = (uint32_t*)(acc_empty + 2);
  int* consumed = (int*)(tmem_slot + 1);   // generation: (chunk, warp) pairs released, in order

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // two accumulation buffers, plus (generation) one region per epilogue
  // group where it keeps its running sums
  uint32_t ncols_alloc = 32;
  while ((int)ncols_alloc < (RULE ? 4 : 2) * bn) ncols_alloc <<= 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], 128); }
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, ncols_alloc);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 4) {
    if (lane == 0) {
      // ---------------- TMA producer
      int g = 0;                                   // k steps issued by this CTA
      bool ok = true;
      const TcChan* last = nullptr;
      for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
        TcItem I;
        tc_item(chs, C, item, bn, I);
        if (I.ch != last) {
          for (int a = 0; a < SA; ++a) tmap_acquire(&I.ch->tmA[a]);
          for (int x = 0; x < SX; ++x) tmap_acquire(&I.ch->tmX[x]);
          last = I.ch;
        }
        for (int it = 0; it < I.nk; ++it) {
          const int s = g % stages;
          const uint32_t ph = (uint32_t)(g / stages) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u)) { set_err(err, DERR_TIMEOUT_TMA); ok = false; break; }
          mbar_arrive_expect_tx(&full[s], (uint32_t)SB);
          unsigned char* st = base + (size_t)s * SB;
          const int kx = (I.kb + it) * BK;
          for (int a = 0; a < SA; ++a) tma_load_2d(st + a * A_TILE_BYTES, &I.ch->tmA[a], &full[s], kx, I.m0);
          for (int x = 0; x < SX; ++x)
            tma_load_2d(st + SA * A_TILE_BYTES + x * bn * BK * 2, &I.ch->tmX[x], &full[s], kx, I.n0);
          ++g;
        }
      }
      // drain: the last copy issued into each stage has landed
      for (int s = 0; s < stages && s < g; ++s) {
        const int lastg = s + ((g - 1 - s) / stages) * stages;
        if (!mbar_wait(&full[s], (uint32_t)(lastg / stages) & 1u)) set_err(err, DERR_TIMEOUT_TMA);
      }
    }
    __syncwarp();
  } else if (warp == 5) {
    if (lane == 0) {
      // ---------------- MMA issuer
      // the tile-rule generator multiplies FP16 factor words, the passes BF16 words
      const uint32_t idesc = RULE ? idesc_f16(bn) : idesc_bf16(bn);
      bool ok = true;
      int g = 0, gc = 0;                           // k steps, chunks consumed by this CTA
      for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
        TcItem I;
        tc_item(chs, C, item, bn, I);
        const int chunk = I.ch->chunk_kt > 0 ? I.ch->chunk_kt : CHUNK_KT;
        const int nchunks = (I.nk + chunk - 1) / chunk;
        int it = 0;
        for (int c = 0; c < nchunks && ok; ++c, ++gc) {
          const int b = gc & 1;
          if (gc >= 2 && !mbar_wait(&acc_empty[b], (uint32_t)((gc >> 1) - 1) & 1u)) {
            set_err(err, DERR_TIMEOUT_MMA);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dt = tmem + (uint32_t)(b * bn);
          const int itend = min(I.nk, it + chunk);
          bool zero = true;                          // first MMA of the chunk overwrites
          for (; it < itend; ++it, ++g) {
            const int s = g % stages;
            const uint32_t ph = (uint32_t)(g / stages) & 1u;
            if (!mbar_wait(&full[s], ph)) { set_err(err, DERR_TIMEOUT_MMA); ok = false; break; }
            tc_fence_after();
            const uint32_t sa0 = smem_addr(base + (size_t)s * SB);
            const uint32_t sx0 = sa0 + SA * A_TILE_BYTES;
            // small word products first, the leading pair (0, 0) last: the
            // round-toward-zero accumulation then loses least while the
            // running sum is small
#pragma unroll
            for (int pr = (SA > SX ? SA : SX) - 1; pr >= 0; --pr) {
#pragma unroll
              for (int a = 0; a < SA; ++a) {
#pragma unroll
                for (int x = 0; x < SX; ++x) {
                  if (a + x != pr) continue;
#pragma unroll
                  for (int kk = 0; kk < BK / 16; ++kk) {
                    const uint64_t ad = sdesc_sw128(sa0 + a * A_TILE_BYTES + kk * 32);
                    const uint64_t bd = sdesc_sw128(sx0 + x * bn * BK * 2 + kk * 32);
                    mma_bf16(dt, ad, bd, idesc, zero ? 0u : 1u);
                    zero = false;
                  }
                }
              }
            }
            mma_commit(&empty[s]);
          }
          mma_commit(&acc_full[b]);     // also issued after an error: completes when prior MMAs do
        }
      }
      // every MMA has completed before TMEM is released (bounded)
      if (gc > 0) {
        const int b = (gc - 1) & 1;
        if (!mbar_wait(&acc_full[b], (uint32_t)((gc - 1) >> 1) & 1u)) set_err(err, DERR_TIMEOUT_MMA);
      }
    }
    __syncwarp();
  } else if constexpr (RULE) {
    // ---------------- generation epilogue: two groups of four warps take the
    // CTA's items alternately (group g: items 2t + g of its sequence); warp w
    // reads TMEM lanes 32 (w mod 4) .. + 31 = rows of the tile.  Chunk sums
    // are added (round to nearest) into the group's own TMEM region, 16
    // columns per rolled step (the per-entry code is long: unrolled over
    // every column it would not fit the instruction cache).  Chunks are taken
    // in order across the groups -- a group waits on a buffer's barrier only
    // once the chunk before it was released, so no parity wait runs two
    // phases ahead (it would alias) -- and the entries (noise, BF16 words,
    // energy and remainder) are made from the group's region after the chunk
    // buffer is back with the MMA warp and the other group.
    const int grp = warp >= 6 ? 1 : 0;
    const int qw = warp & 3;
    int healthy = 1;
    int gc = 0, t = 0;
    for (int item = blockIdx.x; item < items && healthy; item += gridDim.x, ++t) {
      TcItem I;
      tc_item(chs, C, item, bn, I);
      const TcChan* ch = I.ch;
      const int chunk = ch->chunk_kt > 0 ? ch->chunk_kt : CHUNK_KT;
      const int nchunks = (I.nk + chunk - 1) / chunk;
      if ((t & 1) != grp) {                        // the other group's item
        gc += nchunks;
        continue;
      }
      const int row = I.m0 + qw * 32 + lane;
      const uint32_t lanes = (uint32_t)(qw * 32) << 16;
      const uint32_t fin = tmem + lanes + (uint32_t)((2 + grp) * bn);
      const int ncols = ch->ncols, nw = ch->nw, r0 = ch->r0;
      const int64_t ldy = ch->ldy, ldw = ch->ldw;
      const uint32_t key = ch->eta_key;
      const float amp_s = ch->eta_amp3 * 5.9604644775390625e-8f;     // x 2^-24: exact
      const float hinv2 = ch->hinv * ch->hinv;                         // >= 2^-120: normal
      float* Y = ch->Y;
      __nv_bfloat16* W0 = ch->W[0];
      __nv_bfloat16* W1 = ch->W[1];
      __nv_bfloat16* W2 = ch->W[2];
      const bool live = row < ch->m;
      const uint32_t hrow = lowbias32((uint32_t)row * 0x9E3779B1u + key);
      float s2 = 0.0f, r2 = 0.0f;
      for (int c = 0; c < nchunks; ++c, ++gc) {
        const int b = gc & 1;
        int ok = 1;
        if (lane == 0) {
          const long long t0 = clock64();
          // the other group holds the chunks before this one: back off
          // between polls so the spin does not take issue slots from its
          // warps on the same schedulers
          while (*(volatile int*)consumed < 4 * gc) {
            if (clock64() - t0 > (1ll << 32)) { ok = 0; break; }
            __nanosleep(128);
          }
          if (ok) ok = mbar_wait(&acc_full[b], (uint32_t)(gc >> 1) & 1u) ? 1 : 0;
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          if (lane == 0) set_err(err, DERR_TIMEOUT_EPI);
          healthy = 0;
          break;
        }
        tc_fence_after();
        const uint32_t ta = tmem + lanes + (uint32_t)(b * bn);
        // 32 columns per round trip (bn is a multiple of 32 here: gbn <= 128
        // is rounded to 16, and a 16-column tail takes the narrow form)
#pragma unroll 1
        for (int g = 0; g < bn; g += 32) {
          if (g + 32 <= bn) {
            uint32_t r[32], f[32];
            tmem_ld32_nw(ta + (uint32_t)g, r);
            if (c > 0) tmem_ld32_nw(fin + (uint32_t)g, f);
            tmem_wait_ld();
            if (c > 0) {
#pragma unroll
              for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) + __uint_as_float(f[j]));
            }
            tmem_st32(fin + (uint32_t)g, r);
          } else {
            uint32_t r[16], f[16];
            tmem_ld16_nw(ta + (uint32_t)g, r);
            if (c > 0) tmem_ld16_nw(fin + (uint32_t)g, f);
            tmem_wait_ld();
            if (c > 0) {
#pragma unroll
              for (int j = 0; j < 16; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) + __uint_as_float(f[j]));
            }
            tmem_st16(fin + (uint32_t)g, r);
          }
        }
        tmem_wait_st();
        tc_fence_before();
        mbar_arrive(&acc_empty[b]);
        __syncwarp();
        if (lane == 0) {
          __threadfence_block();
          atomicAdd(consumed, 1);
        }
      }
      if (healthy) {
#pragma unroll 1
        for (int g = 0; g < bn; g += 16) {
          const int col0 = I.n0 + g;
          if (col0 >= ncols) break;
          uint32_t r[16];
          tmem_ld16_nw(fin + (uint32_t)g, r);
          tmem_wait_ld();
          if (Y) {
            rule_group<0, true>(r, row, live, col0, ncols, r0, hrow, key, amp_s, hinv2, W0, W1, W2, ldw, Y, ldy, s2, r2, lane);
          } else if (nw == 2) {
            rule_group<2, false>(r, row, live, col0, ncols, r0, hrow, key, amp_s, hinv2, W0, W1, W2, ldw, Y, ldy, s2, r2, lane);
          } else if (nw == 3) {
            rule_group<3, false>(r, row, live, col0, ncols, r0, hrow, key, amp_s, hinv2, W0, W1, W2, ldw, Y, ldy, s2, r2, lane);
          } else {
            rule_group<1, false>(r, row, live, col0, ncols, r0, hrow, key, amp_s, hinv2, W0, W1, W2, ldw, Y, ldy, s2, r2, lane);
          }
        }
      }
      if (healthy) healthy = (*(volatile int*)err == 0);
      healthy = __shfl_sync(0xffffffffu, healthy, 0);
      if (!healthy) break;
      if (ch->part) {
        double ds = (double)s2, dr = (double)r2;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          ds += __shfl_xor_sync(0xffffffffu, ds, o);
          dr += __shfl_xor_sync(0xffffffffu, dr, o);
        }
        if (lane == 0) {
          double* pp = ch->part + ((int64_t)I.local * 4 + qw) * 2;
          pp[0] = ds;
          pp[1] = dr;
        }
      }
    }
  } else {
    // ---------------- epilogue warps 0-3: TMEM lanes 32w..32w+31 = rows of the tile
    int healthy = 1;
    int gc = 0;
    for (int item = blockIdx.x; item < items && healthy; item += gridDim.x) {
      TcItem I;
      tc_item(chs, C, item, bn, I);
      const TcChan* ch = I.ch;
      const int chunk = ch->chunk_kt > 0 ? ch->chunk_kt : CHUNK_KT;
      const int nchunks = (I.nk + chunk - 1) / chunk;
      float acc[BNM];
      for (int c = 0; c < nchunks; ++c, ++gc) {
        const int b = gc & 1;
        int ok = 0;
        if (lane == 0) ok = mbar_wait(&acc_full[b], (uint32_t)(gc >> 1) & 1u) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          if (lane == 0) set_err(err, DERR_TIMEOUT_EPI);
          healthy = 0;
          break;
        }
        tc_fence_after();
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * bn);
        // 32 columns per wait (two 16-column loads in flight)
#pragma unroll
        for (int g32 = 0; g32 < (BNM + 31) / 32; ++g32) {
          if (g32 * 32 < bn) {
            uint32_t r[32];
            tmem_ld16_nw(ta + (uint32_t)(g32 * 32), r);
            const bool two = g32 * 32 + 16 < bn && g32 * 32 + 16 < BNM;
            if (two) tmem_ld16_nw(ta + (uint32_t)(g32 * 32 + 16), r + 16);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              if (g32 * 32 + j < BNM && (j < 16 || two)) {
                const float v = __uint_as_float(r[j]);
                acc[g32 * 32 + j] = c == 0 ? v : acc[g32 * 32 + j] + v;
              }
            }
          }
        }
        tc_fence_before();
        mbar_arrive(&acc_empty[b]);
      }
      if (nchunks == 0) {
#pragma unroll
        for (int j = 0; j < BNM; ++j) acc[j] = 0.0f;
      }
      if (healthy) healthy = (*(volatile int*)err == 0);
      healthy = __shfl_sync(0xffffffffu, healthy, 0);
      if (!healthy) break;
      const int row = I.m0 + warp * 32 + lane;
      const int n0 = I.n0;
      if (row < ch->m) {
        float* Y = ch->Y;
        const int64_t ldy = ch->ldy;
        const int ncols = ch->ncols;
        const int atomic = ch->atomic;
#pragma unroll
        for (int j = 0; j < BNM; ++j) {
          const int col = n0 + j;
          if (j < bn && col < ncols) {
            float* dst = Y + row + (int64_t)col * ldy;
            if (atomic) atomicAdd(dst, acc[j]);
            else *dst = acc[j];
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, ncols_alloc);
}

// ------------------------------------------------------------------ host
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static int get_encode() {
  if (g_encode) return 0;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
          cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return -1;
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  return 0;
}

static int encode2d(CUtensorMap* m, const void* ptr, int64_t inner, int64_t outer, int64_t ld_elems,
                    int box_outer, int f16) {
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)(ld_elems * 2)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_outer};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = g_encode(m, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                              const_cast<void*>(ptr), dims, strides,
                              box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)r;
}

int tc_encode(TcChan* h, const void* const* A, int sa, int64_t lda, const void* const* X, int sx, int64_t ldx,
              int m, int n, int ncols, int bn, int f16) {
  if (get_encode()) return -1;
  for (int a = 0; a < sa; ++a)
    if (int e = encode2d(&h->tmA[a], A[a], n, m, lda, BM, f16)) return e;
  for (int x = 0; x < sx; ++x)
    if (int e = encode2d(&h->tmX[x], X[x], n, ncols, ldx, bn, f16)) return e;
  return 0;
}

template <int SA, int SX, bool RULE, int BNM = BN_NARROW>
static int launch_t(const TcChan* d_ch, int C, int items, int bn, int* d_err, cudaStream_t st, int max_stages) {
  int stages = tc_stages(SA, SX, bn);
  if (max_stages >= 2 && max_stages < stages) stages = max_stages;
  const int smem = stages * tc_stage_bytes(SA, SX, bn) + 1024 + 256;
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<SA, SX, RULE, BNM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return (int)e;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      nsm < 1)
    nsm = 148;
  const int grid = items < nsm ? items : nsm;                  // persistent: one CTA per SM
  k_tc_gemm<SA, SX, RULE, BNM><<<grid, RULE ? NTHREADS_RULE : NTHREADS, smem, st>>>(d_ch, C, items, bn, stages, d_err);
  note_launch();
  return (int)cudaGetLastError();
}

int tc_launch(const TcChan* d_ch, int C, int items, int sa, int sx, int bn, int* d_err, cudaStream_t st,
              bool rule, int max_stages) {
  if (items <= 0) return 0;
  if (bn < 16 || bn > BN_MAX || (bn % 16) != 0) return (int)cudaErrorInvalidValue;
  if (rule) {
    if (sa == 2 && sx == 2 && bn <= 128) return launch_t<2, 2, true>(d_ch, C, items, bn, d_err, st, max_stages);
    return (int)cudaErrorInvalidValue;
  }
  if (bn > BN_NARROW) {
    if (sa == 2 && sx == 2) return launch_t<2, 2, false, BN_MAX>(d_ch, C, items, bn, d_err, st, max_stages);
    if (sa == 3 && sx == 3) return launch_t<3, 3, false, BN_MAX>(d_ch, C, items, bn, d_err, st, max_stages);
    return (int)cudaErrorInvalidValue;
  }
  if (sa == 1 && sx == 1) return launch_t<1, 1, false>(d_ch, C, items, bn, d_err, st, max_stages);
  if (sa == 2 && sx == 1) return launch_t<2, 1, false>(d_ch, C, items, bn, d_err, st, max_stages);
  if (sa == 2 && sx == 2) return launch_t<2, 2, false>(d_ch, C, items, bn, d_err, st, max_stages);
  if (sa == 3 && sx == 1) return launch_t<3, 1, false>(d_ch, C, items, bn, d_err, st, max_stages);
  if (sa == 3 && sx == 3) return launch_t<3, 3, false>(d_ch, C, items, bn, d_err, st, max_stages);
  return (int)cudaErrorInvalidValue;
}

}  // namespace rsvd
