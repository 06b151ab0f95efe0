// Tensor-core passes over V for the mixed path: Y = V X on sm_103a.  The
// same kernel also generates the entries of a tile rule (TC_RULE): with H the
// n x M matrix of sqrt(w_m) g_m(x_j) in BF16 words, a panel of rule rows is
// H H_panel^T, to which the epilogue adds the hash noise before splitting the
// entries into the words the next pass reads.
//
// This is the contraction of Fig. 1 step 1 (Z = V P) and of the projection
// (Y^T = V Q, V symmetric) when V is held as a sum of BF16 words,
// V ~ V_0 + V_1 (+ V_2), and X likewise: Y = sum over word pairs (a, b) with
// a + b < max(SA, SX) of V_a X_b, accumulated in FP32.  Two words carry ~16
// significant bits of each FP64 entry, three ~24.
//
// Structure (one 128-row tile of Y per CTA, all of its columns):
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

#include "tc_gemm.h"

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

// ------------------------------------------------------------- PTX helpers
RSVD_DEV uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

RSVD_DEV void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

RSVD_DEV void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes) : "memory");
}

RSVD_DEV void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

RSVD_DEV bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: ~2^32 clocks (about two seconds) before giving up.
RSVD_DEV bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > (1ll << 32)) return false;
  }
}

RSVD_DEV void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_addr(dst)),
      "l"((uint64_t)map), "r"(smem_addr(bar)), "r"(x), "r"(y)
      : "memory");
}

RSVD_DEV void tmap_acquire(const CUtensorMap* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)map) : "memory");
}

RSVD_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
RSVD_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

RSVD_DEV void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
               "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

RSVD_DEV void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// core groups 1024 bytes apart (stride byte offset), descriptor version 1.
RSVD_DEV uint64_t sdesc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// N = bn, M = 128.
RSVD_DEV uint32_t idesc_bf16(int bn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

RSVD_DEV void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

RSVD_DEV void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

RSVD_DEV void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

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
static constexpr int BN_MAX = 160;            // register accumulator width
static constexpr int NTHREADS = 192;          // warps 0-3 epilogue, 4 producer, 5 MMA

template <int SA, int SX>
__global__ void __launch_bounds__(NTHREADS, 1)
k_tc_gemm(const TcChan* __restrict__ chs, int C, int bn, int stages, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int SB = SA * A_TILE_BYTES + SX * bn * BK * 2;
  uint64_t* full = (uint64_t*)(base + (size_t)stages * SB);
  uint64_t* empty = full + stages;
  uint64_t* acc_full = empty + stages;     // [2] MMA -> epilogue
  uint64_t* acc_empty = acc_full + 2;      // [2] epilogue -> MMA (128 arrivals)
  uint32_t* tmem_slot = (uint32_t*)(acc_empty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // work item -> channel, split, tile
  const int item = blockIdx.x;
  int lo = 0, hi = C - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (chs[mid].item0 <= item) lo = mid; else hi = mid - 1;
  }
  const TcChan* ch = chs + lo;
  int local = item - ch->item0;
  const int per_split = ch->mt * ch->nt;
  const int split = local / per_split;
  local -= split * per_split;
  const int mi = local / ch->nt, ni = local % ch->nt;
  const int m0 = mi * BM, n0 = ni * bn;
  const int kt_total = (ch->n + BK - 1) / BK;
  const int kb = split * ch->kt_per_split;
  const int nk = min(kt_total, kb + ch->kt_per_split) - kb;
  const int chunk = ch->chunk_kt > 0 ? ch->chunk_kt : CHUNK_KT;
  const int nchunks = (nk + chunk - 1) / chunk;
  uint32_t ncols_alloc = 32;
  while ((int)ncols_alloc < 2 * bn) ncols_alloc <<= 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], 128); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, ncols_alloc);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (nk > 0) {
    if (warp == 4) {
      if (lane == 0) {
        // ---------------- TMA producer
        for (int a = 0; a < SA; ++a) tmap_acquire(&ch->tmA[a]);
        for (int x = 0; x < SX; ++x) tmap_acquire(&ch->tmX[x]);
        int issued = 0;
        for (int it = 0; it < nk; ++it) {
          const int s = it % stages;
          const uint32_t ph = (uint32_t)(it / stages) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u)) { set_err(err, DERR_TIMEOUT_TMA); break; }
          mbar_arrive_expect_tx(&full[s], (uint32_t)SB);
          unsigned char* st = base + (size_t)s * SB;
          const int kx = (kb + it) * BK;
          for (int a = 0; a < SA; ++a) tma_load_2d(st + a * A_TILE_BYTES, &ch->tmA[a], &full[s], kx, m0);
          for (int x = 0; x < SX; ++x)
            tma_load_2d(st + SA * A_TILE_BYTES + x * bn * BK * 2, &ch->tmX[x], &full[s], kx, n0);
          issued = it + 1;
        }
        // drain: the last copy issued into each stage has landed
        for (int s = 0; s < stages && s < issued; ++s) {
          const int last = s + ((issued - 1 - s) / stages) * stages;
          if (!mbar_wait(&full[s], (uint32_t)(last / stages) & 1u)) set_err(err, DERR_TIMEOUT_TMA);
        }
      }
      __syncwarp();
    } else if (warp == 5) {
      if (lane == 0) {
        // ---------------- MMA issuer
        const uint32_t idesc = idesc_bf16(bn);
        bool ok = true;
        int it = 0;
        for (int c = 0; c < nchunks && ok; ++c) {
          const int b = c & 1;
          if (c >= 2 && !mbar_wait(&acc_empty[b], (uint32_t)((c >> 1) - 1) & 1u)) {
            set_err(err, DERR_TIMEOUT_MMA);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dt = tmem + (uint32_t)(b * bn);
          const int itend = min(nk, it + chunk);
          for (; it < itend; ++it) {
            const int s = it % stages;
            const uint32_t ph = (uint32_t)(it / stages) & 1u;
            if (!mbar_wait(&full[s], ph)) { set_err(err, DERR_TIMEOUT_MMA); ok = false; break; }
            tc_fence_after();
            const uint32_t sa0 = smem_addr(base + (size_t)s * SB);
            const uint32_t sx0 = sa0 + SA * A_TILE_BYTES;
            bool zero = (it == c * chunk);          // first MMA of the chunk overwrites
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
      __syncwarp();
    } else {
      // ---------------- epilogue warps 0-3: TMEM lanes 32w..32w+31 = rows of the tile
      float acc[BN_MAX];
#pragma unroll
      for (int j = 0; j < BN_MAX; ++j) acc[j] = 0.0f;
      int healthy = 1;
      for (int c = 0; c < nchunks; ++c) {
        const int b = c & 1;
        int ok = 0;
        if (lane == 0) ok = mbar_wait(&acc_full[b], (uint32_t)(c >> 1) & 1u) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          if (lane == 0) set_err(err, DERR_TIMEOUT_EPI);
          healthy = 0;
          break;
        }
        tc_fence_after();
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * bn);
#pragma unroll
        for (int g = 0; g < BN_MAX / 16; ++g) {
          if (g * 16 < bn) {
            uint32_t r[16];
            tmem_ld16(ta + (uint32_t)(g * 16), r);
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[g * 16 + j] += __uint_as_float(r[j]);
          }
        }
        tc_fence_before();
        mbar_arrive(&acc_empty[b]);
      }
      if (healthy) healthy = (*(volatile int*)err == 0);
      healthy = __shfl_sync(0xffffffffu, healthy, 0);
      if (healthy) {
        const int row = m0 + warp * 32 + lane;
        if (ch->mode == TC_RULE) {
          // generated tile-rule entries: add the symmetric noise, split into
          // BF16 words, and keep the energy and the words' remainder
          float s2 = 0.0f, r2 = 0.0f;
          if (row < ch->m) {
            float* Y = ch->Y;
            const int64_t ldy = ch->ldy, ldw = ch->ldw;
            const int ncols = ch->ncols, nw = ch->nw, r0 = ch->r0;
            const uint32_t key = ch->eta_key;
            const float amp3 = ch->eta_amp3;
            __nv_bfloat16* W0 = ch->W[0];
            __nv_bfloat16* W1 = ch->W[1];
            __nv_bfloat16* W2 = ch->W[2];
#pragma unroll
            for (int j = 0; j < BN_MAX; ++j) {
              const int col = n0 + j;
              if (j < bn && col < ncols) {
                const float v = acc[j] + rule_eta(key, amp3, r0 + col, row);
                s2 = fmaf(v, v, s2);
                if (nw > 0) {
                  const int64_t o = row + (int64_t)col * ldw;
                  __nv_bfloat16 q = __float2bfloat16_rn(v);
                  W0[o] = q;
                  float rem = v - __bfloat162float(q);      // exact
                  if (nw > 1) {
                    q = __float2bfloat16_rn(rem);
                    W1[o] = q;
                    rem -= __bfloat162float(q);
                    if (nw > 2) {
                      q = __float2bfloat16_rn(rem);
                      W2[o] = q;
                      rem -= __bfloat162float(q);
                    }
                  }
                  r2 = fmaf(rem, rem, r2);
                }
                if (Y) Y[row + (int64_t)col * ldy] = v;
              }
            }
          }
          if (ch->part) {
            double ds = (double)s2, dr = (double)r2;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              ds += __shfl_xor_sync(0xffffffffu, ds, o);
              dr += __shfl_xor_sync(0xffffffffu, dr, o);
            }
            if (lane == 0) {
              double* pp = ch->part + ((int64_t)(item - ch->item0) * 4 + warp) * 2;
              pp[0] = ds;
              pp[1] = dr;
            }
          }
        } else if (row < ch->m) {
          float* Y = ch->Y;
          const int64_t ldy = ch->ldy;
          const int ncols = ch->ncols;
          const int atomic = ch->atomic;
#pragma unroll
          for (int j = 0; j < BN_MAX; ++j) {
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
                    int box_outer) {
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)(ld_elems * 2)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_outer};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides,
                              box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)r;
}

int tc_encode(TcChan* h, const __nv_bfloat16* const* A, int sa, int64_t lda, const __nv_bfloat16* const* X,
              int sx, int64_t ldx, int m, int n, int ncols, int bn) {
  if (get_encode()) return -1;
  for (int a = 0; a < sa; ++a)
    if (int e = encode2d(&h->tmA[a], A[a], n, m, lda, BM)) return e;
  for (int x = 0; x < sx; ++x)
    if (int e = encode2d(&h->tmX[x], X[x], n, ncols, ldx, bn)) return e;
  return 0;
}

template <int SA, int SX>
static int launch_t(const TcChan* d_ch, int C, int items, int bn, int* d_err, cudaStream_t st) {
  const int stages = tc_stages(SA, SX, bn);
  const int smem = stages * tc_stage_bytes(SA, SX, bn) + 1024 + 256;
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<SA, SX>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return (int)e;
  k_tc_gemm<SA, SX><<<items, NTHREADS, smem, st>>>(d_ch, C, bn, stages, d_err);
  note_launch();
  return (int)cudaGetLastError();
}

int tc_launch(const TcChan* d_ch, int C, int items, int sa, int sx, int bn, int* d_err, cudaStream_t st) {
  if (items <= 0) return 0;
  if (bn < 16 || bn > BN_MAX || (bn % 16) != 0) return (int)cudaErrorInvalidValue;
  if (sa == 1 && sx == 1) return launch_t<1, 1>(d_ch, C, items, bn, d_err, st);
  if (sa == 2 && sx == 1) return launch_t<2, 1>(d_ch, C, items, bn, d_err, st);
  if (sa == 2 && sx == 2) return launch_t<2, 2>(d_ch, C, items, bn, d_err, st);
  if (sa == 3 && sx == 1) return launch_t<3, 1>(d_ch, C, items, bn, d_err, st);
  if (sa == 3 && sx == 3) return launch_t<3, 3>(d_ch, C, items, bn, d_err, st);
  return (int)cudaErrorInvalidValue;
}

}  // namespace rsvd
