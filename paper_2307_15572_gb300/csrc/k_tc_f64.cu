// Tensor-core passes that read the stored FP64 V directly: Y = V X with V
// split into two BF16 words on chip, an alternative for the mixed path
// without power iterations.  There the two passes over V (Fig. 1 step 1,
// Z = V P, and the projection Y^T = V Q) each read V once in FP64 (8 bytes
// per entry, 16 in all) instead of converting V into stored words first
// (8 read + 4 written) and reading the words twice (4 + 4): 20 bytes per
// entry.  Each pass must then round V to FP32 (integer pipe) again, at the
// rate HBM delivers it; on this part that rounding, with only two 64 KiB
// stages beside the MMA operands, holds the pass near 4 TB/s, so the word
// passes stay the default (the caller opts in).
//
// Structure (persistent CTAs, one per SM, work items = 128-row tiles of Y
// with all their columns; no k split):
//   * warp 4, one thread: TMA producer.  Per 64-wide k step: four FP64 boxes
//     of V (128 rows x 16 columns, 128B swizzle, 64 KiB) and the X word
//     tiles (BN x 64);
//   * warps 6-21: converters, four threads per row (one per box).  Each
//     reads its 16 FP64 values; after a named barrier over the converters
//     (every row read) it rounds them to FP32 (integer pipe),
//     splits them into BF16 words hi + lo and writes the words in place: the
//     word tiles are the 128B-swizzled K-major A operands at the first two
//     boxes' addresses, and a row's 128-byte slot in box 0 (box 1) holds
//     exactly that row's k range of word 0 (word 1).  The first pass also sums ||V||^2 and the
//     energy the two words leave out per 8-row block, and flags Inf/NaN;
//   * warp 5, one thread: MMA issuer (as in the word passes): tcgen05.mma
//     over the word pairs (a, x) with a + x < max(2, SX), chunked TMEM
//     accumulation;
//   * warps 0-3: epilogue, chunk sums added into a third TMEM region, the
//     last one stored to Y.
// Every wait is bounded; on expiry the thread records an error code and the
// CTA drains its own copies and frees TMEM before returning.
#include <cudaTypedefs.h>

#include "tc_gemm.h"
#include "tc_ptx.cuh"

namespace rsvd {

namespace {
constexpr int FB_BM = 128;
constexpr int FB_BK = 64;
constexpr int FB_BOX = 128 * 16 * 8;                 // one FP64 box: 128 rows x 16 columns
constexpr int FB_F64_BYTES = 4 * FB_BOX;             // 64 KiB per k step
constexpr int FB_SMEM_BUDGET = 220 * 1024;
constexpr int FB_THREADS = 704;                      // warps 0-3 epilogue, 4 producer, 5 MMA, 6-21 converters
constexpr int FB_CHUNK_KT = 8;
}  // namespace

int f64pass_stage_bytes(int sx, int bn) { return FB_F64_BYTES + sx * bn * FB_BK * 2; }

int f64pass_stages(int sx, int bn) {
  int st = (FB_SMEM_BUDGET - 1024 - 1024) / f64pass_stage_bytes(sx, bn);
  return st > 4 ? 4 : st;
}

RSVD_DEV void fb_item(const TcChan* __restrict__ chs, int C, int item, int bn, int& c, int& m0, int& n0, int& nk) {
  int lo = 0, hi = C - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (chs[mid].item0 <= item) lo = mid; else hi = mid - 1;
  }
  c = lo;
  int local = item - chs[lo].item0;
  const int nt = chs[lo].nt;
  m0 = (local / nt) * FB_BM;
  n0 = (local % nt) * bn;
  nk = (chs[lo].n + FB_BK - 1) / FB_BK;
}

// Named barrier 1 over the 512 converter threads with an AND of `ok`.
RSVD_DEV bool conv_bar_all(bool ok) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "barrier.red.and.pred q, 1, 512, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"(ok ? 1u : 0u)
      : "memory");
  return r != 0;
}

template <int SX, bool STATS>
__global__ void __launch_bounds__(FB_THREADS, 1)
k_tc_f64(const TcChan* __restrict__ chs, int C, int items, int bn, int stages, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int SB = FB_F64_BYTES + SX * bn * FB_BK * 2;
  uint64_t* full = (uint64_t*)(base + (size_t)stages * SB);
  uint64_t* conv = full + stages;
  uint64_t* empty = conv + stages;
  uint64_t* acc_full = empty + stages;     // [2] MMA -> epilogue
  uint64_t* acc_empty = acc_full + 2;      // [2] epilogue -> MMA (128 arrivals)
  uint32_t* tmem_slot = (uint32_t*)(acc_empty + 2);
  float* xsum = (float*)(tmem_slot + 4);   // [3][2][16] converter quarters 1-3 -> quarter 0 block sums

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t ncols_alloc = 32;                          // two chunk buffers and the running sum
  while ((int)ncols_alloc < 3 * bn) ncols_alloc <<= 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) { mbar_init(&full[s], 1); mbar_init(&conv[s], 512); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], 128); }
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
      int g = 0;
      bool ok = true;
      int last = -1;
      for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
        int c, m0, n0, nk;
        fb_item(chs, C, item, bn, c, m0, n0, nk);
        const TcChan* ch = chs + c;
        if (c != last) {
          tmap_acquire(&ch->tmA[0]);
          for (int x = 0; x < SX; ++x) tmap_acquire(&ch->tmX[x]);
          last = c;
        }
        for (int it = 0; it < nk; ++it, ++g) {
          const int s = g % stages;
          const uint32_t ph = (uint32_t)(g / stages) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u)) { set_err(err, DERR_TIMEOUT_TMA); ok = false; break; }
          mbar_arrive_expect_tx(&full[s], (uint32_t)SB);
          unsigned char* st = base + (size_t)s * SB;
          const int kx = it * FB_BK;
#pragma unroll
          for (int b = 0; b < 4; ++b) tma_load_2d(st + b * FB_BOX, &ch->tmA[0], &full[s], kx + 16 * b, m0);
          for (int x = 0; x < SX; ++x)
            tma_load_2d(st + FB_F64_BYTES + x * bn * FB_BK * 2, &ch->tmX[x], &full[s], kx, n0);
        }
      }
      for (int s = 0; s < stages && s < g; ++s) {
        const int lastg = s + ((g - 1 - s) / stages) * stages;
        if (!mbar_wait(&full[s], (uint32_t)(lastg / stages) & 1u)) set_err(err, DERR_TIMEOUT_TMA);
      }
    }
    __syncwarp();
  } else if (warp >= 6) {
    // ---------------- converters: thread = (row r of the tile, quarter h of
    // the k step: one box); the four threads of a row read their boxes, meet
    // at a named barrier, then write the row's words in place
    const int ct = threadIdx.x - 192;
    const int r = ct & 127, half = ct >> 7;            // `half`: the quarter (box) 0..3
    const int sw = r & 7;
    int g = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
      int c, m0, n0, nk;
      fb_item(chs, C, item, bn, c, m0, n0, nk);
      const TcChan* ch = chs + c;
      float s2 = 0.0f, w2 = 0.0f;
      bool bad = false;
      for (int it = 0; it < nk; ++it, ++g) {
        const int s = g % stages;
        const uint32_t ph = (uint32_t)(g / stages) & 1u;
        // every lane observes the phase (acquiring the TMA's writes)
        const bool okw = mbar_wait(&full[s], ph);
        const uint32_t sb = smem_addr(base + (size_t)s * SB) + (uint32_t)(r * 128);
        // the row's 16 values of box h (two FP64 per 16-byte chunk, chunk q
        // of the row at position q ^ (r & 7))
        uint32_t raw[8][4];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const uint32_t a = sb + (uint32_t)(half * FB_BOX) + (uint32_t)((q ^ sw) << 4);
          asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                       : "=r"(raw[q][0]), "=r"(raw[q][1]), "=r"(raw[q][2]), "=r"(raw[q][3])
                       : "r"(a)
                       : "memory");
        }
        // all four boxes of every row are read before any word is written;
        // the same barrier tells every converter whether all waits
        // succeeded, so they stop together (no thread is left at a later
        // barrier)
        if (!conv_bar_all(okw)) {
          if (!okw) set_err(err, DERR_TIMEOUT_EPI);
          ok = false;
          break;
        }
        // FP64 -> FP32, round to nearest even, from the bit fields (integer
        // pipe, no branch); zero, subnormal, overflowing and non-finite values
        // are marked and redone by the conversion instruction in one
        // warp-uniform pass (rare)
        float fv[16];
        uint32_t special = 0;
#pragma unroll
        for (int v = 0; v < 16; ++v) {
          const uint32_t* rr = raw[v >> 1];
          const uint32_t lo = rr[2 * (v & 1)], hi = rr[2 * (v & 1) + 1];
          const uint32_t e = (hi >> 20) & 0x7FFu;
          const int fe = (int)e - 1023 + 127;
          const uint32_t keep = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
          const uint32_t rest = lo & 0x1FFFFFFFu;
          const uint32_t up = (uint32_t)(rest > 0x10000000u) | ((uint32_t)(rest == 0x10000000u) & keep);
          fv[v] = __uint_as_float((hi & 0x80000000u) | (((uint32_t)fe << 23) + keep + (up & 1u)));
          special |= (uint32_t)((uint32_t)(fe - 1) >= 254u) << v;
          bad |= e == 0x7FFu;
        }
        if (__any_sync(0xffffffffu, special != 0)) {
#pragma unroll
          for (int v = 0; v < 16; ++v) {
            if (special & (1u << v)) {
              const uint32_t* rr = raw[v >> 1];
              fv[v] = __double2float_rn(__hiloint2double((int)rr[2 * (v & 1) + 1], (int)rr[2 * (v & 1)]));
            }
          }
        }
        // word chunks 2 h, 2 h + 1 (8 values each)
#pragma unroll
        for (int wq = 0; wq < 2; ++wq) {
          uint32_t w0[4], w1[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const int v = 8 * wq + 2 * p;
            float2 f;
            f.x = fv[v];
            f.y = fv[v + 1];
            if (STATS) {
              s2 = fmaf(f.x, f.x, s2);
              s2 = fmaf(f.y, f.y, s2);
            }
            const __nv_bfloat162 q0 = __float22bfloat162_rn(f);
            const float2 g0 = __bfloat1622float2(q0);
            float2 e;
            e.x = f.x - g0.x;                      // exact
            e.y = f.y - g0.y;
            const __nv_bfloat162 q1 = __float22bfloat162_rn(e);
            if (STATS) {
              const float2 g1 = __bfloat1622float2(q1);
              const float dx = e.x - g1.x, dy = e.y - g1.y;
              w2 = fmaf(dx, dx, w2);
              w2 = fmaf(dy, dy, w2);
            }
            w0[p] = *reinterpret_cast<const uint32_t*>(&q0);
            w1[p] = *reinterpret_cast<const uint32_t*>(&q1);
          }
          const uint32_t pos = (uint32_t)(((2 * half + wq) ^ sw) << 4);
          st_shared_v4(sb + pos, w0[0], w0[1], w0[2], w0[3]);             // word 0 at box 0
          st_shared_v4(sb + FB_BOX + pos, w1[0], w1[1], w1[2], w1[3]);    // word 1 at box 1
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&conv[s]);
      }
      if (!ok) break;
      if (STATS) {
        // per 8-row block (8 consecutive lanes, four quarters): ||V||^2 and
        // the remainder energy; quarters 1-3 hand their sums to quarter 0
        // through shared memory
        float a = s2, b = w2;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (half > 0 && (lane & 7) == 0) {
          xsum[(half - 1) * 32 + (r >> 3)] = a;
          xsum[(half - 1) * 32 + 16 + (r >> 3)] = b;
        }
        asm volatile("bar.sync 1, 512;" ::: "memory");
        const int row = m0 + r;
        if (half == 0 && (lane & 7) == 0 && row < ch->n) {
          const int blk = r >> 3;
          // fixed order: quarter 0 + 1 + 2 + 3
          const float fa = ((a + xsum[blk]) + xsum[32 + blk]) + xsum[64 + blk];
          const float fb = ((b + xsum[16 + blk]) + xsum[48 + blk]) + xsum[80 + blk];
          ch->fro_part[row >> 3] = f32_to_f64(fa);
          if (ch->wres_part) ch->wres_part[row >> 3] = f32_to_f64(fb);
        }
        asm volatile("bar.sync 1, 512;" ::: "memory");
        if (bad) atomicOr(ch->flags, FLAG_NONFINITE);
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      // ---------------- MMA issuer
      const uint32_t idesc = idesc_bf16(bn);
      bool ok = true;
      int g = 0, gc = 0;
      for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
        int c, m0, n0, nk;
        fb_item(chs, C, item, bn, c, m0, n0, nk);
        const int nchunks = (nk + FB_CHUNK_KT - 1) / FB_CHUNK_KT;
        int it = 0;
        for (int cc = 0; cc < nchunks && ok; ++cc, ++gc) {
          const int b = gc & 1;
          if (gc >= 2 && !mbar_wait(&acc_empty[b], (uint32_t)((gc >> 1) - 1) & 1u)) {
            set_err(err, DERR_TIMEOUT_MMA);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dt = tmem + (uint32_t)(b * bn);
          const int itend = min(nk, it + FB_CHUNK_KT);
          bool zero = true;
          for (; it < itend; ++it, ++g) {
            const int s = g % stages;
            const uint32_t ph = (uint32_t)(g / stages) & 1u;
            if (!mbar_wait(&conv[s], ph)) { set_err(err, DERR_TIMEOUT_MMA); ok = false; break; }
            tc_fence_after();
            const uint32_t sa0 = smem_addr(base + (size_t)s * SB);
            const uint32_t sx0 = sa0 + FB_F64_BYTES;
            // small word products first, the leading pair (0, 0) last
#pragma unroll
            for (int pr = (SX > 2 ? SX : 2) - 1; pr >= 0; --pr) {
#pragma unroll
              for (int a = 0; a < 2; ++a) {
#pragma unroll
                for (int x = 0; x < SX; ++x) {
                  if (a + x != pr) continue;
#pragma unroll
                  for (int kk = 0; kk < FB_BK / 16; ++kk) {
                    const uint64_t ad = sdesc_sw128(sa0 + a * FB_BOX + kk * 32);
                    const uint64_t bd = sdesc_sw128(sx0 + x * bn * FB_BK * 2 + kk * 32);
                    mma_bf16(dt, ad, bd, idesc, zero ? 0u : 1u);
                    zero = false;
                  }
                }
              }
            }
            mma_commit(&empty[s]);
          }
          mma_commit(&acc_full[b]);
        }
      }
      if (gc > 0) {
        const int b = (gc - 1) & 1;
        if (!mbar_wait(&acc_full[b], (uint32_t)((gc - 1) >> 1) & 1u)) set_err(err, DERR_TIMEOUT_MMA);
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue warps 0-3: TMEM lanes 32w..32w+31 = rows of the
    // tile.  Chunk sums are added (round to nearest) into a third TMEM region
    // of bn columns, 16 columns per round trip; the last chunk's sum goes to Y.
    int healthy = 1;
    int gc = 0;
    const uint32_t lanes = (uint32_t)(warp * 32) << 16;
    const uint32_t fin = tmem + lanes + (uint32_t)(2 * bn);
    for (int item = blockIdx.x; item < items && healthy; item += gridDim.x) {
      int c, m0, n0, nk;
      fb_item(chs, C, item, bn, c, m0, n0, nk);
      const TcChan* ch = chs + c;
      const int nchunks = (nk + FB_CHUNK_KT - 1) / FB_CHUNK_KT;
      const int row = m0 + warp * 32 + lane;
      const bool live = row < ch->m;
      float* Y = ch->Y;
      const int64_t ldy = ch->ldy;
      const int ncols = ch->ncols;
      for (int cc = 0; cc < nchunks; ++cc, ++gc) {
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
        const uint32_t ta = tmem + lanes + (uint32_t)(b * bn);
        const bool last = cc == nchunks - 1;
#pragma unroll 1
        for (int g0 = 0; g0 < bn; g0 += 16) {           // bn is a multiple of 16
          uint32_t r[16], f[16];
          tmem_ld16_nw(ta + (uint32_t)g0, r);
          if (cc > 0) tmem_ld16_nw(fin + (uint32_t)g0, f);
          tmem_wait_ld();
          if (cc > 0) {
#pragma unroll
            for (int j = 0; j < 16; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) + __uint_as_float(f[j]));
          }
          if (!last) {
            tmem_st16(fin + (uint32_t)g0, r);
          } else if (live) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int col = n0 + g0 + j;
              if (col < ncols) Y[row + (int64_t)col * ldy] = __uint_as_float(r[j]);
            }
          }
        }
        if (!last) tmem_wait_st();
        tc_fence_before();
        mbar_arrive(&acc_empty[b]);
      }
      if (healthy && nchunks == 0 && live) {
        for (int j = 0; j < bn; ++j)
          if (n0 + j < ncols) Y[row + (int64_t)(n0 + j) * ldy] = 0.0f;
      }
      if (healthy) healthy = (*(volatile int*)err == 0);
      healthy = __shfl_sync(0xffffffffu, healthy, 0);
      if (!healthy) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, ncols_alloc);
}

// ------------------------------------------------------------------ host
static PFN_cuTensorMapEncodeTiled_v12000 g_encode64 = nullptr;

static int get_encode64() {
  if (g_encode64) return 0;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
          cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return -1;
  g_encode64 = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  return 0;
}

int f64pass_encode(TcChan* h, const double* V, int64_t ldv, int n, const void* const* X, int sx, int64_t ldx,
                   int ncols, int bn) {
  if (get_encode64()) return -1;
  if ((ldv & 1) || ((uintptr_t)V & 15)) return -2;          // TMA: 16-byte aligned base and row stride
  {
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)(ldv * 8)};
    cuuint32_t box[2] = {16, (cuuint32_t)FB_BM};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = g_encode64(&h->tmA[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(V), dims,
                                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return (int)r;
  }
  for (int x = 0; x < sx; ++x) {
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)ncols};
    cuuint64_t strides[1] = {(cuuint64_t)(ldx * 2)};
    cuuint32_t box[2] = {(cuuint32_t)FB_BK, (cuuint32_t)bn};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = g_encode64(&h->tmX[x], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(X[x]), dims,
                                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return (int)r;
  }
  return 0;
}

template <int SX, bool STATS>
static int f64_launch_t(const TcChan* d_ch, int C, int items, int bn, int* d_err, cudaStream_t st) {
  const int stages = f64pass_stages(SX, bn);
  if (stages < 2) return (int)cudaErrorInvalidValue;
  const int smem = stages * f64pass_stage_bytes(SX, bn) + 1024 + 1024;  // + barriers, TMEM slot, block sums
  auto kf = k_tc_f64<SX, STATS>;
  cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return (int)e;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      nsm < 1)
    nsm = 148;
  const int grid = items < nsm ? items : nsm;
  kf<<<grid, FB_THREADS, smem, st>>>(d_ch, C, items, bn, stages, d_err);
  note_launch();
  return (int)cudaGetLastError();
}

int f64pass_launch(const TcChan* d_ch, int C, int items, int sx, int bn, bool stats, int* d_err, cudaStream_t st) {
  if (items <= 0) return 0;
  if (bn < 16 || bn > TC_BN_NARROW || (bn % 16) != 0) return (int)cudaErrorInvalidValue;
  if (sx == 1 && stats) return f64_launch_t<1, true>(d_ch, C, items, bn, d_err, st);
  if (sx == 1) return f64_launch_t<1, false>(d_ch, C, items, bn, d_err, st);
  if (sx == 2) return f64_launch_t<2, false>(d_ch, C, items, bn, d_err, st);
  return (int)cudaErrorInvalidValue;
}

}  // namespace rsvd
