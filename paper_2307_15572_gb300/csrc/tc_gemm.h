// tcgen05 / TMEM / TMA GEMM used for the passes over V on the mixed path.
#pragma once

#include <cuda.h>

#include "kernels.h"

namespace rsvd {

// Per-channel operand maps and output of one grouped launch.  Must be 64-byte
// aligned (CUtensorMap is), lives in device memory.
enum TcMode { TC_STORE = 0, TC_RULE = 1 };

struct alignas(64) TcChan {
  CUtensorMap tmA[3];   // A operand words: dims {n (k), m (rows)}, box {64, 128}, 128B swizzle
  CUtensorMap tmX[3];   // X words: dims {n (k), ncols}, box {64, BN}, 128B swizzle
  float* Y;             // output, column-major m x ncols, leading dim ldy (TC_RULE: optional copy)
  int64_t ldy;
  int n;                // k extent
  int m;                // rows of the A operand and of Y
  int ncols;            // output columns
  int mt, nt, ks;       // tiles along m (128), n (BN), k splits
  int kt_per_split;     // 64-wide k steps per split
  int item0;            // first work item of this channel
  int atomic;           // 1: accumulate with red.add (k split), 0: store
  int mode;             // TcMode
  int chunk_kt;         // 64-wide k steps per TMEM accumulation chunk (0: the default, 8)
  // TC_RULE (generated entries of a tile rule; ks must be 1): output element
  // (row, col) is the matrix entry (r0 + col, row); v = acc + eta is split
  // into nw BF16 words W[w][row + col * ldw], and each (work item, epilogue
  // warp) writes {sum v^2, sum (v - words)^2} to part (if non-null).
  __nv_bfloat16* W[3];
  int64_t ldw;
  int nw;
  int r0;
  uint32_t eta_key;
  float eta_amp3;       // sqrt(3) * eta amplitude
  float hinv;           // 1 / hscale of the FP16 factor words: entry = acc * hinv * hinv
  double* part;
  // FP64-input passes (k_tc_f64): tmA[0] maps the FP64 V (box 16 x 128);
  // the first pass writes ||V||^2 and the word remainder energy per 8-row
  // block and flags Inf/NaN
  double* fro_part;
  double* wres_part;
  int* flags;
};

// FP64-input passes: maps of one channel (V FP64 with leading dim ldv, even,
// 16-byte aligned; X words as in tc_encode); 0 on success, -2 for a V the
// TMA cannot address.  Stages and launch (sx = 1 or 2 X words, bn <=
// TC_BN_NARROW, one column tile per item, no k split); the launch returns a
// cudaError_t value.
int f64pass_encode(TcChan* h, const double* V, int64_t ldv, int n, const void* const* X, int sx, int64_t ldx,
                   int ncols, int bn);
int f64pass_stages(int sx, int bn);
int f64pass_launch(const TcChan* d_ch, int C, int items, int sx, int bn, bool stats, int* d_err, cudaStream_t st);

// Encode the maps of one channel (host).  Returns 0 on success.  f16: the
// words are FP16 (the tile-rule factor), else BF16.
int tc_encode(TcChan* h, const void* const* A, int sa, int64_t lda_elems, const void* const* X, int sx,
              int64_t ldx_elems, int m, int n, int ncols, int bn, int f16 = 0);

// Widest output-column tile of one work item (the epilogue's register
// accumulator): up to TC_BN_NARROW for every word combination, up to
// TC_BN_MAX for the two-word passes (2, 2) and (3, 3).
constexpr int TC_BN_NARROW = 160;
constexpr int TC_BN_MAX = 176;

// Shared memory bytes per stage and stage count for a configuration.
int tc_stage_bytes(int sa, int sx, int bn);
int tc_stages(int sa, int sx, int bn);

// Launch over `items` work items (sum over channels of mt*nt*ks).
// Returns a cudaError_t value.
// rule: the tile-rule generation instantiation (<2, 2> FP16 words, TC_RULE
// channels only).
// max_stages: cap on the shared-memory pipeline depth (0: as many stages as
// shared memory holds, at most 8; values below 2 mean no cap).
int tc_launch(const TcChan* d_ch, int C, int items, int sa, int sx, int bn, int* d_err,
              cudaStream_t st, bool rule = false, int max_stages = 0);

}  // namespace rsvd
