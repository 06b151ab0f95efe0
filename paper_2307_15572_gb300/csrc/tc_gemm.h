// tcgen05 / TMEM / TMA GEMM used for the passes over V on the mixed path.
#pragma once

#include <cuda.h>

#include "kernels.h"

namespace rsvd {

// Per-channel operand maps and output of one grouped launch.  Must be 64-byte
// aligned (CUtensorMap is), lives in device memory.
struct alignas(64) TcChan {
  CUtensorMap tmA[3];   // V slices: dims {n (k), n (m)}, box {64, 128}, 128B swizzle
  CUtensorMap tmX[3];   // X slices: dims {n (k), ncols (n)}, box {64, BN}, 128B swizzle
  float* Y;             // output, column-major n x ncols, leading dim ldy
  int64_t ldy;
  int n;                // rows of V (= k extent)
  int ncols;            // output columns
  int mt, nt, ks;       // tiles along m (128), n (BN), k splits
  int kt_per_split;     // 64-wide k steps per split
  int item0;            // first work item of this channel
  int atomic;           // 1: accumulate with red.add (k split), 0: store
};

// Encode the maps of one channel (host).  Returns 0 on success.
int tc_encode(TcChan* h, const __nv_bfloat16* const* A, int sa, int64_t lda_elems,
              const __nv_bfloat16* const* X, int sx, int64_t ldx_elems, int n, int ncols,
              int bn);

// Shared memory bytes per stage and stage count for a configuration.
int tc_stage_bytes(int sa, int sx, int bn);
int tc_stages(int sa, int sx, int bn);

// Launch over `items` work items (sum over channels of mt*nt*ks).
// Returns a cudaError_t value.
int tc_launch(const TcChan* d_ch, int C, int items, int sa, int sx, int bn, int* d_err,
              cudaStream_t st);

}  // namespace rsvd
