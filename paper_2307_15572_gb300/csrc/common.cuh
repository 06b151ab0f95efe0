// Shared device helpers and per-channel descriptors of the rSVD pipeline.
//
// Everything here is device-side arithmetic of the method or plumbing
// (bounded waits, batched tile lookup).  Nothing is shared with the CPU
// oracle.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/rsvd.h"

#define RSVD_DEV __device__ __forceinline__
#define RSVD_HD __host__ __device__ __forceinline__

namespace rsvd {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11, Sec. 3): ten rounds of
// two 32x32->64 multiplies with xor of the other counter words and the key;
// the key is bumped by the Weyl constants between rounds.  Counter layout
// (row i, column j, tag, 0), key (seed lo, seed hi).
// ---------------------------------------------------------------------------
struct Philox4 { uint32_t x, y, z, w; };

RSVD_DEV Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                               uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  return {c0, c1, c2, c3};
}

enum : uint32_t { TAG_OMEGA = 0, TAG_PROBE = 1, TAG_NOISE = 2, TAG_RESID = 3 };

// FP64 Box-Muller entry from two 53-bit uniforms (the all-FP64 path's form).
RSVD_DEV double gauss_f64(uint64_t seed, uint32_t i, uint32_t j, uint32_t tag) {
  const Philox4 w = philox4x32_10(i, j, tag, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double u1 = ((double)(w.x >> 5) * 67108864.0 + (double)(w.y >> 6) + 0.5) * 0x1.0p-53;
  const double u2 = ((double)(w.z >> 5) * 67108864.0 + (double)(w.w >> 6) + 0.5) * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// FP32 Box-Muller entry from the top 24 bits of words 0 and 2 (mixed path).
RSVD_DEV float gauss_f32(uint64_t seed, uint32_t i, uint32_t j, uint32_t tag) {
  const Philox4 w = philox4x32_10(i, j, tag, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
  const float u1 = ((float)(w.x >> 8) + 0.5f) * 0x1.0p-24f;
  const float u2 = ((float)(w.z >> 8) + 0.5f) * 0x1.0p-24f;
  return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

// FP64 -> FP32 with round-to-nearest-even done on the integer pipe (the FP64
// units are a small fraction of this part's throughput).  Normal results are
// assembled from the bit fields; zeros, subnormal or overflowing results and
// non-finite inputs take the conversion instruction.
static __device__ __noinline__ float f64_to_f32_slow(double a) { return __double2float_rn(a); }

RSVD_DEV float f64_to_f32_rn(double a) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(a);
  const unsigned int e = (unsigned int)(b >> 52) & 0x7FFu;
  const int fe = (int)e - 1023 + 127;
  if (fe <= 0 || fe >= 255) return f64_to_f32_slow(a);   // out of line: never if-converted
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const unsigned int keep = (unsigned int)(m >> 29);
  const unsigned int rest = (unsigned int)(m & 0x1FFFFFFFull);
  const unsigned int up = (rest > 0x10000000u) || (rest == 0x10000000u && (keep & 1u));
  const unsigned int r = ((unsigned int)fe << 23) + keep + up;     // carry into the exponent is RN's overflow
  return __uint_as_float((unsigned int)(b >> 32 & 0x80000000u) | r);
}

// The same rounding from the two 32-bit halves of the FP64 bit pattern (hi
// holds sign, exponent and the top 20 mantissa bits), 32-bit integer ops only.
// Sets `bad` for Inf/NaN.
RSVD_DEV float f64w_to_f32_rn(unsigned int hi, unsigned int lo, bool& bad) {
  const unsigned int e = (hi >> 20) & 0x7FFu;
  bad |= (e == 0x7FFu);
  const int fe = (int)e - 1023 + 127;
  if (fe <= 0 || fe >= 255)
    return f64_to_f32_slow(__hiloint2double((int)hi, (int)lo));
  const unsigned int keep = ((hi & 0xFFFFFu) << 3) | (lo >> 29);     // top 23 mantissa bits
  const unsigned int rest = lo & 0x1FFFFFFFu;                         // the 29 dropped bits
  const unsigned int up = (rest > 0x10000000u) | ((rest == 0x10000000u) & keep);
  return __uint_as_float((hi & 0x80000000u) | (((unsigned int)fe << 23) + keep + (up & 1u)));
}

// Exact FP32 -> FP64 widening on the integer pipe for normal numbers and
// zero; subnormal, Inf and NaN inputs take the conversion instruction.
static __device__ __noinline__ double f32_to_f64_slow(float x) { return (double)x; }

RSVD_DEV double f32_to_f64(float x) {
  const unsigned int u = __float_as_uint(x);
  const unsigned int e = (u >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) {
    if ((u & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)((unsigned long long)(u >> 31) << 63));
    return f32_to_f64_slow(x);
  }
  const unsigned long long b = ((unsigned long long)(u >> 31) << 63) |
                               ((unsigned long long)(e + 896u) << 52) |
                               ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)b);
}

// Exponent all ones: Inf or NaN (integer test, no FP64 instruction).
RSVD_DEV bool f64_nonfinite(double a) {
  return (((unsigned long long)__double_as_longlong(a) >> 52) & 0x7FFull) == 0x7FFull;
}

// ---------------------------------------------------------------------------
// Batched tiling: channel c owns tiles [off[c], off[c+1]).
// ---------------------------------------------------------------------------
RSVD_DEV int find_chan(const int* __restrict__ off, int C, int t) {
  int lo = 0, hi = C - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Device error word codes (set with atomicCAS so the first error wins).
enum : int { DERR_NONE = 0, DERR_TIMEOUT_TMA = 1, DERR_TIMEOUT_MMA = 2, DERR_TIMEOUT_EPI = 3,
             DERR_BAD_ARG = 4, DERR_TIMEOUT_BARRIER = 5 };

RSVD_DEV void set_err(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

// ---------------------------------------------------------------------------
// Tile-rule noise: the 32-bit "lowbias32" integer hash (C. Wellons, "Hash
// function prospector", 2018) and the symmetric entry noise built from it,
//   h = mix(mix(min(i,j) * 0x9E3779B1 + key) ^ (max(i,j) * 0x85EBCA77)),
//   eta_ij = a sqrt(3) (2 u - 1),  u = ((h >> 8) + 1/2) 2^-24,
// uniform with standard deviation a; key = mix(seed_lo ^ mix(seed_hi)).
RSVD_HD uint32_t lowbias32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7FEB352Du;
  x ^= x >> 15;
  x *= 0x846CA68Bu;
  x ^= x >> 16;
  return x;
}

// 2u - 1 = (2 (h >> 8) + 1 - 2^24) 2^-24: the numerator is an odd integer
// below 2^24 in magnitude, so the FP32 value is exact.
RSVD_DEV float rule_eta(uint32_t key, float amp3, int i, int j) {
  const uint32_t lo = (uint32_t)min(i, j), hi = (uint32_t)max(i, j);
  uint32_t h = lowbias32(lo * 0x9E3779B1u + key);
  h = lowbias32(h ^ (hi * 0x85EBCA77u));
  const int num = 2 * (int)(h >> 8) + 1 - (1 << 24);
  return amp3 * ((float)num * 5.9604644775390625e-8f);
}

// Per-channel results written by the device and read once by the host.
struct ChanResult {
  int k_out;
  int l_used;
  int status;
  int flags;        // bit0: shifted CholeskyQR used, bit1: jacobi cap hit, bit2: nonfinite
  double err_est;
  double fro2;      // ||A||_F^2
  int sweeps;       // Jacobi sweeps used (diagnostics)
  int pad_;
  double wres2;     // mixed path: ||A - (sum of its BF16 words)||_F^2 (FP32 remainders)
};

enum : int { FLAG_SHIFTED = 1, FLAG_JACOBI_CAP = 2, FLAG_NONFINITE = 4, FLAG_CHOL_FAIL = 8 };

// ---------------------------------------------------------------------------
// Per-channel pointers of one batched call (device-resident array).
// Tall-skinny matrices are column-major with leading dimension `ldt`;
// l x l matrices column-major with leading dimension `l`.
// ---------------------------------------------------------------------------
struct Chan {
  int n, l, k_cap, k_fixed;
  int col0;                 // first global column of the random matrix for this channel
  double tol;               // this channel's tolerance (0: the plan's)
  int64_t lda;
  const double* A;          // FP64 input (device)
  int64_t ldt;              // leading dim of n x l buffers
  // FP64 path
  double* X;                // n x l   (Omega, then Q)
  double* Y;                // n x l   (products)
  double* Q2;               // n x l   (second basis, FP64 path)
  // small l x l (FP64)
  double* G;                // Gram
  double* R;                // Cholesky factor (upper), accumulates R = R2 R1
  double* Ri;               // inverse of the last Cholesky factor
  float* Ri32;              // optional FP32 copy of Ri (mixed path, l <= 128), then of the lift's X
  double* M;                // Jacobi working matrix (then left vectors X_svd)
  double* J;                // Jacobi rotations (right vectors)
  double* sig;              // singular values (l)
  double* scr;              // l doubles of scratch (unsorted column norms)
  double* gpart;            // Gram partials
  int gsplit;               // number of row splits of the Gram
  float* gtc_part;          // tensor-core Gram tile partials (mixed path, l <= 128), or null
  int* gtc_exp;             // their column exponents
  void* nn_bimg;            // tensor-core tall x small products: the small operand's slice image
  int* nn_fexp;             // and its column exponents
  double* fro_part;         // ||A||^2 partials (one per 64-row block; 8-row on the mixed path)
  // mixed path
  double* wres_part;        // word-split remainder energy partials (one per 8-row block)
  __nv_bfloat16* Ab[3];     // V slices, row-major n x ldb
  __nv_bfloat16* Xb[3];     // X slices, K-major: column j at Xb + j*ldb
  int64_t ldb;
  float* Y32;               // n x lw (sketch / projection output)
  float* Q32;               // n x l
  float* T32;               // n x s probe residual scratch
  int lw;                   // columns of the last product (l + probes)
  int nprobe;
  double* C64;              // l x s  (Q^T A G)
  float* C32;               // l x 32 FP32 copy of C for the probe kernels (mixed path)
  double* est_part;         // probe residual partials
  // outputs
  double* U; int64_t ldu;   // device (internal or user)
  double* V; int64_t ldv;
  double* S;
  ChanResult* res;
  float* feat;              // learned-rank features (19 floats) or null
};

}  // namespace rsvd
