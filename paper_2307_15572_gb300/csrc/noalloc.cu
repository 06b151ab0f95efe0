// rsvd_reconstruct_error_noalloc: the exact-residual check with no device
// allocation at call time.
//
// Who needs it: callers whose device memory is fully reserved up front by
// their own pool (a further cudaMalloc would fail or break the budget), and
// callers that must not let cudaMalloc/cudaFree synchronise the device in
// the middle of a pipeline.  rsvd_reconstruct_error keeps its per-CTA
// partial sums in the plan's workspace, which a plan may have to grow with
// cudaMalloc; this variant keeps them in the fixed array below instead.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it until the process exits, and every call on that GPU
// shares it.  Host code cannot use the symbol as a device address (in host
// code it is only a stand-in), so the address is looked up with
// cudaGetSymbolAddress once per device, with that device current, the first
// time the entry point runs there.  The looked-up address belongs to the
// device's context of that moment: after cudaDeviceReset the entry point
// must not be called again in the same process.
#include <mutex>

#include "kernels.h"

namespace rsvd {

// two doubles per residual CTA: residual^2 and ||A||^2 partials; every call
// writes all of the pairs it then reads, so nothing needs clearing
static constexpr int NOALLOC_MAX_PARTS = 152 * 8;
static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_MAX_PARTS];

// Fixed-order sum of the partials; writes sqrt(r2 / a2) to *out (the
// absolute residual sqrt(r2) when A = 0, where the ratio is undefined).
__global__ void k_noalloc_finish(const double* __restrict__ part, int parts, double* __restrict__ out) {
  __shared__ double s0[256], s1[256];
  double r2 = 0.0, a2 = 0.0;
  for (int t = threadIdx.x; t < parts; t += blockDim.x) {
    r2 += part[2 * t];
    a2 += part[2 * t + 1];
  }
  s0[threadIdx.x] = r2;
  s1[threadIdx.x] = a2;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      s0[threadIdx.x] += s0[threadIdx.x + h];
      s1[threadIdx.x] += s1[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s1[0] > 0.0 ? sqrt(s0[0] / s1[0]) : sqrt(s0[0]);
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_ptr(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = (double*)p;
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}
}  // namespace

}  // namespace rsvd

extern "C" rsvd_status rsvd_reconstruct_error_noalloc(const double* A, int64_t lda, int64_t n,
                                                      const double* U, int64_t ldu, const double* S,
                                                      const double* V, int64_t ldv, int32_t k,
                                                      double* rel_err, void* stream) {
  using namespace rsvd;
  clear_error_text();
  if (n < 1 || n > RSVD_NOALLOC_MAX_N)
    return set_error_text(RSVD_ERR_INVALID_ARG, "n = %lld outside [1, %d] (RSVD_NOALLOC_MAX_N)", (long long)n,
                          RSVD_NOALLOC_MAX_N);
  if (!A || lda < n || !rel_err || k < 0)
    return set_error_text(RSVD_ERR_INVALID_ARG, "bad matrix, leading dimension, output pointer or k");
  if (k > 0 && (!U || !S || !V || ldu < n || ldv < n))
    return set_error_text(RSVD_ERR_INVALID_ARG, "bad factor pointer or leading dimension");
  const int parts = resid_blocks(n);
  if (parts > NOALLOC_MAX_PARTS) return set_error_text(RSVD_ERR_INVALID_ARG, "too many partial sums");
  double* part = nullptr;
  if (cudaError_t e = scratch_ptr(&part))
    return set_error_text(RSVD_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  (void)cudaGetLastError();   // a launch error left by an earlier, unrelated call is not this call's
  cudaStream_t st = (cudaStream_t)stream;
  launch_resid(A, lda, U, ldu, V, ldv, S, (int)n, k, part, st);
  k_noalloc_finish<<<1, 256, 0, st>>>(part, parts, rel_err);
  note_launch(1);
  if (cudaError_t e = cudaGetLastError())
    return set_error_text(RSVD_ERR_CUDA, "residual launch: %s", cudaGetErrorString(e));
  return RSVD_OK;
}
