// rsvd_reconstruct_error_noalloc: the exact-residual check with no device
// allocation at call time.
//
// Who needs it: callers whose device memory is fully reserved up front by
// their own pool (a further cudaMalloc would fail or break the budget), and
// callers that must not let cudaMalloc/cudaFree synchronise the device in
// the middle of a pipeline.  rsvd_reconstruct_error keeps its per-tile
// partial sums in the plan's workspace, which a plan may have to grow with
// cudaMalloc; this variant keeps them in the fixed array below instead.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (1 MiB) until the process exits, and every call on that
// GPU shares it.  Host code cannot use the symbol as a device address (in
// host code it is only a stand-in), so the address is looked up with
// cudaGetSymbolAddress once per device, with that device current, the first
// time the entry point runs there.
#include <mutex>

#include "kernels.h"

namespace rsvd {

static constexpr int NOALLOC_MAX_N = RSVD_NOALLOC_MAX_N;
static constexpr int NOALLOC_MAX_TILES = ((NOALLOC_MAX_N + 63) / 64) * ((NOALLOC_MAX_N + 63) / 64);

// two doubles per 64 x 64 tile: residual^2 and ||A||^2 partials
static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_MAX_TILES];

// Fixed-order sum of the tile partials; writes sqrt(r2 / a2) to *out.
__global__ void k_noalloc_finish(const double* __restrict__ part, int tiles, double* __restrict__ out) {
  __shared__ double s0[256], s1[256];
  double r2 = 0.0, a2 = 0.0;
  for (int t = threadIdx.x; t < tiles; t += blockDim.x) {
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
  if (n < 1 || n > NOALLOC_MAX_N) return RSVD_ERR_INVALID_ARG;
  if (!A || lda < n || !rel_err || k < 0) return RSVD_ERR_INVALID_ARG;
  if (k > 0 && (!U || !S || !V || ldu < n || ldv < n)) return RSVD_ERR_INVALID_ARG;
  double* part = nullptr;
  if (scratch_ptr(&part) != cudaSuccess) return RSVD_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const int tiles = resid_tiles((int)n);
  // every tile writes its own pair of partials, so nothing needs clearing
  launch_resid(A, lda, U, ldu, V, ldv, S, (int)n, k, part, st);
  k_noalloc_finish<<<1, 256, 0, st>>>(part, tiles, rel_err);
  note_launch(1);
  return cudaGetLastError() == cudaSuccess ? RSVD_OK : RSVD_ERR_CUDA;
}
