// Rank-prediction network: forward, backward (chain rule, d tanh = 1 - tanh^2)
// and Adam, FP32, on the GPU.  The matrices are tiny (batch x 128), so every
// kernel assigns one thread per output element and sums in a fixed order:
// results do not depend on the launch configuration.
#include "../../include/rsvd_mlp.h"
#include "kernels.h"

namespace rsvd {

static constexpr int H = RSVD_MLP_HIDDEN;

struct MlpView {
  const float *W1, *b1, *W2, *b2, *W3, *b3;
};

static __host__ __device__ MlpView view(const float* th, int d) {
  MlpView v;
  v.W1 = th;
  v.b1 = v.W1 + (int64_t)d * H;
  v.W2 = v.b1 + H;
  v.b2 = v.W2 + (int64_t)H * H;
  v.W3 = v.b2 + H;
  v.b3 = v.W3 + (int64_t)H * 2;
  return v;
}

// Y (B x O) = act(X (B x I) W (I x O) + b), act = tanh if `tanh_act`.
__global__ void k_linear(const float* __restrict__ X, const float* __restrict__ W, const float* __restrict__ b,
                         float* __restrict__ Y, int B, int I, int O, int tanh_act) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * O) return;
  const int r = e / O, o = e % O;
  float s = b[o];
  for (int i = 0; i < I; ++i) s = fmaf(X[(int64_t)r * I + i], W[(int64_t)i * O + o], s);
  Y[e] = tanh_act ? tanhf(s) : s;
}

// gy = 2 (y - t) / (B * 2); loss = mean (y - t)^2 (one block)
__global__ void k_loss(const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ gy,
                       float* __restrict__ loss, int B) {
  __shared__ float sh[256];
  float s = 0.0f;
  for (int e = threadIdx.x; e < 2 * B; e += blockDim.x) {
    const float r = Y[e] - T[e];
    gy[e] = 2.0f * r / (float)(2 * B);
    s = fmaf(r, r, s);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = sh[0] / (float)(2 * B);
}

// gW (I x O) = X^T G (over the batch), gb (O) = column sums of G.
__global__ void k_wgrad(const float* __restrict__ X, const float* __restrict__ G, float* __restrict__ gW,
                        float* __restrict__ gb, int B, int I, int O) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < I * O) {
    const int i = e / O, o = e % O;
    float s = 0.0f;
    for (int r = 0; r < B; ++r) s = fmaf(X[(int64_t)r * I + i], G[(int64_t)r * O + o], s);
    gW[e] = s;
  } else if (e < I * O + O) {
    const int o = e - I * O;
    float s = 0.0f;
    for (int r = 0; r < B; ++r) s += G[(int64_t)r * O + o];
    gb[o] = s;
  }
}

// Gz (B x I) = (G (B x O) W^T) * (1 - Hact^2), Hact (B x I) the tanh outputs.
__global__ void k_back(const float* __restrict__ G, const float* __restrict__ W, const float* __restrict__ Hact,
                       float* __restrict__ Gz, int B, int I, int O) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * I) return;
  const int r = e / I, i = e % I;
  float s = 0.0f;
  for (int o = 0; o < O; ++o) s = fmaf(G[(int64_t)r * O + o], W[(int64_t)i * O + o], s);
  const float h = Hact[e];
  Gz[e] = s * (1.0f - h * h);
}

__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float gi = g[e];
  const float mi = b1 * m[e] + (1.0f - b1) * gi;
  const float vi = b2 * v[e] + (1.0f - b2) * gi * gi;
  m[e] = mi;
  v[e] = vi;
  th[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

static inline int nb(int64_t n) { return (int)((n + 255) / 256); }

// Fused inference: one block (128 threads, one per hidden unit) per sample;
// the input and both hidden layers stay in shared memory.
__global__ void __launch_bounds__(H) k_mlp_infer(const float* __restrict__ theta, int d,
                                                 const float* __restrict__ X, float* __restrict__ Y) {
  extern __shared__ float xs[];
  __shared__ float h1[H], h2[H], red[2][H / 32];
  const MlpView w = view(theta, d);
  const int r = blockIdx.x, j = threadIdx.x;
  for (int i = j; i < d; i += H) xs[i] = X[(int64_t)r * d + i];
  __syncthreads();
  float s = w.b1[j];
  for (int i = 0; i < d; ++i) s = fmaf(xs[i], w.W1[(int64_t)i * H + j], s);
  h1[j] = tanhf(s);
  __syncthreads();
  s = w.b2[j];
  for (int i = 0; i < H; ++i) s = fmaf(h1[i], w.W2[(int64_t)i * H + j], s);
  h2[j] = tanhf(s);
  __syncthreads();
  // y_o = b3_o + sum_j h2_j W3[j][o]: warp sums then a fixed-order total
  for (int o = 0; o < 2; ++o) {
    float p = h2[j] * w.W3[(int64_t)j * 2 + o];
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) p += __shfl_xor_sync(0xffffffffu, p, k);
    if ((j & 31) == 0) red[o][j >> 5] = p;
  }
  __syncthreads();
  if (j < 2) {
    float t = w.b3[j];
    for (int q = 0; q < H / 32; ++q) t += red[j][q];
    Y[(int64_t)r * 2 + j] = t;
  }
}

}  // namespace rsvd

using namespace rsvd;

// Column statistics of X (N x d, row-major): mean and standard deviation
// (population, floored at sd_floor), sums in FP64 in a fixed order (one block
// per column); then Xn = (X - mean) / sd.
__global__ void k_colstats(const float* __restrict__ X, int N, int d, float sd_floor, float* __restrict__ mean,
                           float* __restrict__ sd) {
  __shared__ double s1[256], s2[256];
  const int col = blockIdx.x;
  double a = 0.0, b = 0.0;
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    const double x = X[(int64_t)r * d + col];
    a += x;
    b = fma(x, x, b);
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      s1[threadIdx.x] += s1[threadIdx.x + h];
      s2[threadIdx.x] += s2[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double m = s1[0] / N;
    const double var = s2[0] / N - m * m;
    mean[col] = (float)m;
    sd[col] = fmaxf((float)sqrt(var > 0.0 ? var : 0.0), sd_floor);
  }
}

__global__ void k_standardize(const float* __restrict__ X, int N, int d, const float* __restrict__ mean,
                              const float* __restrict__ sd, float* __restrict__ Xn) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)N * d) return;
  const int col = (int)(e % d);
  Xn[e] = (X[e] - mean[col]) / sd[col];
}

// A network trained on standardised inputs and targets, rewritten to take
// raw ones: x_n W1 + b1 = x (W1 / sd_x) + (b1 - (mu_x / sd_x) W1), and
// y = y_n sd_t + mu_t, i.e. W3 sd_t and b3 sd_t + mu_t (one thread per output
// parameter; the b1 sums run over d in order).
__global__ void k_fold(const float* __restrict__ th, int d, const float* __restrict__ mx, const float* __restrict__ sx,
                       const float* __restrict__ mt, const float* __restrict__ st, float* __restrict__ out) {
  const MlpView v = view(th, d);
  const MlpView o = view(out, d);
  const int64_t np = (int64_t)d * H + H + (int64_t)H * H + H + 2 * H + 2;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= np) return;
  const int64_t ob1 = (int64_t)d * H, oW2 = ob1 + H, ob2 = oW2 + (int64_t)H * H, oW3 = ob2 + H, ob3 = oW3 + 2 * H;
  float* w = (float*)o.W1;
  if (e < ob1) {
    const int i = (int)(e / H);
    w[e] = v.W1[e] / sx[i];
  } else if (e < oW2) {
    const int h = (int)(e - ob1);
    float s = v.b1[h];
    for (int i = 0; i < d; ++i) s -= (mx[i] / sx[i]) * v.W1[(int64_t)i * H + h];
    w[e] = s;
  } else if (e < oW3) {
    w[e] = th[e];
  } else if (e < ob3) {
    w[e] = th[e] * st[(e - oW3) % 2];
  } else {
    const int j = (int)(e - ob3);
    w[e] = th[e] * st[j] + mt[j];
  }
}

// dst[r, :] = src[idx[r], :] (rows of `cols` floats).
__global__ void k_gather_rows(const float* __restrict__ src, const int64_t* __restrict__ idx, int B, int cols,
                              float* __restrict__ dst) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)B * cols) return;
  const int r = (int)(e / cols), c = (int)(e % cols);
  dst[e] = src[idx[r] * cols + c];
}

extern "C" {

int64_t rsvd_mlp_param_count(int32_t d) {
  return d < 1 ? 0 : (int64_t)d * H + H + (int64_t)H * H + H + (int64_t)H * 2 + 2;
}

int64_t rsvd_mlp_work_floats(int32_t d, int32_t B) {
  (void)d;
  // h1, h2, y, gy, gz2, gz1
  return B < 1 ? 0 : (int64_t)B * (H + H + 2 + 2 + H + H);
}

rsvd_status rsvd_mlp_forward(const float* theta, int32_t d, const float* X, int32_t B, float* Y,
                             void* stream) {
  if (!theta || !X || !Y || d < 1 || d > 1024 || B < 1) return RSVD_ERR_INVALID_ARG;
  k_mlp_infer<<<B, H, (size_t)d * sizeof(float), (cudaStream_t)stream>>>(theta, d, X, Y);
  note_launch(1);
  return cudaGetLastError() == cudaSuccess ? RSVD_OK : RSVD_ERR_CUDA;
}

rsvd_status rsvd_mlp_loss_grad(const float* theta, int32_t d, const float* X, const float* T, int32_t B,
                               float* grad, float* loss, float* work, void* stream) {
  if (!theta || !X || !T || !grad || !loss || !work || d < 1 || B < 1) return RSVD_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const MlpView w = view(theta, d);
  float* h1 = work;
  float* h2 = h1 + (int64_t)B * H;
  float* y = h2 + (int64_t)B * H;
  float* gy = y + (int64_t)B * 2;
  float* gz2 = gy + (int64_t)B * 2;
  float* gz1 = gz2 + (int64_t)B * H;
  float* gW1 = grad;
  float* gb1 = gW1 + (int64_t)d * H;
  float* gW2 = gb1 + H;
  float* gb2 = gW2 + (int64_t)H * H;
  float* gW3 = gb2 + H;
  float* gb3 = gW3 + (int64_t)H * 2;
  k_linear<<<nb((int64_t)B * H), 256, 0, st>>>(X, w.W1, w.b1, h1, B, d, H, 1);
  k_linear<<<nb((int64_t)B * H), 256, 0, st>>>(h1, w.W2, w.b2, h2, B, H, H, 1);
  k_linear<<<nb((int64_t)B * 2), 256, 0, st>>>(h2, w.W3, w.b3, y, B, H, 2, 0);
  k_loss<<<1, 256, 0, st>>>(y, T, gy, loss, B);
  k_wgrad<<<nb((int64_t)H * 2 + 2), 256, 0, st>>>(h2, gy, gW3, gb3, B, H, 2);
  k_back<<<nb((int64_t)B * H), 256, 0, st>>>(gy, w.W3, h2, gz2, B, H, 2);
  k_wgrad<<<nb((int64_t)H * H + H), 256, 0, st>>>(h1, gz2, gW2, gb2, B, H, H);
  k_back<<<nb((int64_t)B * H), 256, 0, st>>>(gz2, w.W2, h1, gz1, B, H, H);
  k_wgrad<<<nb((int64_t)d * H + H), 256, 0, st>>>(X, gz1, gW1, gb1, B, d, H);
  note_launch(9);
  return cudaGetLastError() == cudaSuccess ? RSVD_OK : RSVD_ERR_CUDA;
}

rsvd_status rsvd_mlp_adam(float* theta, const float* grad, float* m, float* v, int64_t nparams, int32_t t,
                          float lr, float beta1, float beta2, float eps, void* stream) {
  if (!theta || !grad || !m || !v || nparams < 1 || t < 1) return RSVD_ERR_INVALID_ARG;
  const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
  k_adam<<<nb(nparams), 256, 0, (cudaStream_t)stream>>>(theta, grad, m, v, nparams, lr, beta1, beta2, eps, c1, c2);
  note_launch(1);
  return cudaGetLastError() == cudaSuccess ? RSVD_OK : RSVD_ERR_CUDA;
}

rsvd_status rsvd_mlp_standardize(const float* X, int32_t N, int32_t d, float sd_floor, float* mean, float* sd,
                                 float* Xn, void* stream) {
  if (!X || !mean || !sd || !Xn || N < 1 || d < 1 || !(sd_floor > 0.0f)) return RSVD_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  k_colstats<<<d, 256, 0, st>>>(X, N, d, sd_floor, mean, sd);
  const int64_t tot = (int64_t)N * d;
  k_standardize<<<(int)((tot + 255) / 256), 256, 0, st>>>(X, N, d, mean, sd, Xn);
  note_launch(2);
  return cudaGetLastError() == cudaSuccess ? RSVD_OK : RSVD_ERR_CUDA;
}

rsvd_status rsvd_mlp_fold(const float* theta, int32_t d, const float* mean_x, const float* sd_x,
                          const float* mean_t, const float* sd_t, float* out, void* stream) {
  if (!theta || !mean_x || !sd_x || !mean_t || !sd_t || !out || d < 1 || out == theta) return RSVD_ERR_INVALID_ARG;
  const int64_t np = rsvd_mlp_param_count(d);
  k_fold<<<(int)((np + 255) / 256), 256, 0, (cudaStream_t)stream>>>(theta, d, mean_x, sd_x, mean_t, sd_t, out);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? RSVD_OK : RSVD_ERR_CUDA;
}

rsvd_status rsvd_mlp_gather_rows(const float* src, const int64_t* idx, int32_t B, int32_t cols, float* dst,
                                 void* stream) {
  if (!src || !idx || !dst || B < 1 || cols < 1) return RSVD_ERR_INVALID_ARG;
  const int64_t tot = (int64_t)B * cols;
  k_gather_rows<<<(int)((tot + 255) / 256), 256, 0, (cudaStream_t)stream>>>(src, idx, B, cols, dst);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? RSVD_OK : RSVD_ERR_CUDA;
}

}  // extern "C"
