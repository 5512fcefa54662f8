// Cost model of the autotuner (include/bandred_tune.h): a two-hidden-layer tanh
// perceptron in FP32 with its forward pass, its mean-squared-error gradient by
// back-propagation and the Adam update (Kingma & Ba 2015, Algorithm 1).
//
// The data are tiny (hundreds of timed configurations, a few thousand parameters), so
// the kernels favour determinism over parallel width: the forward and delta pass runs
// one thread per row, the gradient pass one thread per parameter summing its rows in
// index order, and no atomics are used anywhere.
#include <cmath>

#include "bandred.h"
#include "bandred_tune.h"
#include "prof.h"

namespace bandred {
namespace {

constexpr int kMaxD = 32;
constexpr int kMaxH = 64;
constexpr int kRowThreads = 128;

struct Layout {
  int D, H;
  __host__ __device__ int W1() const { return 0; }
  __host__ __device__ int b1() const { return H * D; }
  __host__ __device__ int W2() const { return H * D + H; }
  __host__ __device__ int b2() const { return H * D + H + H * H; }
  __host__ __device__ int w3() const { return H * D + 2 * H + H * H; }
  __host__ __device__ int b3() const { return H * D + 3 * H + H * H; }
  __host__ __device__ int count() const { return H * D + 3 * H + H * H + 1; }
};

// Per-row work arrays of the gradient pass, rows x H each (row-major) plus two of rows.
struct Work {
  float *h1, *h2, *d1, *d2, *d3, *sq;
};

__host__ __device__ inline Work carve(void* base, int H, int rows) {
  float* f = static_cast<float*>(base);
  const size_t rh = (size_t)rows * H;
  Work w;
  w.h1 = f;
  w.h2 = f + rh;
  w.d1 = f + 2 * rh;
  w.d2 = f + 3 * rh;
  w.d3 = f + 4 * rh;
  w.sq = f + 4 * rh + rows;
  return w;
}

__device__ void load_params(const float* params, float* sp, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) sp[i] = params[i];
  __syncthreads();
}

// Hidden layers of row x: h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2); returns y.
__device__ float row_forward(const Layout& L, const float* sp, const float* x, float* h1, float* h2) {
  for (int h = 0; h < L.H; ++h) {
    float a = sp[L.b1() + h];
    for (int d = 0; d < L.D; ++d) a = fmaf(sp[L.W1() + h * L.D + d], x[d], a);
    h1[h] = tanhf(a);
  }
  float y = sp[L.b3()];
  for (int h = 0; h < L.H; ++h) {
    float a = sp[L.b2() + h];
    for (int g = 0; g < L.H; ++g) a = fmaf(sp[L.W2() + h * L.H + g], h1[g], a);
    h2[h] = tanhf(a);
    y = fmaf(sp[L.w3() + h], h2[h], y);
  }
  return y;
}

__global__ void __launch_bounds__(kRowThreads) mlp_forward_kernel(Layout L, const float* params, const float* X,
                                                                   int rows, float* y) {
  extern __shared__ float sp[];
  load_params(params, sp, L.count());
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  float x[kMaxD], h1[kMaxH], h2[kMaxH];
  for (int d = 0; d < L.D; ++d) x[d] = X[(size_t)r * L.D + d];
  y[r] = row_forward(L, sp, x, h1, h2);
}

// Forward pass and deltas of one row: d3 = dL/dy = 2 (y - t) / rows,
// d2 = d3 w3 * (1 - h2^2), d1 = (W2^T d2) * (1 - h1^2).
__global__ void __launch_bounds__(kRowThreads) mlp_delta_kernel(Layout L, const float* params, const float* X,
                                                                 const float* t, int rows, Work w) {
  extern __shared__ float sp[];
  load_params(params, sp, L.count());
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  float x[kMaxD], h1[kMaxH], h2[kMaxH];
  for (int d = 0; d < L.D; ++d) x[d] = X[(size_t)r * L.D + d];
  const float y = row_forward(L, sp, x, h1, h2);
  const float e = y - t[r];
  const float d3 = 2.0f * e / (float)rows;
  w.d3[r] = d3;
  w.sq[r] = e * e;
  float d2[kMaxH];
  for (int h = 0; h < L.H; ++h) {
    d2[h] = d3 * sp[L.w3() + h] * (1.0f - h2[h] * h2[h]);
    w.h1[(size_t)r * L.H + h] = h1[h];
    w.h2[(size_t)r * L.H + h] = h2[h];
    w.d2[(size_t)r * L.H + h] = d2[h];
  }
  for (int g = 0; g < L.H; ++g) {
    float a = 0.0f;
    for (int h = 0; h < L.H; ++h) a = fmaf(sp[L.W2() + h * L.H + g], d2[h], a);
    w.d1[(size_t)r * L.H + g] = a * (1.0f - h1[g] * h1[g]);
  }
}

// One thread per parameter (and one for the loss): the sum over rows of the product of
// the parameter's upstream activation and downstream delta, rows in index order.
__global__ void mlp_grad_kernel(Layout L, const float* X, int rows, Work w, float* grad, float* loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int P = L.count();
  if (p > P) return;
  float s = 0.0f;
  if (p == P) {
    for (int r = 0; r < rows; ++r) s += w.sq[r];
    *loss = s / (float)rows;
    return;
  }
  const int H = L.H, D = L.D;
  if (p < L.b1()) {
    const int h = p / D, d = p % D;
    for (int r = 0; r < rows; ++r) s = fmaf(w.d1[(size_t)r * H + h], X[(size_t)r * D + d], s);
  } else if (p < L.W2()) {
    const int h = p - L.b1();
    for (int r = 0; r < rows; ++r) s += w.d1[(size_t)r * H + h];
  } else if (p < L.b2()) {
    const int q = p - L.W2(), h = q / H, g = q % H;
    for (int r = 0; r < rows; ++r) s = fmaf(w.d2[(size_t)r * H + h], w.h1[(size_t)r * H + g], s);
  } else if (p < L.w3()) {
    const int h = p - L.b2();
    for (int r = 0; r < rows; ++r) s += w.d2[(size_t)r * H + h];
  } else if (p < L.b3()) {
    const int g = p - L.w3();
    for (int r = 0; r < rows; ++r) s = fmaf(w.d3[r], w.h2[(size_t)r * H + g], s);
  } else {
    for (int r = 0; r < rows; ++r) s += w.d3[r];
  }
  grad[p] = s;
}

__global__ void mlp_adam_kernel(int count, float* params, const float* grad, float* m, float* v, float lr,
                                float beta1, float beta2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float g = grad[i];
  const float mi = beta1 * m[i] + (1.0f - beta1) * g;
  const float vi = beta2 * v[i] + (1.0f - beta2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const float mhat = mi / c1;
  const float vhat = vi / c2;
  params[i] -= lr * mhat / (sqrtf(vhat) + eps);
}

int check_shape(int d_in, int hidden) {
  if (d_in < 1 || d_in > kMaxD) return -1;
  if (hidden < 1 || hidden > kMaxH) return -2;
  return 0;
}

}  // namespace
}  // namespace bandred

using namespace bandred;

extern "C" size_t bandred_mlp_param_count(int d_in, int hidden) {
  if (check_shape(d_in, hidden)) return 0;
  return (size_t)Layout{d_in, hidden}.count();
}

extern "C" size_t bandred_mlp_workspace(int d_in, int hidden, int rows) {
  if (check_shape(d_in, hidden) || rows < 0) return 0;
  return ((size_t)4 * rows * hidden + 2 * (size_t)rows) * sizeof(float) + 256;
}

extern "C" int bandred_mlp_forward(int d_in, int hidden, const float* params, const float* X, int rows, float* y,
                                   cudaStream_t stream) {
  if (int rc = check_shape(d_in, hidden)) return rc;
  if (!params) return -3;
  if (rows < 0) return -5;
  if (rows > 0 && (!X || !y)) return !X ? -4 : -6;
  if (rows == 0) return 0;
  const Layout L{d_in, hidden};
  prof::count_launch();
  mlp_forward_kernel<<<(rows + kRowThreads - 1) / kRowThreads, kRowThreads, L.count() * sizeof(float), stream>>>(
      L, params, X, rows, y);
  return cudaGetLastError() == cudaSuccess ? 0 : BANDRED_ERR_CUDA;
}

extern "C" int bandred_mlp_loss_grad(int d_in, int hidden, const float* params, const float* X, const float* t,
                                     int rows, float* grad, float* loss, void* work, size_t work_bytes,
                                     cudaStream_t stream) {
  if (int rc = check_shape(d_in, hidden)) return rc;
  if (!params) return -3;
  if (rows < 1) return -6;
  if (!X) return -4;
  if (!t) return -5;
  if (!grad) return -7;
  if (!loss) return -8;
  if (!work || work_bytes < bandred_mlp_workspace(d_in, hidden, rows)) return -9;
  const Layout L{d_in, hidden};
  const Work w = carve(work, hidden, rows);
  prof::count_launch(2);
  mlp_delta_kernel<<<(rows + kRowThreads - 1) / kRowThreads, kRowThreads, L.count() * sizeof(float), stream>>>(
      L, params, X, t, rows, w);
  const int P = L.count() + 1;
  mlp_grad_kernel<<<(P + 127) / 128, 128, 0, stream>>>(L, X, rows, w, grad, loss);
  return cudaGetLastError() == cudaSuccess ? 0 : BANDRED_ERR_CUDA;
}

extern "C" int bandred_mlp_adam(int count, float* params, const float* grad, float* m, float* v, int step, float lr,
                                float beta1, float beta2, float eps, cudaStream_t stream) {
  if (count < 0) return -1;
  if (count > 0 && !params) return -2;
  if (count > 0 && !grad) return -3;
  if (count > 0 && !m) return -4;
  if (count > 0 && !v) return -5;
  if (step < 1) return -6;
  if (!(lr > 0.0f)) return -7;
  if (!(beta1 >= 0.0f && beta1 < 1.0f)) return -8;
  if (!(beta2 >= 0.0f && beta2 < 1.0f)) return -9;
  if (!(eps > 0.0f)) return -10;
  if (count == 0) return 0;
  // bias corrections 1 - beta^step, computed on the host in double
  const float c1 = (float)(1.0 - std::pow((double)beta1, step));
  const float c2 = (float)(1.0 - std::pow((double)beta2, step));
  prof::count_launch();
  mlp_adam_kernel<<<(count + 255) / 256, 256, 0, stream>>>(count, params, grad, m, v, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? 0 : BANDRED_ERR_CUDA;
}
