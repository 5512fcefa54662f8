// Diagnostics declared in include/bandred.h: direct evaluation of the panel kernels'
// Newton-Raphson reciprocal square root and reciprocal (so that they can be checked
// against their error bounds on their own), and an FP64 fused-multiply-add throughput
// probe (the FP64 roofline of the plain FP64 path and of the panels).
#include <algorithm>
#include <cstdint>

#include "driver.h"
#include "panel_common.cuh"
#include "prof.h"

namespace bandred {
namespace {

__global__ void newton_eval_kernel(int64_t count, const double* x, double* rs, double* rc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    if (rs) rs[i] = panel_detail::rsqrt_newton(v);
    if (rc) rc[i] = panel_detail::rcp_newton(v);
  }
}

// 8 independent chains per thread hide the FMA latency; the coefficients keep every chain
// bounded (a fixed point near 1), so no value overflows whatever `iters` is.
__global__ void fp64_probe_kernel(int iters, double* sink) {
  double a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  const double m = 0.999999, k = 1e-6;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = fma(a[c], m, k);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += a[c];
  sink[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace bandred

extern "C" int bandred_newton_eval(int64_t count, const double* x, double* rsqrt, double* rcp, cudaStream_t stream) {
  if (count < 0) return -1;
  if (count > 0 && !x) return -2;
  if (count == 0) return 0;
  bandred::DeviceGuard dg;
  if (!dg.select(x)) return -2;
  const int blocks = (int)std::min<int64_t>((count + 255) / 256, 4096);
  bandred::prof::count_launch();
  bandred::newton_eval_kernel<<<blocks, 256, 0, stream>>>(count, x, rsqrt, rcp);
  if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return bandred::record_cuda_error(e, "newton_eval_kernel");
  return 0;
}

extern "C" int bandred_fp64_probe(int blocks, int threads, int iters, double* sink, cudaStream_t stream) {
  if (blocks < 1) return -1;
  if (threads < 32 || threads > 1024 || threads % 32) return -2;
  if (iters < 1) return -3;
  if (!sink) return -4;
  bandred::DeviceGuard dg;
  if (!dg.select(sink)) return -4;
  bandred::prof::count_launch();
  bandred::fp64_probe_kernel<<<blocks, threads, 0, stream>>>(iters, sink);
  if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return bandred::record_cuda_error(e, "fp64_probe_kernel");
  return 0;
}
