// Device helpers shared by the panel kernels (panel.cu: cooperative grid over all SMs;
// panel_cluster.cu: one thread-block cluster per panel).
#pragma once
#include <cmath>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace bandred {
namespace panel_detail {

constexpr int kPanelThreads = 256;

// The per-reflector reductions are accumulated with FP64 atomic adds in L2 (one value per
// 256-byte line, three rotating buffers), so no CTA spends its FP64 pipe on summing the
// partials of the others.  The order of those additions is not fixed: results agree
// across runs to rounding, not bit for bit.
constexpr int kAccStride = 32;  // doubles between accumulated values (one 256-byte line)

// One accumulator buffer holds, kAccStride doubles apart: the sums of a step (2 bk + 2 for
// the pair kernel, 4 bk + 2 for the four-reflector kernel), then, from entry
// kRescaleSlot bk + 2, the bk sums of the rare path's scaled second pass.
constexpr int kRescaleSlot = 4;
__host__ __device__ inline size_t panel_acc_entries(int bk) { return (size_t)(kRescaleSlot + 1) * bk + 2; }

// Reciprocal square root and reciprocal of a positive normal FP64 number by Newton-Raphson
// iteration.  The start is the FP32 hardware estimate for the mantissa (rsqrtf / __frcp_rn,
// about 22 correct bits), with the exponent handled by integer operations; two
// Newton-Raphson steps in FP64 follow, r <- r (3/2 - (q/2) r^2) for 1/sqrt(q) and
// r <- r + r (1 - s r) for 1/s, each roughly doubling the number of correct bits, so the
// result is within a few units in the last place of the exact value.  They stand in for
// FP64 square root and division on the reflector's critical path: 6 and 4 dependent FP64
// operations.
__device__ __forceinline__ double rsqrt_newton(double q) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(q);
  const int e = (int)((u >> 52) & 0x7FF) - 1023;
  const int k = e >> 1;  // floor(e / 2)
  const int em = e - 2 * k;  // 0 or 1: q = m 2^(2k), m in [1, 4)
  const double hm = __longlong_as_double((long long)((u & 0x000FFFFFFFFFFFFFull) | ((unsigned long long)(1022 + em) << 52)));
  const float mf = __uint_as_float(((uint32_t)(127 + em) << 23) | (uint32_t)((u >> 29) & 0x7FFFFFu));
  double r = tc::f32_to_f64(rsqrtf(mf));
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double t = fma(-hm, r * r, 1.5);
    r = r * t;
  }
  return __longlong_as_double(__double_as_longlong(r) - ((long long)k << 52));
}

__device__ __forceinline__ double rcp_newton(double s) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(s);
  const int e = (int)((u >> 52) & 0x7FF) - 1023;
  const double m = __longlong_as_double((long long)((u & 0x000FFFFFFFFFFFFFull) | (1023ull << 52)));
  const float mf = __uint_as_float((127u << 23) | (uint32_t)((u >> 29) & 0x7FFFFFu));
  double r = tc::f32_to_f64(__frcp_rn(mf));
#pragma unroll
  for (int it = 0; it < 2; ++it) r = fma(r, fma(-m, r, 1.0), r);
  return __longlong_as_double(__double_as_longlong(r) - ((long long)e << 52));
}

// Range and sign tests of FP64 values by integer compares of their bit patterns (no FP64
// instruction, so they do not queue behind the scalar chain on the FP64 pipe).  For
// x >= 0 and for NaN the order of the patterns as signed 64-bit integers is the order of
// the values (NaN above +inf, or below zero when its sign bit is set), so each test below
// gives the same answer as the FP64 comparison it replaces.
constexpr long long kBits2p1000 = 0x7E70000000000000LL;   // 2^1000
constexpr long long kBits2p500 = 0x5F30000000000000LL;    // 2^500
constexpr long long kBits2m450 = 0x23D0000000000000LL;    // 2^-450
constexpr long long kBits2m900 = 0x07B0000000000000LL;    // 2^-900
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ long long abits(double x) { return __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL; }
// x >= 0.0 (true for -0.0 as well)
__device__ __forceinline__ bool nonneg(double x) {
  const long long u = dbits(x);
  return u >= 0 || (u << 1) == 0;
}
// -x when c, else x (a sign flip, exact)
__device__ __forceinline__ double neg_if(double x, bool c) {
  return __longlong_as_double(dbits(x) ^ (c ? (long long)0x8000000000000000ULL : 0LL));
}

// FP64 -> FP32 by integer truncation of the mantissa (no FP64 instruction); values
// outside FP32's normal range take the ordinary conversion.
__device__ __forceinline__ float f64_to_f32_rz(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7FF) - 1023;
  if (e < -126 || e > 127) return (float)x;
  return __uint_as_float((uint32_t)((u >> 32) & 0x80000000u) | ((uint32_t)(e + 127) << 23) |
                         (uint32_t)((u >> 29) & 0x7FFFFFu));
}

// W(:, i) in FP32 (used when W only feeds split-precision products, whose bf16 slices
// keep 24 bits): same recurrence, eight lanes per row.
// Threads t0 .. t0 + nth - 1 of the CTA take part (nth a multiple of 8).
__device__ __forceinline__ void w_column_f32(int i, float tau, const float* g, const double* slab, int Rp, int rb,
                                             int nr, float* wl, int t0 = 0, int nth = kPanelThreads) {
  constexpr int PARTS = 8;
  const int lt = (int)threadIdx.x - t0;
  const int part = lt % PARTS;
  for (int r0 = 0; r0 < nr; r0 += nth / PARTS) {
    const int r = r0 + lt / PARTS;
    float s = 0.f;
    if (r < nr)
      for (int q = part; q < i; q += PARTS) s = fmaf(wl[r + q * Rp], g[q], s);
#pragma unroll
    for (int o = PARTS / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (part == 0 && r < nr) {
      const int gr = rb + r;
      const float y = gr > i ? f64_to_f32_rz(slab[(size_t)i * Rp + r]) : (gr == i ? 1.f : 0.f);
      wl[r + i * Rp] = -tau * (y + s);
    }
  }
}

// W(:, i) = -tau_i (y_i + W(:, 0:i) g) for this CTA's rows, g = Y(:, 0:i)^T y_i.  Eight
// lanes share a row (each sums every eighth term), so every warp of the CTA takes part:
// an FP64 instruction costs the same pipe time whether one lane or 32 are active.
__device__ __forceinline__ void w_column(int i, double tau, const double* g, const double* slab, int Rp, int rb,
                                         int nr, double* wl, int64_t wld, int t0 = 0, int nth = kPanelThreads) {
  constexpr int PARTS = 8;
  const int lt = (int)threadIdx.x - t0;
  const int part = lt % PARTS;
  for (int r0 = 0; r0 < nr; r0 += nth / PARTS) {
    const int r = r0 + lt / PARTS;
    double s0 = 0.0, s1 = 0.0;
    if (r < nr) {
      int q = part;
      for (; q + PARTS < i; q += 2 * PARTS) {
        s0 = fma(wl[r + (int64_t)q * wld], g[q], s0);
        s1 = fma(wl[r + (int64_t)(q + PARTS) * wld], g[q + PARTS], s1);
      }
      if (q < i) s0 = fma(wl[r + (int64_t)q * wld], g[q], s0);
    }
    s0 += s1;
#pragma unroll
    for (int o = PARTS / 2; o > 0; o >>= 1) s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    if (part == 0 && r < nr) {
      const int gr = rb + r;
      const double y = gr > i ? slab[(size_t)i * Rp + r] : (gr == i ? 1.0 : 0.0);
      wl[r + (int64_t)i * wld] = -tau * (y + s0);
    }
  }
}

}  // namespace panel_detail
}  // namespace bandred
