// Second stage after the band form (the step the paper's eigenvalue experiments take with
// SBRDT and DSTERF): the symmetric band B (bandwidth w) is reduced to a tridiagonal T by
// Householder bulge chasing, and the eigenvalues of T are found by trisection on Sturm
// counts.
//
// Bulge chasing.  Sweep c (c = 0 .. n-3) annihilates B(c+2 : c+w+1, c) with a reflector
// on the index range [c+1, c+1+w), applied from both sides; its right application to
// the rows below the range fills a triangle below the band, and the sweep's next
// reflector annihilates that bulge's first column below its in-band entry, on the range
// shifted by w, down to the end of the matrix (the bulge's other columns are taken by
// the sweeps that follow).  Each reflector follows the larfg convention (beta =
// -sign(alpha) ||x||, sign(0) = +1; tau = 0 for a zero tail).
//
// GB300 mapping.  The band lives in a compact lower band store of 2w rows per column
// (offsets 0 .. 2w-1 hold the band and the bulge), which stays in L2 (n = 8192, w = 64:
// 8 MB).  One persistent cooperative kernel: CTA g runs sweeps g, g + G, ... in order, and
// each sweep publishes its progress in a counter that the next sweep waits on (bounded:
// past the time limit the kernel records BANDRED_DEV_TIMEOUT and returns).  Step t of
// sweep c, range start s, touches entries whose column lies in [s - w, s + w) and whose
// row lies in [s, s + 2w); step t'' of sweep c - 1 those with columns from s - 1 +
// (t'' - t - 1) w and rows from s - 1 + (t'' - t) w.  Every entry must see the sweeps'
// updates in sequential order, so step t of sweep c needs step t + 1 of sweep c - 1
// finished; of step t + 2 it shares a single entry, (s + 2w - 1, s + w - 1), the first
// entry of that step's column.
//   * The L2 kernel (w <= 128) waits for step t + 2 of the sweep before.
//   * The shared-memory kernel (w <= 64) writes each step's column (beta, 0, ..) during
//     the step before, as soon as that step's right application has made it final, and a
//     sweep's counter at t + 1 means "steps <= t done and step t + 1's column written":
//     step t waits for t + 2 on the counter of the sweep before, a lag of two steps.
// Either way the result equals the one-sweep-at-a-time algorithm up to the rounding of
// the sums.  Within a step the three blocks the reflector touches (the bulge columns to
// the left of the range, the symmetric diagonal block, the rows below the range) are
// independent vectors.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "driver.h"
#include "panel_common.cuh"
#include "kernels.h"
#include "launch.h"
#include "prof.h"
#include "tc.cuh"

namespace bandred {
namespace {

using panel_detail::abits;
using panel_detail::dbits;
using panel_detail::kBits2m450;
using panel_detail::kBits2p1000;
using panel_detail::kBits2p500;
using panel_detail::neg_if;
using panel_detail::nonneg;

constexpr int kChaseThreads = 256;
constexpr int kMaxW = 128;  // reflector length <= w <= 128: four entries per lane
constexpr int kDone = 1 << 30;
constexpr int kPhaseSlots = 16;

struct ChaseParams {
  int n, w, LB;       // LB = 2w: rows of the band store per column
  double* Bs;         // entry (i, k), 0 <= i - k < LB, at Bs[(i - k) + k * LB]
  int* prog;          // prog[c]: steps sweep c has finished (kDone when finished)
  int* status;
  unsigned long long limit_ns;
  long long* phases;  // diagnostic: clock64 at kPhaseSlots points of each step of sweep phase_sweep, or nullptr
  int phase_steps, phase_sweep;
};

// Loads go to L2 (ld.cg): another CTA may have changed a line this SM read before.
__device__ __forceinline__ double ldb(const ChaseParams& p, int i, int k) {
  return __ldcg(&p.Bs[(int64_t)(i - k) + (int64_t)k * p.LB]);
}
__device__ __forceinline__ void stb(const ChaseParams& p, int i, int k, double x) {
  p.Bs[(int64_t)(i - k) + (int64_t)k * p.LB] = x;
}
// q / d for 0 <= q < 2^20, 1 <= d <= 128, from the FP32 reciprocal rd of d plus one
// integer correction each way (the product is within one of the quotient): the staging
// loops divide by the block's runtime row count many times a step
__device__ __forceinline__ int fdiv(int q, int d, float rd) {
  int j = __float2int_rz((float)q * rd);
  j += (j + 1) * d <= q;
  j -= j * d > q;
  return j;
}

// symmetric read of the band store (either triangle)
__device__ __forceinline__ double bsym(const ChaseParams& p, int i, int k) {
  return i >= k ? ldb(p, i, k) : ldb(p, k, i);
}

__device__ __forceinline__ int ld_acquire_int(const int* q) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(q) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_int(int* q, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(q), "r"(v) : "memory");
}

__global__ void __launch_bounds__(kChaseThreads) sb2st_chase_kernel(ChaseParams p) {
  __shared__ double v[kMaxW];       // the reflector (v[0] = 1)
  __shared__ double pdiag[kMaxW];   // tau * B(R, R) v, then K = p - (tau/2)(p.v) v
  __shared__ double red[kChaseThreads / 32];
  __shared__ double s_tau, s_beta, s_scal, s_sx, s_half;
  __shared__ int s_ok;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kChaseThreads / 32;
  const int n = p.n, w = p.w;
  for (int c = blockIdx.x; c + 2 < n; c += gridDim.x) {
    int col = c, s = c + 1, t = 0;
    while (true) {
      const int end = min(s + w, n), len = end - s;
      if (len < 2) break;
      // wait for sweep c - 1 to pass step t + 2 (or to finish)
      if (tid == 0) {
        int ok = 1;
        if (c > 0) {
          unsigned long long t0 = 0;
          unsigned int spins = 0;
          while (ld_acquire_int(&p.prog[c - 1]) < t + 3) {
            if ((++spins & 63u) == 0u) {
              const unsigned long long now = global_ns();
              if (t0 == 0) t0 = now;
              else if (now - t0 > p.limit_ns) {
                if (p.status) atomicCAS(p.status, 0, BANDRED_DEV_TIMEOUT);
                ok = 0;
                break;
              }
              if (p.status && ld_acquire_int(p.status) != 0) { ok = 0; break; }
            }
          }
        }
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok) return;

      // reflector from x = B(s : end, col): warp 0 forms max |x2| and the scaled sum
      if (warp == 0) {
        double xv[4], amax = 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = lane + 32 * u;
          xv[u] = (i < len) ? ldb(p, s + i, col) : 0.0;
          if (i >= 1 && i < len) amax = fmax(amax, fabs(xv[u]));
          if (i < len) v[i] = xv[u];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        // tiny vectors by exact power-of-two scalings (see chase_reflector)
        const double alpha = __shfl_sync(0xffffffffu, xv[0], 0);
        const double sx = fmax(amax, fabs(alpha)) < 0x1p-900 ? 0x1p600 : 1.0;
        const double am = amax * sx, ns = am < 0x1p-900 ? 0x1p600 : 1.0;
        double ss = 0.0;
        if (amax > 0.0) {
          const double inv = 1.0 / (am * ns);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = lane + 32 * u;
            if (i >= 1 && i < len) {
              const double q = ((xv[u] * sx) * ns) * inv;
              ss = fma(q, q, ss);
            }
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) {
          double tau = 0.0, beta = alpha, scal = 1.0;
          if (amax > 0.0) {
            const double as = alpha * sx;
            const double h = hypot(as, am * sqrt(ss));
            const double bs = as >= 0.0 ? -h : h;
            tau = (bs - as) / bs;
            scal = 1.0 / (as - bs);
            beta = bs * (1.0 / sx);
          }
          s_tau = tau;
          s_beta = beta;
          s_scal = scal;
          s_sx = sx;
        }
      }
      __syncthreads();
      const double tau = s_tau;
      // v = [1; x2 scal]; the column becomes [beta; 0 ...]
      for (int i = tid; i < len; i += kChaseThreads) {
        stb(p, s + i, col, i == 0 ? s_beta : 0.0);
      }
      __syncthreads();
      if (tid < len) v[tid] = tid == 0 ? 1.0 : (v[tid] * s_sx) * s_scal;
      __syncthreads();

      if (tau != 0.0) {
        // phase A, one warp per vector: the bulge columns j in (col, s) (left
        // application), the rows i in [end, end + w) below the range (right application),
        // and p = tau B(R, R) v over the symmetric diagonal block
        const int nb = s - col - 1;                 // bulge columns
        const int nl = min(end + w, n) - end;       // rows below
        const int items = nb + nl + len;
        for (int it = warp; it < items; it += NW) {
          double vv[4], a[4];
          if (it < nb) {
            const int j = col + 1 + it;
            double z = 0.0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int i = lane + 32 * u;
              vv[u] = i < len ? v[i] : 0.0;
              a[u] = i < len ? ldb(p, s + i, j) : 0.0;
              z = fma(vv[u], a[u], z);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
            z *= tau;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int i = lane + 32 * u;
              if (i < len) stb(p, s + i, j, fma(-z, vv[u], a[u]));
            }
          } else if (it < nb + nl) {
            const int i = end + (it - nb);
            double y = 0.0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int k = lane + 32 * u;
              vv[u] = k < len ? v[k] : 0.0;
              a[u] = k < len ? ldb(p, i, s + k) : 0.0;
              y = fma(a[u], vv[u], y);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
            y *= tau;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int k = lane + 32 * u;
              if (k < len) stb(p, i, s + k, fma(-y, vv[u], a[u]));
            }
          } else {
            const int i = it - nb - nl;
            double y = 0.0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int k = lane + 32 * u;
              if (k < len) y = fma(bsym(p, s + i, s + k), v[k], y);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
            if (lane == 0) pdiag[i] = tau * y;
          }
        }
        __syncthreads();
        // K = p - (tau/2)(p.v) v
        double pv = 0.0;
        if (tid < len) pv = pdiag[tid] * v[tid];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pv += __shfl_xor_sync(0xffffffffu, pv, o);
        if (lane == 0) red[warp] = pv;
        __syncthreads();
        if (tid == 0) {
          double sum = 0.0;
          for (int q = 0; q < NW; ++q) sum += red[q];
          s_half = 0.5 * tau * sum;
        }
        __syncthreads();
        if (tid < len) pdiag[tid] = fma(-s_half, v[tid], pdiag[tid]);
        __syncthreads();
        // phase B: B(R, R) -= v K^T + K v^T on the stored lower triangle
        for (int q = tid; q < len * len; q += kChaseThreads) {
          const int i = q % len, k = q / len;
          if (i >= k) stb(p, s + i, s + k, fma(-v[i], pdiag[k], fma(-pdiag[i], v[k], ldb(p, s + i, s + k))));
        }
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release_int(&p.prog[c], t + 1);
      }
      col = s;
      s += w;
      ++t;
    }
    if (tid == 0) {
      __threadfence();
      st_release_int(&p.prog[c], kDone);
    }
  }
}

// The same chase with the step's blocks in shared memory (w <= 64), one thread per
// vector (no warp reductions: every FP64 instruction does useful work).
//
// Carry.  After step t's right application, the rows below its range, B(end : end + w,
// s : end), are exactly the column that step t + 1 annihilates (their first column) and
// step t + 1's bulge columns (the others), and nothing else writes them in between (the
// sweep before has finished with them; of the sweep after, step t - 1 reads only their
// first entry, the next step's column, written to global memory early, and step t waits
// for step t + 1).  So they stay in shared memory and reach global memory once, as step
// t + 1's bulge columns.
//
// Copies.  A step's own blocks (its diagonal block and the rows below it) are final once
// its wait is over (the sweep before has finished its step t + 1 and written the column of
// its step t + 2); they go to shared memory on the TMA engine, each warp issuing the bulk
// copies of eight columns, completing on an mbarrier.  In the band store, column j of a
// step's range holds its diagonal-block part (offsets 0 .. len - j) and its rows-below
// part (offsets len - j .. len - j + nl) back to back, so one bulk copy per column brings
// both (rounded up to whole 16-byte pairs), into a column block with a stride of kCLd
// doubles: (i, j) of the diagonal block (i >= j) at kC j + i, and row r of the rows
// below in column k at kC k + len + r, kC = kCLd - 1 = 129.  A thread per row and a thread
// per column both step by 1 or by 129 = 1 (mod 16) words, and across the diagonal (k > i)
// the word kC i + k has the bank of kC k + i: no access pattern here has bank conflicts.
// While the copies are in flight the step forms its reflector's vector from the carried
// column.
//
// Buffers: two column blocks used in turn: this step's, and the one of the step before
// (whose rows below are this step's column and bulge).
constexpr int kSMaxW = 64;
constexpr int kCLd = 2 * kSMaxW + 2;  // even: every column starts on 16 bytes
constexpr int kC = kCLd - 1;
constexpr size_t kCBlk = (size_t)kSMaxW * kCLd;
constexpr int kChaseWarps = kChaseThreads / 32;
constexpr int kTri = kSMaxW * (kSMaxW + 1) / 2;  // entries of a diagonal block's lower triangle
constexpr size_t kSmemChase = sizeof(double) * (2 * kCBlk + 10 * kSMaxW) + sizeof(uint16_t) * kTri;
static_assert(kChaseThreads == 4 * kSMaxW && kChaseWarps == 8, "phase A's split over eight warps");
static_assert((kCBlk * sizeof(double)) % 16 == 0, "blocks on 16-byte boundaries");
static_assert(kSmemChase <= 227 * 1024, "shared memory of one CTA");

// The copy of column j of the step with range length lx and nx rows below: offsets
// 0 .. lx - j + nx of the band store's column, rounded up to whole pairs.
__device__ __forceinline__ uint32_t chase_col_bytes(int lx, int nx, int j) {
  const int m = lx - j + nx;
  return 8u * (uint32_t)(m + (m & 1));
}

// Issues the copies of the step with range [sx, sx + lx) and nx rows below into C,
// completing on bar (expected arrivals: one per warp).  Called by every warp: warp g
// takes columns g, g + 8, ...
__device__ __forceinline__ void chase_issue(const ChaseParams& p, int sx, int lx, int nx, double* C, uint64_t* bar,
                                            int g, int lane) {
  uint32_t bytes = 0;
  const int j = g + kChaseWarps * lane;
  if (j < lx) bytes = chase_col_bytes(lx, nx, j);
  bytes = __reduce_add_sync(0xffffffffu, bytes);
  // the band columns were written by other CTAs (generic stores, seen through this
  // sweep's acquire of the counter) and are read here by the TMA engine (async proxy)
  tc::fence_proxy_async_global();
  tc::fence_proxy_async();
  if (lane == 0) tc::mbar_arrive_expect_tx(bar, bytes);
  __syncwarp();
  if (j < lx) tc::bulk_g2s(C + (size_t)j * kCLd, p.Bs + (int64_t)(sx + j) * p.LB, chase_col_bytes(lx, nx, j), bar);
}

// One warp's half of a vector of phase A (k in [k0, k0 + 32)): y[kk] = b[kk st] for
// k0 + kk < len, in registers; returns sum v[k0 + kk] y[kk] (four chains).
__device__ __forceinline__ double half_load_dot(const double* b, int st, const double* v, int k0, int len,
                                                double (&y)[32]) {
#pragma unroll
  for (int kk = 0; kk < 32; ++kk) y[kk] = k0 + kk < len ? b[kk * st] : 0.0;
  double z0 = 0.0, z1 = 0.0, z2 = 0.0, z3 = 0.0;
#pragma unroll
  for (int kk = 0; kk < 32; kk += 4) {
    if (k0 + kk < len) z0 = fma(v[k0 + kk], y[kk], z0);
    if (k0 + kk + 1 < len) z1 = fma(v[k0 + kk + 1], y[kk + 1], z1);
    if (k0 + kk + 2 < len) z2 = fma(v[k0 + kk + 2], y[kk + 2], z2);
    if (k0 + kk + 3 < len) z3 = fma(v[k0 + kk + 3], y[kk + 3], z3);
  }
  return (z0 + z1) + (z2 + z3);
}
// b[kk st] = y[kk] - z v[k0 + kk] for k0 + kk < len
__device__ __forceinline__ void half_update(double* b, int st, const double* v, int k0, int len, double z,
                                            const double (&y)[32]) {
#pragma unroll
  for (int kk = 0; kk < 32; ++kk) {
    if (k0 + kk < len) b[kk * st] = fma(-z, v[k0 + kk], y[kk]);
  }
}

// The reflector of x[0 .. len) (one whole warp; lane 0 writes tau, beta and the tail's
// scale, v = (x sx) scal), larfg convention.  Common path: the plain sum of squares when it
// and |alpha| are safely in range (max |x2| from the bit patterns, integer compares off the
// FP64 pipe), then h = ||x|| = q / sqrt(q), tau = 1 + |alpha| / h and 1 / (alpha - beta) by
// Newton-Raphson; otherwise the max-scaled sum and hypot.  Along a long chase the bulge's
// far entries decay towards the underflow threshold, so in the latter path tiny vectors
// take exact power-of-two scalings: when every entry is below 2^-900 the reflector is
// formed from x 2^600 (the same tau and v, beta scaled back), and a tail below 2^-900
// beside a larger alpha is scaled by 2^600 in the sum of squares, where 1 / max would
// overflow.
__device__ __forceinline__ void chase_reflector(const double* x, int len, int lane, double* o_tau, double* o_beta,
                                                double* o_scal, double* o_sx) {
  unsigned long long um = 0ull;
  double ss = 0.0;
  for (int i = 1 + lane; i < len; i += 32) {
    const double xi = x[i];
    const unsigned long long u = (unsigned long long)__double_as_longlong(xi) & 0x7FFFFFFFFFFFFFFFull;
    um = u > um ? u : um;
    ss = fma(xi, xi, ss);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, um, o);
    um = u > um ? u : um;
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
  }
  const double amax = __longlong_as_double((long long)um), alpha = x[0];
  const bool plain = (long long)um > kBits2m450 && dbits(ss) < kBits2p1000 && abits(alpha) < kBits2p500;
  const double sx = (!plain && fmax(amax, fabs(alpha)) < 0x1p-900) ? 0x1p600 : 1.0;
  const double am = amax * sx;
  if (um != 0ull && !plain) {  // rare: scaled sum (warp-uniform branch)
    const double ns = am < 0x1p-900 ? 0x1p600 : 1.0;
    const double inv = 1.0 / (am * ns);
    ss = 0.0;
    for (int i = 1 + lane; i < len; i += 32) {
      const double q = ((x[i] * sx) * ns) * inv;
      ss = fma(q, q, ss);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  }
  if (lane == 0) {
    double tau = 0.0, beta = alpha, scal = 1.0;
    if (um != 0ull) {
      if (plain) {
        const double q = fma(alpha, alpha, ss);
        const double rq = panel_detail::rsqrt_newton(q);
        const double h = q * rq, aa = __longlong_as_double(abits(alpha));
        const bool apos = nonneg(alpha);
        beta = neg_if(h, apos);
        tau = fma(aa, rq, 1.0);
        scal = neg_if(panel_detail::rcp_newton(aa + h), !apos);
      } else {
        const double as = alpha * sx;
        const double h = hypot(as, am * sqrt(ss));
        const double bs = as >= 0.0 ? -h : h;
        tau = (bs - as) / bs;
        scal = 1.0 / (as - bs);
        beta = bs * (1.0 / sx);
      }
    }
    *o_tau = tau;
    *o_beta = beta;
    *o_scal = scal;
    *o_sx = sx;
  }
}

// (i, k), k <= i < len, of entry q of a lower triangle packed column by column:
// q = off(k) + i - k, off(k) = k len - k (k - 1) / 2
__device__ __forceinline__ void tri_entry(int q, int len, int& i, int& k) {
  const float a = 2.0f * (float)len + 1.0f;
  k = (int)((a - sqrtf(a * a - 8.0f * (float)q)) * 0.5f);
  k = max(0, min(k, len - 1));
  while (k > 0 && k * len - k * (k - 1) / 2 > q) --k;
  while (k + 1 < len && (k + 1) * len - (k + 1) * k / 2 <= q) ++k;
  i = k + q - (k * len - k * (k - 1) / 2);
}

__global__ void __launch_bounds__(kChaseThreads, 1) sb2st_chase_smem_kernel(ChaseParams p) {
  extern __shared__ __align__(16) double cs_smem[];
  __shared__ __align__(8) uint64_t s_bar[2];  // the copies of the steps with t even, odd
  double* sC0 = cs_smem;                 // two column blocks
  double* v = sC0 + 2 * kCBlk;           // the reflector
  double* pd = v + kSMaxW;               // tau B(R, R) v, then K
  double* zb = pd + kSMaxW;              // the bulge columns' dot products, k < 32 and k >= 32
  double* zl = zb + 2 * kSMaxW;          // the rows below's
  double* pq = zl + 2 * kSMaxW;          // B(R, R) v over the four quarters of k
  uint16_t* tri = reinterpret_cast<uint16_t*>(pq + 4 * kSMaxW);  // (i, k) of the packed index q at len = w
  __shared__ double s_tau, s_beta, s_scal, s_sx;
  __shared__ int s_ok;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = p.n, w = p.w;
  for (int q = tid; q < w * (w + 1) / 2; q += kChaseThreads) {
    int i, k;
    tri_entry(q, w, i, k);
    tri[q] = (uint16_t)(i | (k << 8));
  }
  if (tid == 0) {
    tc::mbar_init(&s_bar[0], kChaseWarps);
    tc::mbar_init(&s_bar[1], kChaseWarps);
    tc::fence_mbar_init();
  }
  __syncthreads();
  uint32_t ph0 = 0, ph1 = 0;  // parity of the next completion of s_bar[0], s_bar[1]
  // waits for the copies of step t (all threads); false past the time limit
  auto copies_wait = [&](int t) {
    uint32_t& ph = (t & 1) ? ph1 : ph0;
    const bool ok = tc::mbar_wait(&s_bar[t & 1], ph, global_ns() + p.limit_ns);
    ph ^= 1u;
    return ok;
  };
  for (int c = blockIdx.x; c + 2 < n; c += gridDim.x) {
    int col = c, s = c + 1, t = 0;
    while (true) {
      const int end = min(s + w, n), len = end - s;
      if (len < 2) break;
      auto stamp = [&](int q, int who = 0) {
        if (p.phases && c == p.phase_sweep && tid == who && t < p.phase_steps) p.phases[t * kPhaseSlots + q] = clock64();
      };
      stamp(0);
      if (tid == 0) {
        int ok = 1;
        if (c > 0) {
          unsigned long long t0 = 0;
          unsigned int spins = 0;
          while (ld_acquire_int(&p.prog[c - 1]) < t + 2) {
            if ((++spins & 63u) == 0u) {
              const unsigned long long now = global_ns();
              if (t0 == 0) t0 = now;
              else if (now - t0 > p.limit_ns) {
                if (p.status) atomicCAS(p.status, 0, BANDRED_DEV_TIMEOUT);
                ok = 0;
                break;
              }
              if (p.status && ld_acquire_int(p.status) != 0) { ok = 0; break; }
            }
          }
        }
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok) return;  // (no copies are in flight between steps)
      stamp(1);
      // nb = s - col - 1 bulge columns (0 at t = 0, else w - 1); nl rows below, which is
      // the next step's len: the step after this one runs iff nl >= 2
      const int nb = s - col - 1, nl = min(end + w, n) - end;
      const bool next = nl >= 2;
      double* Cc = sC0 + (size_t)(t & 1) * kCBlk;  // this step's blocks
      // the step before's: its rows below (laid out for len = w) hold x in column 0 and
      // bulge column j in column 1 + j, row i at kC k + w + i
      double* Cp = sC0 + (size_t)((t + 1) & 1) * kCBlk;
      const float rlen = 1.0f / (float)len;
      // this step's blocks, all final now: the sweep before has finished its step t + 1
      // and written its step t + 2's column
      const double x0 = (t == 0 && tid < len) ? ldb(p, s + tid, col) : 0.0;
      chase_issue(p, s, len, nl, Cc, &s_bar[t & 1], warp, lane);
      if (t == 0) {
        // a sweep's first column and reflector; each later one is formed, and its column
        // written, by the step before as soon as that step's right application is done
        if (tid < len) Cp[w + tid] = x0;
        __syncthreads();
        if (warp == 0) chase_reflector(Cp + w, len, lane, &s_tau, &s_beta, &s_scal, &s_sx);
        __syncthreads();
        for (int i = tid; i < len; i += kChaseThreads) stb(p, s + i, col, i == 0 ? s_beta : 0.0);
      }
      const double tau = s_tau;
      if (tid < len) v[tid] = tid == 0 ? 1.0 : (Cp[w + tid] * s_sx) * s_scal;
      if (!__syncthreads_and(copies_wait(t))) {
        if (tid == 0 && p.status) atomicCAS(p.status, 0, BANDRED_DEV_TIMEOUT);
        tc::mbar_wait(&s_bar[t & 1], ((t & 1) ? ph1 : ph0) ^ 1u, global_ns() + p.limit_ns);  // still in flight
        return;
      }
      stamp(2);
      stamp(5);
      // the bulge columns (their final values) and, when no step follows, the rows below
      // go to global memory; the rows below otherwise stay for the next step
      // the next step's reflector, from its column (the first of the rows below, final
      // once this step's right application is done), and that column written as
      // (beta, 0, ..): the one entry of the next step that the sweep after needs before it
      // may start its step t - 1 (warp 1)
      auto next_column = [&]() {
        chase_reflector(Cc + len, nl, lane, &s_tau, &s_beta, &s_scal, &s_sx);
        __syncwarp();
        for (int i = lane; i < nl; i += 32) stb(p, end + i, s, i == 0 ? s_beta : 0.0);
      };
      auto write_back = [&](int t0, int nt) {
        for (int q = t0; q < nb * len; q += nt) {
          const int j = fdiv(q, len, rlen), i = q - j * len;
          stb(p, s + i, col + 1 + j, Cp[(size_t)kC * (1 + j) + w + i]);
        }
        if (nl == 1) {
          for (int k = t0; k < len; k += nt) stb(p, end, s + k, Cc[(size_t)kC * k + len]);
        }
      };
      if (tau != 0.0) {
        // phase A in two halves around a barrier, with the same FP64 work for every warp
        // (some 86 instructions at len = 64), whichever warps share an SM sub-partition.
        // Warp g takes the vector job g & 3 (bulge columns 0..31, 32..63, rows below
        // 0..31, 32..63) over k in [32 (g >> 2), 32 (g >> 2) + 32), and rows 32 (g & 1) +
        // lane of B(R, R) v over k in [16 (g >> 1), 16 (g >> 1) + 16) (the lower triangle
        // read across the diagonal).  First the partial dot products; then, with the two
        // halves summed, the updates of the same entries, held in registers in between.
        const int job = warp & 3, kh = warp >> 2, k0 = 32 * kh;
        const bool bulge = job < 2;
        const int q = 32 * (job & 1) + lane;  // the bulge column or the row below
        const bool have = bulge ? q < nb : q < nl;
        double* b = bulge ? Cp + (size_t)kC * (1 + q) + w + k0 : Cc + len + q + (size_t)kC * k0;
        const int st = bulge ? 1 : kC;
        double* zs = bulge ? zb : zl;
        double y[32];
        if (have) zs[kSMaxW * kh + q] = half_load_dot(b, st, v, k0, len, y);
        {
          const int i = 32 * (warp & 1) + lane, kq = warp >> 1;
          if (i < len) {
            double y0 = 0.0, y1 = 0.0;
#pragma unroll
            for (int kk = 0; kk < 16; kk += 2) {
              const int k = 16 * kq + kk;
              if (k < len) y0 = fma(Cc[k <= i ? kC * k + i : kC * i + k], v[k], y0);
              if (k + 1 < len) y1 = fma(Cc[k + 1 <= i ? kC * (k + 1) + i : kC * i + k + 1], v[k + 1], y1);
            }
            pq[kSMaxW * kq + i] = y0 + y1;
          }
        }
        __syncthreads();
        stamp(10);
        if (have) half_update(b, st, v, k0, len, tau * (zs[q] + zs[kSMaxW + q]), y);
        __syncthreads();
        stamp(6);
        // warp 0 forms p = tau B(R, R) v and K = p - (tau/2)(p.v) v, warp 1 the next step's
        // reflector, and the others write back
        if (tid < 32) {
          double y[kSMaxW / 32], pv = 0.0;
#pragma unroll
          for (int u = 0; u < kSMaxW / 32; ++u) {
            const int i = lane + 32 * u;
            y[u] = i < len ? tau * ((pq[i] + pq[kSMaxW + i]) + (pq[2 * kSMaxW + i] + pq[3 * kSMaxW + i])) : 0.0;
            pv = fma(y[u], i < len ? v[i] : 0.0, pv);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) pv += __shfl_xor_sync(0xffffffffu, pv, o);
          const double half = 0.5 * tau * pv;
#pragma unroll
          for (int u = 0; u < kSMaxW / 32; ++u) {
            const int i = lane + 32 * u;
            if (i < len) pd[i] = fma(-half, v[i], y[u]);
          }
        } else if (next && warp == 1) {
          next_column();
        } else {
          const int w0 = next ? 64 : 32;
          write_back(tid - w0, kChaseThreads - w0);
        }
        __syncthreads();
        stamp(7);
        // the diagonal block's rank-2 update over the packed lower triangle only (each FP64
        // warp instruction costs the same whatever the number of active lanes), column by
        // column (index q = off(k) + i - k, off(k) = k len - k (k - 1) / 2, so that a warp's
        // stores are contiguous); a thread forms all its entries before it stores any, so
        // that their FP64 chains overlap
        {
          constexpr int kPer = (kSMaxW * (kSMaxW + 1) / 2 + kChaseThreads - 1) / kChaseThreads;
          const int nq = len * (len + 1) / 2;
          double r[kPer];
          int ri[kPer], rk[kPer];
#pragma unroll
          for (int u = 0; u < kPer; ++u) {
            const int q = tid + u * kChaseThreads < nq ? tid + u * kChaseThreads : 0;
            int i, k;
            if (len == w) {  // every step but a sweep's last: the table
              i = tri[q] & 255;
              k = tri[q] >> 8;
            } else {
              tri_entry(q, len, i, k);
            }
            ri[u] = i;
            rk[u] = k;
            r[u] = fma(-v[i], pd[k], fma(-pd[i], v[k], Cc[kC * k + i]));
          }
          stamp(11);
#pragma unroll
          for (int u = 0; u < kPer; ++u) {
            if (tid + u * kChaseThreads < nq) stb(p, s + ri[u], s + rk[u], r[u]);
          }
        }
        stamp(8);
      } else {
        if (next && warp == 1) {
          next_column();
        } else {
          const int w0 = next ? 32 : 0;
          write_back(tid - (warp > 1 ? w0 : 0), kChaseThreads - w0);
        }
      }
      tc::fence_proxy_async();  // this step's shared-memory accesses before the copies that reuse the buffers
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release_int(&p.prog[c], t + 1);
      }
      stamp(9);
      col = s;
      s += w;
      ++t;
    }
    if (tid == 0) {
      __threadfence();
      st_release_int(&p.prog[c], kDone);
    }
  }
}

// Band store from the packed sy2sb output: offsets 0 .. w from A's lower band, zeros
// above (the bulge rows).
__global__ void band_in_kernel(int n, int w, int LB, const double* A, int64_t lda, double* Bs) {
  const int64_t total = (int64_t)n * LB;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int off = (int)(q % LB), k = (int)(q / LB), i = k + off;
    Bs[q] = (off <= w && i < n) ? A[i + (int64_t)k * lda] : 0.0;
  }
}

__global__ void band_out_kernel(int n, int LB, const double* Bs, double* d, double* e) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    d[k] = Bs[(int64_t)k * LB];
    if (k + 1 < n) e[k] = Bs[1 + (int64_t)k * LB];
  }
}

}  // namespace

namespace {

// ---------------------------------------------------------------- eigenvalues
// Gershgorin interval [gl, gu], the stopping width and the pivot guard of the trisection,
// and e^2 (one CTA): prm = {gl, gu, tol, pivmin}.
constexpr int kGThreads = 256;
// Also the scale sc = 2^-k with max |T| sc in [1/2, 1) (prm[4]) and the scaled copy of T in
// FP32 for the first pass: d32 = d sc, e32 = e^2 sc^2.
__global__ void sterf_setup_kernel(int n, const double* d, const double* e, double* e2, double* prm, float* d32,
                                   float* e32) {
  __shared__ double s_lo[kGThreads], s_hi[kGThreads], s_mx[kGThreads], s_e2[kGThreads];
  pdl_wait_and_release();
  const int tid = threadIdx.x;
  double lo = 1e300, hi = -1e300, mx = 0.0, em = 0.0;
  for (int i = tid; i < n; i += kGThreads) {
    const double el = i > 0 ? fabs(e[i - 1]) : 0.0, er = i + 1 < n ? fabs(e[i]) : 0.0;
    lo = fmin(lo, d[i] - (el + er));
    hi = fmax(hi, d[i] + (el + er));
    mx = fmax(mx, fmax(fabs(d[i]), er));
    if (i + 1 < n) {
      const double q = e[i] * e[i];
      e2[i] = q;
      em = fmax(em, q);
    }
  }
  s_lo[tid] = lo;
  s_hi[tid] = hi;
  s_mx[tid] = mx;
  s_e2[tid] = em;
  __syncthreads();
  for (int h = kGThreads / 2; h > 0; h >>= 1) {
    if (tid < h) {
      s_lo[tid] = fmin(s_lo[tid], s_lo[tid + h]);
      s_hi[tid] = fmax(s_hi[tid], s_hi[tid + h]);
      s_mx[tid] = fmax(s_mx[tid], s_mx[tid + h]);
      s_e2[tid] = fmax(s_e2[tid], s_e2[tid + h]);
    }
    __syncthreads();
  }
  if (tid == 0) {
    const double tol = 4.0 * 0x1p-53 * (s_mx[0] > 0.0 ? s_mx[0] : 1.0);
    prm[0] = s_lo[0] - tol;
    prm[1] = s_hi[0] + tol;
    prm[2] = tol;
    prm[3] = fmax(s_e2[0], 1.0) * 0x1p-1020;
    int k = 0;
    if (s_mx[0] > 0.0) frexp(s_mx[0], &k);
    prm[4] = ldexp(1.0, -k);
  }
  __syncthreads();
  const double sc = prm[4];
  for (int i = tid; i < n; i += kGThreads) {
    d32[i] = (float)(d[i] * sc);
    if (i + 1 < n) e32[i] = (float)((e2[i] * sc) * sc);
  }
}

// Sturm count of the scaled FP32 copy of T at x (entries below 1 in magnitude; the pivot
// guard 2^-100), FP32 arithmetic throughout: a quick first pass, whose counts are exact
// for a matrix within about 7 units of FP32 roundoff of max |T| (the recurrence's backward
// error, with the rounding of the copy itself).
__device__ __forceinline__ int sturm_count32(int n, const float* d, const float* e2, float x) {
  constexpr float kPiv = 0x1p-100f;
  float q = d[0] - x;
  if (fabsf(q) < kPiv) q = -kPiv;
  int neg = q < 0.0f;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - e2[i - 1] * __frcp_rn(q);
    if (fabsf(q) < kPiv) q = -kPiv;
    neg += q < 0.0f;
  }
  return neg;
}

// 1/s for a normal s > 0: an FP32 seed r0 of the mantissa m, then one cubic Newton step
// r = r0 (1 + d + d^2), d = 1 - m r0 (|d| < 2^-22, so the dropped d^3 term is below
// 2^-66): three dependent FP64 operations, a unit or so in the last place
__device__ __forceinline__ double rcp_cubic(double s) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(s);
  const int e = (int)((u >> 52) & 0x7FF) - 1023;
  const double m = __longlong_as_double((long long)((u & 0x000FFFFFFFFFFFFFull) | (1023ull << 52)));
  const float mf = __uint_as_float((127u << 23) | (uint32_t)((u >> 29) & 0x7FFFFFu));
  const double r0 = tc::f32_to_f64(__frcp_rn(mf));
  const double dd = fma(-m, r0, 1.0);
  const double r = fma(r0, fma(dd, dd, dd), r0);
  return __longlong_as_double(__double_as_longlong(r) - ((long long)e << 52));
}

// Sturm count of T at x: the sequence q_0 = d_0 - x, q_i = d_i - x - e_{i-1}^2 / q_{i-1}
// has as many negative terms as T has eigenvalues below x (a term below the pivot guard
// counts as -pivmin).  One step costs five FP64 operations (rcp_cubic's three, d_i - x,
// and the FMA), well inside the recurrence's own backward error; the pivot guard and the
// sign test are integer compares of the bit patterns.
__device__ __forceinline__ int sturm_count(int n, const double* d, const double* e2, double x, double pivmin) {
  const long long piv = dbits(pivmin);
  const double npiv = -pivmin;
  double q = d[0] - x;
  if (abits(q) < piv) q = npiv;
  int neg = dbits(q) < 0;
  for (int i = 1; i < n; ++i) {
    const double r = neg_if(rcp_cubic(__longlong_as_double(abits(q))), dbits(q) < 0);
    q = fma(-e2[i - 1], r, d[i] - x);
    if (abits(q) < piv) q = npiv;
    neg += dbits(q) < 0;
  }
  return neg;
}

// Eigenvalue k of T by trisection on Sturm counts.  Two lanes per eigenvalue: each round
// the pair counts at the two points that cut [lo, hi) into thirds, one point per lane, and
// both lanes keep the third that holds eigenvalue k.  The bracket shrinks threefold per
// round from the same Gershgorin interval for every eigenvalue, so all pairs run the same
// number of rounds (no divergence).  The Sturm chain is bound by GB300's FP64 throughput
// (a single chain already keeps a sub-partition's FP64 pipe busy; four points per
// eigenvalue and round, two chains per lane, were measured slower): two lanes per
// eigenvalue give twice the warps of bisection (512 at n = 8192, for 608 sub-partitions)
// at a third fewer sequential rounds.
// Eigenvalues k0 .. k0 + count - 1 (ascending) into lam[0 .. count).
__global__ void sterf_trisect_kernel(int n, const double* d, const double* e2, const double* prm, double* lam,
                                     int k0, int count, const float* d32, const float* e32) {
  pdl_wait_and_release();
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = k0 + min(g >> 1, count - 1), half = g & 1;
  const double tol = prm[2], pivmin = prm[3], sc = prm[4];
  double lo = prm[0], hi = prm[1];
  // First pass in FP32 on T sc (max |T sc| in [1/2, 1)), by the same trisection, down to a
  // width of 2^-14; the bracket then widens by 2^-16 on each side, far beyond the FP32
  // pass's error (about 7 x 2^-24), and the FP64 rounds start from there.
  {
    float lo32 = (float)(lo * sc), hi32 = (float)(hi * sc);
    int r32 = 0;
    for (double wd = (double)hi32 - (double)lo32; wd > 0x1p-14 && r32 < 60; wd *= (1.0 / 3.0)) ++r32;
    for (int it = 0; it < r32; ++it) {
      const float h = (hi32 - lo32) * (1.0f / 3.0f);
      const float x1 = lo32 + h, x2 = hi32 - h;
      const int c = sturm_count32(n, d32, e32, half ? x2 : x1);
      const int c1 = __shfl_xor_sync(0xffffffffu, c, 1);
      const int ca = half ? c1 : c, cb = half ? c : c1;
      if (ca > k) {
        hi32 = x1;
      } else if (cb > k) {
        lo32 = x1;
        hi32 = x2;
      } else {
        lo32 = x2;
      }
    }
    const double m = 0x1p-16 / sc;
    lo = fmax(prm[0], (double)lo32 / sc - m);
    hi = fmin(prm[1], (double)hi32 / sc + m);
  }
  // FP64 rounds until the width falls to tol, from the widest bracket the first pass can
  // leave: the same for every pair
  int rounds = 0;
  const double w0 = fmin(prm[1] - prm[0], (0x1p-14 * 1.001 + 0x1p-15) / sc);
  for (double wd = w0; wd > tol && rounds < 120; wd *= (1.0 / 3.0)) ++rounds;
  for (int it = 0; it < rounds; ++it) {
    const double h = (hi - lo) * (1.0 / 3.0);
    const double x1 = lo + h, x2 = hi - h;
    const int c = sturm_count(n, d, e2, half ? x2 : x1, pivmin);
    const int c1 = __shfl_xor_sync(0xffffffffu, c, 1);
    const int ca = half ? c1 : c, cb = half ? c : c1;  // counts at x1, x2
    if (ca > k) {
      hi = x1;
    } else if (cb > k) {
      lo = x1;
      hi = x2;
    } else {
      lo = x2;
    }
  }
  if (!half && (g >> 1) < count) lam[k - k0] = 0.5 * (lo + hi);
}

struct Sb2stWs {
  double* Bs;
  int* prog;
  int* status;
  size_t bytes;
};

Sb2stWs carve_sb2st(void* work, int64_t n, int64_t w) {
  char* base = static_cast<char*>(work);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = base ? base + off : nullptr;
    off += (bytes + 255) / 256 * 256;
    return q;
  };
  Sb2stWs ws{};
  ws.Bs = reinterpret_cast<double*>(take(sizeof(double) * (size_t)std::max<int64_t>(n, 1) * 2 * w));
  ws.prog = reinterpret_cast<int*>(take(sizeof(int) * (size_t)std::max<int64_t>(n, 1)));
  ws.status = reinterpret_cast<int*>(take(256));
  ws.bytes = off;
  return ws;
}

}  // namespace

size_t sb2st_workspace_bytes(int64_t n, int64_t w) { return carve_sb2st(nullptr, n, w).bytes; }

size_t sterf_workspace_bytes(int64_t n) {
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  return (sizeof(double) * nn + 255) / 256 * 256 + 256 + 2 * ((sizeof(float) * nn + 255) / 256 * 256);
}

#define CKS(call)                                                 \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return record_cuda_error(e_, #call);   \
  } while (0)

int sb2st_run(int64_t n, int64_t w, const double* A, int64_t lda, double* d, double* e, unsigned long long limit_ns,
              void* work, int* dev_status, cudaStream_t s) {
  Sb2stWs ws = carve_sb2st(work, n, w);
  int* status = dev_status ? dev_status : ws.status;
  CKS(cudaMemsetAsync(status, 0, sizeof(int), s));
  if (n <= 0) return 0;
  const int LB = (int)(2 * w);
  {
    const int blocks = (int)std::min<int64_t>((n * LB + 255) / 256, 4096);
    prof::count_launch();
    band_in_kernel<<<blocks, 256, 0, s>>>((int)n, (int)w, LB, A, lda, ws.Bs);
    CKS(cudaGetLastError());
  }
  if (n > 2 && w > 1) {
    CKS(cudaMemsetAsync(ws.prog, 0, sizeof(int) * (size_t)n, s));
    int dev = 0, sms = 0;
    CKS(cudaGetDevice(&dev));
    CKS(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // one CTA per SM (each sweep's FP64 work keeps its SM's FP64 units busy), all
    // co-resident: the cooperative launch guarantees it
    const int G = (int)std::min<int64_t>(n - 2, sms);
    ChaseParams p{(int)n, (int)w, LB, ws.Bs, ws.prog, status, limit_ns, nullptr, 0, 0};
    p.phases = prof::chase_phase_take(&p.phase_steps);
    p.phase_sweep = (int)((n - 2) / 2);
    void* args[] = {&p};
    prof::count_launch();
    if (w <= kSMaxW) {
      static int configured = -1;
      if (configured != dev) {
        CKS(cudaFuncSetAttribute(sb2st_chase_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemChase));
        configured = dev;
      }
      CKS(cudaLaunchCooperativeKernel((const void*)sb2st_chase_smem_kernel, dim3(G), dim3(kChaseThreads), args,
                                      kSmemChase, s));
    } else {
      CKS(cudaLaunchCooperativeKernel((const void*)sb2st_chase_kernel, dim3(G), dim3(kChaseThreads), args, 0, s));
    }
  }
  {
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
    prof::count_launch();
    band_out_kernel<<<blocks, 256, 0, s>>>((int)n, LB, ws.Bs, d, e);
    CKS(cudaGetLastError());
  }
  return 0;
}

int sterf_run(int64_t n, const double* d, const double* e, double* lam, void* work, cudaStream_t s) {
  return sterf_range_run(n, d, e, lam, 0, n, work, s);
}

int sterf_range_run(int64_t n, const double* d, const double* e, double* lam, int64_t k0, int64_t count, void* work,
                    cudaStream_t s) {
  if (n <= 0 || count <= 0) return 0;
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  char* base = static_cast<char*>(work);
  double* e2 = reinterpret_cast<double*>(base);
  double* prm = reinterpret_cast<double*>(base + (sizeof(double) * nn + 255) / 256 * 256);
  float* d32 = reinterpret_cast<float*>(reinterpret_cast<char*>(prm) + 256);
  float* e32 = reinterpret_cast<float*>(reinterpret_cast<char*>(d32) + (sizeof(float) * nn + 255) / 256 * 256);
  prof::count_launch();
  CKS(launch_pdl(sterf_setup_kernel, dim3(1), dim3(kGThreads), 0, s, (int)n, d, e, e2, prm, d32, e32));
  prof::count_launch();
  CKS(launch_pdl(sterf_trisect_kernel, dim3((unsigned)((2 * count + 63) / 64)), dim3(64), 0, s, (int)n, d,
                 static_cast<const double*>(e2), static_cast<const double*>(prm), lam, (int)k0, (int)count,
                 static_cast<const float*>(d32), static_cast<const float*>(e32)));
  return 0;
}

}  // namespace bandred
