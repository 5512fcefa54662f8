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
// 8 MB).  One persistent cooperative kernel: CTA g runs sweeps g, g + G, ... in order.
// A step of sweep c with range start s writes only entries whose column index lies in
// [s - w, s + w) (the annihilated column, the bulge columns, the range), and step t'' of
// sweep c - 1 only entries whose column index is at least its own s'' - w = s - 1 +
// (t'' - t - 1) w.  They share entries only for t'' <= t + 2, so step t of sweep c waits
// until sweep c - 1 has finished its step t + 2: every entry sees the sweeps' updates in
// sequential order, and the result equals the one-sweep-at-a-time algorithm up to the
// rounding of the sums.  The
// waits are bounded: past the time limit the kernel records BANDRED_DEV_TIMEOUT and
// returns.  Within a step the three blocks the reflector touches (the bulge columns to
// the left of the range, the symmetric diagonal block, the rows below the range) are
// independent vectors, one warp each at a time.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "driver.h"
#include "panel_common.cuh"
#include "kernels.h"
#include "launch.h"
#include "prof.h"

namespace bandred {
namespace {

constexpr int kChaseThreads = 256;
constexpr int kMaxW = 128;  // reflector length <= w <= 128: four entries per lane
constexpr int kDone = 1 << 30;

struct ChaseParams {
  int n, w, LB;       // LB = 2w: rows of the band store per column
  double* Bs;         // entry (i, k), 0 <= i - k < LB, at Bs[(i - k) + k * LB]
  int* prog;          // prog[c]: steps sweep c has finished (kDone when finished)
  int* status;
  unsigned long long limit_ns;
  long long* phases;  // diagnostic: clock64 at 8 points of each step of sweep phase_sweep, or nullptr
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
  __shared__ double s_tau, s_beta, s_scal, s_half;
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
        double ss = 0.0;
        if (amax > 0.0) {
          const double inv = 1.0 / amax;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = lane + 32 * u;
            if (i >= 1 && i < len) {
              const double q = xv[u] * inv;
              ss = fma(q, q, ss);
            }
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) {
          const double alpha = xv[0];
          double tau = 0.0, beta = alpha, scal = 1.0;
          if (amax > 0.0) {
            const double xnorm = amax * sqrt(ss);
            const double h = hypot(alpha, xnorm);
            beta = alpha >= 0.0 ? -h : h;
            tau = (beta - alpha) / beta;
            scal = 1.0 / (alpha - beta);
          }
          s_tau = tau;
          s_beta = beta;
          s_scal = scal;
        }
      }
      __syncthreads();
      const double tau = s_tau;
      // v = [1; x2 scal]; the column becomes [beta; 0 ...]
      for (int i = tid; i < len; i += kChaseThreads) {
        stb(p, s + i, col, i == 0 ? s_beta : 0.0);
      }
      __syncthreads();
      if (tid < len) v[tid] = tid == 0 ? 1.0 : v[tid] * s_scal;
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
// sweep before has finished with them, the sweep after waits for step t + 1).  So they
// stay in shared memory and reach global memory once, as step t + 1's bulge columns.
//
// Prefetch.  Step t + 1's own blocks (its diagonal block and the rows below it) have
// column indices from end on, which step t does not write; of the sweep before, only
// its step t + 3 writes any of them (column end + w - 1 at rows from end + 2w - 1, the
// last column of the rows below).  So step t issues their loads into registers as soon
// as its own wait is over, parks them in shared memory after its phase A, and step
// t + 1 reloads the last column of its rows below after its wait.
//
// Buffers: two diagonal blocks (lower triangle, (i, k) at k * kSLd + i) and three
// rows-below blocks ((r, k) at r * kSLd + k) used in turn: this step's, the carried one
// of the step before, and the next step's.  A thread per row and a thread per carried
// column both see stride-1 or stride-65 addresses, free of bank conflicts.
constexpr int kSMaxW = 64;
constexpr int kSLd = kSMaxW + 1;
constexpr size_t kSBlk = (size_t)kSMaxW * kSLd;
constexpr size_t kSmemChase = sizeof(double) * (5 * kSBlk + 4 * kSMaxW);
constexpr int kSPer = kSMaxW * kSMaxW / kChaseThreads;  // block entries per thread
static_assert(kChaseThreads == 4 * kSMaxW, "phase A gives 64 threads to each of four jobs");

__global__ void __launch_bounds__(kChaseThreads) sb2st_chase_smem_kernel(ChaseParams p) {
  extern __shared__ double cs_smem[];
  double* sD0 = cs_smem;                 // two diagonal blocks
  double* sL0 = sD0 + 2 * kSBlk;         // three blocks of rows below
  double* v = sL0 + 3 * kSBlk;           // the reflector
  double* pd = v + kSMaxW;               // tau B(R, R) v, then K
  double* pa = pd + kSMaxW;              // B(R, R) v over the first and second half of k
  double* pb = pa + kSMaxW;
  __shared__ double s_tau, s_beta, s_scal, s_half;
  __shared__ int s_ok;
  const int tid = threadIdx.x, lane = tid & 31;
  const int n = p.n, w = p.w;
  double rd[kSPer], rl[kSPer];  // one step's blocks on their way to shared memory
  // loads of the blocks of the step with range [sx, sx + lx) and nx rows below
  auto fetch = [&](int sx, int lx, int nx) {
    const float rx = 1.0f / (float)lx, ry = nx > 0 ? 1.0f / (float)nx : 0.0f;
#pragma unroll
    for (int u = 0; u < kSPer; ++u) {
      const int q = tid + u * kChaseThreads;
      const int j = fdiv(q, lx, rx), i = q - j * lx;
      rd[u] = (q < lx * lx && i >= j) ? ldb(p, sx + i, sx + j) : 0.0;
      const int kl = nx > 0 ? fdiv(q, nx, ry) : 0, r = nx > 0 ? q - kl * nx : 0;
      rl[u] = (nx > 0 && q < nx * lx) ? ldb(p, sx + lx + r, sx + kl) : 0.0;
    }
  };
  auto park = [&](double* D, double* L, int lx, int nx) {
    const float rx = 1.0f / (float)lx, ry = nx > 0 ? 1.0f / (float)nx : 0.0f;
#pragma unroll
    for (int u = 0; u < kSPer; ++u) {
      const int q = tid + u * kChaseThreads;
      const int j = fdiv(q, lx, rx), i = q - j * lx;
      if (q < lx * lx && i >= j) D[j * kSLd + i] = rd[u];
      if (nx > 0 && q < nx * lx) {
        const int kl = fdiv(q, nx, ry), r = q - kl * nx;
        L[r * kSLd + kl] = rl[u];
      }
    }
  };
  for (int c = blockIdx.x; c + 2 < n; c += gridDim.x) {
    int col = c, s = c + 1, t = 0, li = 0;  // li = t mod 3
    while (true) {
      const int end = min(s + w, n), len = end - s;
      if (len < 2) break;
      auto stamp = [&](int q) {
        if (p.phases && c == p.phase_sweep && tid == 0 && t < p.phase_steps) p.phases[t * 8 + q] = clock64();
      };
      stamp(0);
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
      stamp(1);
      // nb = s - col - 1 bulge columns (0 at t = 0, else w - 1); nl rows below, which is
      // the next step's len: the step after this one runs iff nl >= 2
      const int nb = s - col - 1, nl = min(end + w, n) - end;
      const bool next = nl >= 2;
      const int nl1 = next ? min(end + nl + w, n) - (end + nl) : 0;  // the next step's rows below
      double* Dc = sD0 + (size_t)(t & 1) * kSBlk;
      double* Dn = sD0 + (size_t)((t + 1) & 1) * kSBlk;
      double* Lc = sL0 + (size_t)li * kSBlk;                         // this step's rows below
      double* Ln = sL0 + (size_t)(li == 2 ? 0 : li + 1) * kSBlk;     // the next step's
      double* Lp = sL0 + (size_t)(li == 0 ? 2 : li - 1) * kSBlk;     // carried: x at (i, 0), bulge column j at (i, 1 + j)
      const float rlen = 1.0f / (float)len;
      if (t == 0) {  // this step's blocks and the column, from global memory
        const double xs = tid < len ? ldb(p, s + tid, col) : 0.0;
        fetch(s, len, nl);
        if (tid < len) Lp[tid * kSLd] = xs;
        park(Dc, Lc, len, nl);
        if (next) fetch(end, nl, nl1);
        __syncthreads();
      } else {
        // the last column of the rows below, which the sweep before could write until
        // this step's wait; then the next step's blocks
        const int r = tid - 32;
        const double xr = (r >= 0 && r < nl) ? ldb(p, end + r, end - 1) : 0.0;
        if (next) fetch(end, nl, nl1);
        if (r >= 0 && r < nl) Lc[r * kSLd + len - 1] = xr;
      }
      stamp(2);
      // the reflector (warp 0), larfg convention.  Common path: the plain sum of squares
      // when it and |alpha| are safely in range (max |x2| from the bit patterns, integer
      // compares), then h = ||x|| = q / sqrt(q), tau = 1 + |alpha| / h and
      // 1 / (alpha - beta) by Newton-Raphson; otherwise the max-scaled sum and hypot.
      if (tid < 32) {
        unsigned long long um = 0ull;
        double ss = 0.0;
        for (int i = 1 + lane; i < len; i += 32) {
          const double x = Lp[i * kSLd];
          const unsigned long long u = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
          um = u > um ? u : um;
          ss = fma(x, x, ss);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const unsigned long long u = __shfl_xor_sync(0xffffffffu, um, o);
          um = u > um ? u : um;
          ss += __shfl_xor_sync(0xffffffffu, ss, o);
        }
        const double amax = __longlong_as_double((long long)um), alpha = Lp[0];
        const bool plain = amax > 0x1p-450 && ss < 0x1p1000 && fabs(alpha) < 0x1p500;
        if (amax > 0.0 && !plain) {  // rare: scaled sum (warp-uniform branch)
          const double inv = 1.0 / amax;
          ss = 0.0;
          for (int i = 1 + lane; i < len; i += 32) {
            const double q = Lp[i * kSLd] * inv;
            ss = fma(q, q, ss);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        }
        if (lane == 0) {
          double tau = 0.0, beta = alpha, scal = 1.0;
          if (amax > 0.0) {
            if (plain) {
              const double q = fma(alpha, alpha, ss);
              const double rq = panel_detail::rsqrt_newton(q);
              const double h = q * rq, aa = fabs(alpha);
              beta = alpha >= 0.0 ? -h : h;
              tau = fma(aa, rq, 1.0);
              const double rs = panel_detail::rcp_newton(aa + h);
              scal = alpha >= 0.0 ? rs : -rs;
            } else {
              const double h = hypot(alpha, amax * sqrt(ss));
              beta = alpha >= 0.0 ? -h : h;
              tau = (beta - alpha) / beta;
              scal = 1.0 / (alpha - beta);
            }
          }
          s_tau = tau;
          s_beta = beta;
          s_scal = scal;
        }
      }
      __syncthreads();
      const double tau = s_tau;
      stamp(3);
      if (tid < len) v[tid] = tid == 0 ? 1.0 : Lp[tid * kSLd] * s_scal;
      for (int i = tid; i < len; i += kChaseThreads) stb(p, s + i, col, i == 0 ? s_beta : 0.0);
      __syncthreads();
      // the bulge columns (their final values) and, when no step follows, the rows below
      // go to global memory; the rows below otherwise stay for the next step
      auto write_back = [&](int t0, int nt) {
        for (int q = t0; q < nb * len; q += nt) {
          const int j = fdiv(q, len, rlen), i = q - j * len;
          stb(p, s + i, col + 1 + j, Lp[i * kSLd + 1 + j]);
        }
        if (nl == 1) {
          for (int k = t0; k < len; k += nt) stb(p, end, s + k, Lc[k]);
        }
      };
      // x -= z v over len entries at stride ld (a bulge column or a row below), eight at a
      // time so that the loads are not held behind the stores
      auto axpy = [&](double* b, int ld, double z) {
        for (int i0 = 0; i0 < len; i0 += 8) {
          double bb[8], vv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int i = min(i0 + u, len - 1);
            bb[u] = b[i * ld];
            vv[u] = v[i];
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            if (i0 + u < len) b[(i0 + u) * ld] = fma(-z, vv[u], bb[u]);
          }
        }
      };
      auto dot = [&](const double* b, int ld) {
        double z0 = 0.0, z1 = 0.0;
        int i = 0;
        for (; i + 1 < len; i += 2) {
          z0 = fma(v[i], b[i * ld], z0);
          z1 = fma(v[i + 1], b[(i + 1) * ld], z1);
        }
        if (i < len) z0 = fma(v[i], b[i * ld], z0);
        return z0 + z1;
      };
      if (tau != 0.0) {
        // phase A, one thread per vector, 64 threads per job so that each SM sub-partition
        // (warp % 4) gets the same FP64 work: threads 0..63 the bulge columns (left
        // application), 64..127 the rows below (right application), 128..255 the rows of
        // B(R, R) v over the first and the second half of k (the lower triangle read
        // across the diagonal)
        if (tid < kSMaxW) {
          if (tid < nb) {
            double* b = Lp + 1 + tid;
            axpy(b, kSLd, tau * dot(b, kSLd));
          }
        } else if (tid < 2 * kSMaxW) {
          if (tid - kSMaxW < nl) {
            double* b = Lc + (tid - kSMaxW) * kSLd;
            axpy(b, 1, tau * dot(b, 1));
          }
        } else {
          const int h = tid >= 3 * kSMaxW, i = tid - 2 * kSMaxW - h * kSMaxW;
          if (i < len) {
            const int k1 = h ? len : len / 2;
            double y0 = 0.0, y1 = 0.0;
            int k = h ? len / 2 : 0;
            for (; k + 1 < k1; k += 2) {
              y0 = fma(Dc[k <= i ? k * kSLd + i : i * kSLd + k], v[k], y0);
              y1 = fma(Dc[k + 1 <= i ? (k + 1) * kSLd + i : i * kSLd + k + 1], v[k + 1], y1);
            }
            if (k < k1) y0 = fma(Dc[k <= i ? k * kSLd + i : i * kSLd + k], v[k], y0);
            (h ? pb : pa)[i] = y0 + y1;
          }
        }
        __syncthreads();
        stamp(4);
        // warp 0 forms p and p.v while the others write back; then the next step's blocks
        // go to shared memory
        if (tid < 32) {
          double pv = 0.0;
          for (int i = lane; i < len; i += 32) {
            const double y = tau * (pa[i] + pb[i]);
            pd[i] = y;
            pv = fma(y, v[i], pv);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) pv += __shfl_xor_sync(0xffffffffu, pv, o);
          if (lane == 0) s_half = 0.5 * tau * pv;
        } else {
          write_back(tid - 32, kChaseThreads - 32);
        }
        if (next) park(Dn, Ln, nl, nl1);
        __syncthreads();
        if (tid < len) pd[tid] = fma(-s_half, v[tid], pd[tid]);
        __syncthreads();
        stamp(7);
        // the diagonal block's rank-2 update over the packed lower triangle only (each FP64
        // warp instruction costs the same whatever the number of active lanes), row-major
        // index q = i (i + 1) / 2 + k, written straight back
        for (int q = tid; q < len * (len + 1) / 2; q += kChaseThreads) {
          int i = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
          while (i * (i + 1) / 2 > q) --i;
          while ((i + 1) * (i + 2) / 2 <= q) ++i;
          const int k = q - i * (i + 1) / 2;
          stb(p, s + i, s + k, fma(-v[i], pd[k], fma(-pd[i], v[k], Dc[k * kSLd + i])));
        }
        stamp(5);
      } else {
        write_back(tid, kChaseThreads);
        if (next) park(Dn, Ln, nl, nl1);
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release_int(&p.prog[c], t + 1);
      }
      stamp(6);
      col = s;
      s += w;
      ++t;
      li = li == 2 ? 0 : li + 1;
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
__global__ void sterf_setup_kernel(int n, const double* d, const double* e, double* e2, double* prm) {
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
  }
}

// Eigenvalue k of T by trisection on Sturm counts: the sequence q_0 = d_0 - x,
// q_i = d_i - x - e_{i-1}^2 / q_{i-1} has as many negative terms as T has eigenvalues below
// x (a term below the pivot guard counts as -pivmin).  Two lanes per eigenvalue: each
// iteration the pair counts at the two points that cut [lo, hi) into thirds, one point per
// lane, and both lanes keep the third that holds eigenvalue k.  The bracket shrinks
// threefold per iteration from the same Gershgorin interval for every eigenvalue, so all
// pairs run the same number of iterations (no divergence).  On GB300 the FP64 division
// chain is latency-bound, so two lanes per eigenvalue (twice the warps) and a third fewer
// sequential counts than bisection beat the extra count per iteration.
// One Sturm step costs a reciprocal and one FMA: 1/q by the panel's Newton-Raphson
// reciprocal (FP32 seed, two FP64 steps: a few units in the last place, well inside the
// recurrence's own backward error), the pivot guard and the sign test as integer
// compares of the bit patterns.
__device__ __forceinline__ int sturm_count(int n, const double* d, const double* e2, double x, double pivmin) {
  const long long piv = panel_detail::dbits(pivmin);
  const double npiv = -pivmin;
  int neg = 0;
  double q = d[0] - x;
  if (panel_detail::abits(q) < piv) q = npiv;
  neg += panel_detail::dbits(q) < 0;
  for (int i = 1; i < n; ++i) {
    const double aq = fabs(q);
    const double r = panel_detail::neg_if(panel_detail::rcp_newton(aq), panel_detail::dbits(q) < 0);
    q = fma(-e2[i - 1], r, d[i] - x);
    if (panel_detail::abits(q) < piv) q = npiv;
    neg += panel_detail::dbits(q) < 0;
  }
  return neg;
}

__global__ void sterf_trisect_kernel(int n, const double* d, const double* e2, const double* prm, double* lam) {
  pdl_wait_and_release();
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = min(g >> 1, n - 1), half = g & 1;
  const double tol = prm[2], pivmin = prm[3];
  double lo = prm[0], hi = prm[1];
  // iterations until the width falls to tol: the same for every pair
  int iters = 0;
  for (double wd = hi - lo; wd > tol && iters < 120; wd *= (1.0 / 3.0)) ++iters;
  for (int it = 0; it < iters; ++it) {
    const double h = (hi - lo) * (1.0 / 3.0);
    const double x = half ? hi - h : lo + h;
    const int c = sturm_count(n, d, e2, x, pivmin);
    const int c1 = __shfl_xor_sync(0xffffffffu, c, 1);
    const double x1 = lo + h, x2 = hi - h;
    const int ca = half ? c1 : c, cb = half ? c : c1;  // counts at x1, x2
    if (ca > k)
      hi = x1;
    else if (cb > k) {
      lo = x1;
      hi = x2;
    } else
      lo = x2;
  }
  if (!half && (g >> 1) < n) lam[k] = 0.5 * (lo + hi);
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

size_t sterf_workspace_bytes(int64_t n) { return (sizeof(double) * (size_t)std::max<int64_t>(n, 1) + 255) / 256 * 256 + 256; }

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
  if (n <= 0) return 0;
  double* e2 = static_cast<double*>(work);
  double* prm = reinterpret_cast<double*>(static_cast<char*>(work) +
                                          (sizeof(double) * (size_t)std::max<int64_t>(n, 1) + 255) / 256 * 256);
  prof::count_launch();
  CKS(launch_pdl(sterf_setup_kernel, dim3(1), dim3(kGThreads), 0, s, (int)n, d, e, e2, prm));
  prof::count_launch();
  CKS(launch_pdl(sterf_trisect_kernel, dim3((unsigned)((2 * n + 63) / 64)), dim3(64), 0, s, (int)n, d,
                 static_cast<const double*>(e2), static_cast<const double*>(prm), lam));
  return 0;
}

}  // namespace bandred
