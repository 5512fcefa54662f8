// Second stage for the SVD.  The paper's introduction gives the SVD's compact form as an
// upper triangular-band matrix (upper bandwidth w), which a second stage reduces to
// bidiagonal form before the singular values are computed.  Here the band goes to an
// upper bidiagonal B by Householder bulge chasing, and the singular values of B come
// from the eigenvalues of its Golub-Kahan tridiagonal (trisection on Sturm counts, the
// eigenvalue kernel of the symmetric second stage).
//
// Bulge chasing.  Sweep c (c = 0 .. n-2) alternates right and left reflectors on index
// ranges [a, a + w) that move down by w (a = c + 1 first).  The right reflector
// annihilates row r's entries past its first (r = c first, then r = the previous range's
// first row) and is applied to rows (r, a + w); on rows [a, a + w) it fills the triangle
// below their diagonal.  The left reflector annihilates column a below its diagonal and is
// applied to columns (a, a + 2w); on rows [a, a + w) it fills the entries past the band,
// whose first row the next right reflector takes.  The other rows and columns of each
// bulge are annihilated by the sweeps that follow.  Each reflector follows the larfg
// convention (beta = -sign(alpha) ||x||, sign(0) = +1; tau = 0 for a zero tail).  Those
// application ranges hold every nonzero the reflectors meet: entries never sit more than
// 2w - 1 above or w - 1 below the diagonal (measured over many shapes on a dense copy,
// and what the ranges' geometry allows).
//
// GB300 mapping.  The band lives in a compact store of 3w rows per column (offsets
// 0 .. 3w - 1 for i - j from -(2w - 1) to w), resident in L2 (n = 8192, w = 64: 12.6 MB).
// One persistent cooperative kernel: CTA g runs sweeps g, g + G, ... in order, and each
// sweep publishes its progress in a counter.  On a dense copy, step t
// of sweep c touches entries of sweep c - 1's steps up to t + 2, at t + 2 a single entry:
// the first of that step's right-reflector row.  The L2 kernel (w <= 128) waits until
// sweep c - 1 has finished its step t + 2.  The shared-memory kernel (w <= 64) forms each
// step's right reflector during the step before, as soon as that row is final, and
// writes the row then; a counter value of t + 1 means "steps <= t done and step t + 1's
// row written", and step t waits for t + 2 (a CPU simulation that interleaves concurrent
// sweeps phase by phase under either rule reproduces the sequential result bit for bit).
// The waits are bounded: past the time limit the kernel records BANDRED_DEV_TIMEOUT and
// returns.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "driver.h"
#include "kernels.h"
#include "launch.h"
#include "prof.h"

namespace bandred {
namespace {

constexpr int kGbThreads = 256;
constexpr int kGbWarps = kGbThreads / 32;
constexpr int kGbMaxW = 128;  // reflector length <= w <= 128: four entries per lane
constexpr int kGbDone = 1 << 30;

struct GbParams {
  int n, w, up, LB;  // entry (i, j), -up <= i - j <= w, at Bs[(i - j + up) + j LB]
  double* Bs;
  int* prog;         // prog[c]: steps sweep c has finished (kGbDone when finished)
  int* status;
  unsigned long long limit_ns;
};

// Loads go to L2 (ld.cg): another CTA may have changed a line this SM read before.
__device__ __forceinline__ double gld(const GbParams& p, int i, int j) {
  return __ldcg(&p.Bs[(int64_t)(i - j + p.up) + (int64_t)j * p.LB]);
}
__device__ __forceinline__ void gst(const GbParams& p, int i, int j, double x) {
  p.Bs[(int64_t)(i - j + p.up) + (int64_t)j * p.LB] = x;
}
__device__ __forceinline__ int gb_ld_acquire(const int* q) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(q) : "memory");
  return v;
}
__device__ __forceinline__ void gb_st_release(int* q, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(q), "r"(v) : "memory");
}

// The reflector of x (one warp; x[lane + 32 u] in xv[u], len <= 128), larfg convention
// with the max-scaled sum of squares: tau, beta, and the tail's scale, v = (x sx) scal, on
// every lane.  Along a long chase the bulge's far entries decay towards the underflow
// threshold, so tiny vectors are handled by exact power-of-two scalings: when every entry
// is below 2^-900 the reflector is formed from x 2^600 (the same tau and v, beta scaled
// back), and a tail below 2^-900 beside a larger alpha is scaled by 2^600 in the sum of
// squares, where 1 / max would overflow.
__device__ __forceinline__ void warp_reflector(const double (&xv)[4], int len, int lane, double& tau, double& beta,
                                               double& scal, double& sx) {
  double amax = 0.0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = lane + 32 * u;
    if (i >= 1 && i < len) amax = fmax(amax, fabs(xv[u]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  const double alpha = __shfl_sync(0xffffffffu, xv[0], 0);
  const double big = fmax(amax, fabs(alpha));
  sx = big < 0x1p-900 ? 0x1p600 : 1.0;
  const double am = amax * sx;
  const double ns = am < 0x1p-900 ? 0x1p600 : 1.0;
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
  tau = 0.0;
  beta = alpha;
  scal = 1.0;
  if (amax > 0.0) {
    const double as = alpha * sx;
    const double h = hypot(as, am * sqrt(ss));
    const double bs = as >= 0.0 ? -h : h;
    tau = (bs - as) / bs;
    scal = 1.0 / (as - bs);
    beta = bs * (1.0 / sx);
  }
}

__global__ void __launch_bounds__(kGbThreads) gb2bd_chase_kernel(GbParams p) {
  __shared__ double v[kGbMaxW];
  __shared__ double s_tau;
  __shared__ int s_ok;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = p.n, w = p.w;
  for (int c = blockIdx.x; c + 1 < n; c += gridDim.x) {
    int r = c, a = c + 1, t = 0;
    while (true) {
      const int end = min(a + w, n), len = end - a;
      if (len < 2) break;
      // wait for sweep c - 1 to pass step t + 2 (or to finish)
      if (tid == 0) {
        int ok = 1;
        if (c > 0) {
          unsigned long long t0 = 0;
          unsigned int spins = 0;
          while (gb_ld_acquire(&p.prog[c - 1]) < t + 3) {
            if ((++spins & 63u) == 0u) {
              const unsigned long long now = global_ns();
              if (t0 == 0) t0 = now;
              else if (now - t0 > p.limit_ns) {
                if (p.status) atomicCAS(p.status, 0, BANDRED_DEV_TIMEOUT);
                ok = 0;
                break;
              }
              if (p.status && gb_ld_acquire(p.status) != 0) { ok = 0; break; }
            }
          }
        }
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok) return;

      // right reflector from row r, columns [a, end); row r becomes (beta, 0, ..)
      if (warp == 0) {
        double xv[4], tau, beta, scal, sx;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = lane + 32 * u;
          xv[u] = j < len ? gld(p, r, a + j) : 0.0;
        }
        warp_reflector(xv, len, lane, tau, beta, scal, sx);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = lane + 32 * u;
          if (j < len) {
            v[j] = j == 0 ? 1.0 : (xv[u] * sx) * scal;
            gst(p, r, a + j, j == 0 ? beta : 0.0);
          }
        }
        if (lane == 0) s_tau = tau;
      }
      __syncthreads();
      double tau = s_tau;
      if (tau != 0.0) {
        // rows (r, min(a + w, n)), one warp each: y = row v, row -= tau y v^T
        for (int i = r + 1 + warp; i < min(a + w, n); i += kGbWarps) {
          double yv[4], z = 0.0;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = lane + 32 * u;
            yv[u] = j < len ? gld(p, i, a + j) : 0.0;
            if (j < len) z = fma(yv[u], v[j], z);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
          z *= tau;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = lane + 32 * u;
            if (j < len) gst(p, i, a + j, fma(-z, v[j], yv[u]));
          }
        }
      }
      __syncthreads();

      // left reflector from column a, rows [a, end); column a becomes (beta, 0, ..)^T
      if (warp == 0) {
        double xv[4], tl, beta, scal, sx;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = lane + 32 * u;
          xv[u] = i < len ? gld(p, a + i, a) : 0.0;
        }
        warp_reflector(xv, len, lane, tl, beta, scal, sx);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = lane + 32 * u;
          if (i < len) {
            v[i] = i == 0 ? 1.0 : (xv[u] * sx) * scal;
            gst(p, a + i, a, i == 0 ? beta : 0.0);
          }
        }
        if (lane == 0) s_tau = tl;
      }
      __syncthreads();
      tau = s_tau;
      if (tau != 0.0) {
        // columns (a, min(a + 2w, n)), one warp each: z = v^T col, col -= tau v z
        for (int j = a + 1 + warp; j < min(a + 2 * w, n); j += kGbWarps) {
          double yv[4], z = 0.0;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = lane + 32 * u;
            yv[u] = i < len ? gld(p, a + i, j) : 0.0;
            if (i < len) z = fma(v[i], yv[u], z);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
          z *= tau;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = lane + 32 * u;
            if (i < len) gst(p, a + i, j, fma(-z, v[i], yv[u]));
          }
        }
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        gb_st_release(&p.prog[c], t + 1);
      }
      r = a;
      a += w;
      ++t;
    }
    if (tid == 0) {
      __threadfence();
      gb_st_release(&p.prog[c], kGbDone);
    }
  }
}

// The same chase with the step's entries in shared memory (w <= 64), two threads per
// vector (each half of its entries, so all eight warps apply each reflector; the halves'
// dot products meet in shared memory).  A step touches the rows (r, a + w) of columns [a, a + w) (right reflector) and
// the rows [a, a + w) of columns (a, a + 2w) (left reflector); both sit in the tile of rows
// (r, a + w) by columns [a, a + 2w), staged once (its top-right corner, rows (r, a) by
// columns [a + w, a + 2w), lies outside the band store and is neither read nor written),
// with a row stride of kGTLd = 129 doubles: threads along a row step by 1 and threads
// along a column by 129 = 1 (mod 16) words, free of bank conflicts.  The left reflector's column a
// and the next step's right-reflector row a are set to (beta, 0, ..) in the tile and go
// out with its write-back; a sweep's first right-reflector row goes out directly.
constexpr int kGTMaxW = 64;
constexpr int kGTLd = 2 * kGTMaxW + 1;
// the tile, the two reflectors, the two halves' dot products
constexpr size_t kSmemGbTile = sizeof(double) * ((size_t)(2 * kGTMaxW - 1) * kGTLd + 2 * kGTMaxW + 4 * kGTMaxW);
static_assert(kGTMaxW == 64 && kGbThreads == 256, "two threads per vector, 32 entries each");

// Half of a vector (entries k0 .. k0 + 31 below len): y[kk] = b[kk st] in registers, and
// sum v[k0 + kk] y[kk] (four chains); then b[kk st] = y[kk] - z v[k0 + kk].
__device__ __forceinline__ double gb_half_load_dot(const double* b, int st, const double* v, int k0, int len,
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
__device__ __forceinline__ void gb_half_update(double* b, int st, const double* v, int k0, int len, double z,
                                               const double (&y)[32]) {
#pragma unroll
  for (int kk = 0; kk < 32; ++kk) {
    if (k0 + kk < len) b[kk * st] = fma(-z, v[k0 + kk], y[kk]);
  }
}

__global__ void __launch_bounds__(kGbThreads) gb2bd_chase_smem_kernel(GbParams p) {
  extern __shared__ double gt_smem[];
  double* U = gt_smem;                                       // (i, j) at (i - r - 1) kGTLd + (j - a)
  double* v = U + (size_t)(2 * kGTMaxW - 1) * kGTLd;         // the left reflector
  double* vr = v + kGTMaxW;                                  // the right reflector (formed a step early)
  double* zp = vr + kGTMaxW;                                 // the two halves' dot products, per vector
  __shared__ double s_tau, s_taur;
  __shared__ int s_ok;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = p.n, w = p.w;
  for (int c = blockIdx.x; c + 1 < n; c += gridDim.x) {
    int r = c, a = c + 1, t = 0;
    while (true) {
      const int end = min(a + w, n), len = end - a;
      if (len < 2) break;
      if (tid == 0) {
        int ok = 1;
        if (c > 0) {
          unsigned long long t0 = 0;
          unsigned int spins = 0;
          while (gb_ld_acquire(&p.prog[c - 1]) < t + 2) {
            if ((++spins & 63u) == 0u) {
              const unsigned long long now = global_ns();
              if (t0 == 0) t0 = now;
              else if (now - t0 > p.limit_ns) {
                if (p.status) atomicCAS(p.status, 0, BANDRED_DEV_TIMEOUT);
                ok = 0;
                break;
              }
              if (p.status && gb_ld_acquire(p.status) != 0) { ok = 0; break; }
            }
          }
        }
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok) return;
      // the tile: rows (r, rend), columns [a, cend); entry (i, j) belongs to the step when
      // j < end (right reflector) or a <= i < end (left reflector)
      const int rend = min(a + w, n), cend = min(a + 2 * w, n);
      const int nr = rend - r - 1, nc = cend - a;
      for (int q = tid; q < nr * nc; q += kGbThreads) {
        const int jj = q / nr, ii = q - jj * nr;
        const int i = r + 1 + ii, j = a + jj;
        const bool mine = j < end || (i >= a && i < end);
        U[(size_t)ii * kGTLd + jj] = mine ? gld(p, i, j) : 0.0;
      }
      if (t == 0 && warp == 0) {
        // a sweep's first right reflector, from row r; row r becomes (beta, 0, ..).  The
        // later ones are formed by the step before (below), from its final row a
        double xv[4], tau, beta, scal, sx;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = lane + 32 * u;
          xv[u] = j < len ? gld(p, r, a + j) : 0.0;
        }
        warp_reflector(xv, len, lane, tau, beta, scal, sx);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = lane + 32 * u;
          if (j < len) {
            vr[j] = j == 0 ? 1.0 : (xv[u] * sx) * scal;
            gst(p, r, a + j, j == 0 ? beta : 0.0);
          }
        }
        if (lane == 0) s_taur = tau;
      }
      __syncthreads();
      double tau = s_taur;
      // the right reflector on the tile's rows (columns [a, end)): two threads per row,
      // thread q + 128 h taking columns a + 32 h .. a + 32 h + 31, so all eight warps work
      {
        const int q = tid & 127, h = tid >> 7, k0 = 32 * h;
        const bool have = tau != 0.0 && q < nr;
        double* b = U + (size_t)q * kGTLd + k0;
        double y[32];
        if (have) zp[h * 128 + q] = gb_half_load_dot(b, 1, vr, k0, len, y);
        __syncthreads();
        if (have) gb_half_update(b, 1, vr, k0, len, tau * (zp[q] + zp[128 + q]), y);
      }
      __syncthreads();

      // left reflector from column a, rows [a, end) (tile rows a - r - 1 ..); the column
      // becomes (beta, 0, ..)^T, in the tile and in global memory
      const int ia = a - r - 1;
      if (warp == 0) {
        double xv[4], tl, beta, scal, sx;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = lane + 32 * u;
          xv[u] = i < len ? U[(size_t)(ia + i) * kGTLd] : 0.0;
        }
        warp_reflector(xv, len, lane, tl, beta, scal, sx);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = lane + 32 * u;
          if (i < len) {
            v[i] = i == 0 ? 1.0 : (xv[u] * sx) * scal;
            U[(size_t)(ia + i) * kGTLd] = i == 0 ? beta : 0.0;
          }
        }
        if (lane == 0) s_tau = tl;
      }
      __syncthreads();
      tau = s_tau;
      // the left reflector on columns (a, cend) (rows [a, end)): two threads per column,
      // thread q + 128 h taking rows a + 32 h .. a + 32 h + 31
      {
        const int q = tid & 127, h = tid >> 7, i0 = 32 * h;
        const bool have = tau != 0.0 && q >= 1 && q < nc;
        double* b = U + (size_t)(ia + i0) * kGTLd + q;
        double y[32];
        if (have) zp[h * 128 + q] = gb_half_load_dot(b, kGTLd, v, i0, len, y);
        __syncthreads();
        if (have) gb_half_update(b, kGTLd, v, i0, len, tau * (zp[q] + zp[128 + q]), y);
      }
      __syncthreads();
      // the next step's right reflector, from row a (tile row ia) over columns
      // [a + w, a + w + nl), final now; the row becomes (beta, 0, ..) in the tile and goes
      // out with the write-back below.  This row's first entry is the one entry the sweep
      // after shares with the next step, so with it written at this step's release the
      // sweep after may run two steps behind instead of three.
      const int nl = min(a + 2 * w, n) - (a + w);
      if (nl >= 2 && warp == 0) {
        double xv[4], tn, beta, scal, sx;
        double* row = U + (size_t)ia * kGTLd + w;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = lane + 32 * u;
          xv[u] = j < nl ? row[j] : 0.0;
        }
        warp_reflector(xv, nl, lane, tn, beta, scal, sx);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = lane + 32 * u;
          if (j < nl) {
            vr[j] = j == 0 ? 1.0 : (xv[u] * sx) * scal;
            row[j] = j == 0 ? beta : 0.0;
          }
        }
        if (lane == 0) s_taur = tn;
      }
      __syncthreads();
      // the step's entries back to the band store, column by column
      for (int q = tid; q < nr * nc; q += kGbThreads) {
        const int jj = q / nr, ii = q - jj * nr;
        const int i = r + 1 + ii, j = a + jj;
        if (j < end || (i >= a && i < end)) gst(p, i, j, U[(size_t)ii * kGTLd + jj]);
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        gb_st_release(&p.prog[c], t + 1);
      }
      r = a;
      a += w;
      ++t;
    }
    if (tid == 0) {
      __threadfence();
      gb_st_release(&p.prog[c], kGbDone);
    }
  }
}

// Band store from the upper band of A (0 <= j - i <= w; everything else of A, such as the
// reflectors of a packed ge2gb result, is not read), zeros elsewhere.
__global__ void gb_band_in_kernel(int n, int w, int up, int LB, const double* A, int64_t lda, double* Bs) {
  const int64_t total = (int64_t)n * LB;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int off = (int)(q % LB), j = (int)(q / LB), i = j + off - up;
    Bs[q] = (i >= 0 && j - i >= 0 && j - i <= w) ? A[i + (int64_t)j * lda] : 0.0;
  }
}

__global__ void gb_band_out_kernel(int n, int up, int LB, const double* Bs, double* d, double* e) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    d[k] = Bs[up + (int64_t)k * LB];
    if (k + 1 < n) e[k] = Bs[(up - 1) + (int64_t)(k + 1) * LB];
  }
}

// The Golub-Kahan tridiagonal of the upper bidiagonal (d, e): zero diagonal, off-diagonal
// d_0, e_0, d_1, e_1, .., d_{n-1} (2n - 1 entries; o[2n - 1] = 0 is not read).
__global__ void tgk_kernel(int n, const double* d, const double* e, double* z, double* o) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < 2 * n; q += gridDim.x * blockDim.x) {
    z[q] = 0.0;
    const int i = q >> 1;
    o[q] = (q & 1) ? (i + 1 < n ? e[i] : 0.0) : d[i];
  }
}

// The singular values, descending, from the n largest eigenvalues of the Golub-Kahan
// tridiagonal (its eigenvalues are +-sigma_k), ascending in lam[0 .. n).
__global__ void sv_out_kernel(int n, const double* lam, double* sig) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) sig[k] = lam[n - 1 - k];
}

struct GbWs {
  double* Bs;
  int* prog;
  int* status;
  size_t bytes;
};

GbWs carve_gb2bd(void* work, int64_t n, int64_t w) {
  char* base = static_cast<char*>(work);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = base ? base + off : nullptr;
    off += (bytes + 255) / 256 * 256;
    return q;
  };
  GbWs ws{};
  ws.Bs = reinterpret_cast<double*>(take(sizeof(double) * (size_t)std::max<int64_t>(n, 1) * 3 * w));
  ws.prog = reinterpret_cast<int*>(take(sizeof(int) * (size_t)std::max<int64_t>(n, 1)));
  ws.status = reinterpret_cast<int*>(take(256));
  ws.bytes = off;
  return ws;
}

#define CKG(call)                                                 \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return record_cuda_error(e_, #call);   \
  } while (0)

}  // namespace

size_t gb2bd_workspace_bytes(int64_t n, int64_t w) { return carve_gb2bd(nullptr, n, w).bytes; }

int gb2bd_run(int64_t n, int64_t w, const double* A, int64_t lda, double* d, double* e, unsigned long long limit_ns,
              void* work, int* dev_status, cudaStream_t s) {
  GbWs ws = carve_gb2bd(work, n, w);
  int* status = dev_status ? dev_status : ws.status;
  CKG(cudaMemsetAsync(status, 0, sizeof(int), s));
  if (n <= 0) return 0;
  const int LB = (int)(3 * w), up = (int)(2 * w - 1);
  {
    const int blocks = (int)std::min<int64_t>((n * LB + 255) / 256, 4096);
    prof::count_launch();
    gb_band_in_kernel<<<blocks, 256, 0, s>>>((int)n, (int)w, up, LB, A, lda, ws.Bs);
    CKG(cudaGetLastError());
  }
  if (n > 2 && w > 1) {
    CKG(cudaMemsetAsync(ws.prog, 0, sizeof(int) * (size_t)n, s));
    int dev = 0, sms = 0;
    CKG(cudaGetDevice(&dev));
    CKG(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // one CTA per SM, all co-resident (the cooperative launch guarantees it): a sweep
    // waits only on the sweep before it, which another CTA runs
    const int G = (int)std::min<int64_t>(n - 1, sms);
    GbParams p{(int)n, (int)w, up, LB, ws.Bs, ws.prog, status, limit_ns};
    void* args[] = {&p};
    prof::count_launch();
    if (w <= kGTMaxW) {
      static int configured = -1;
      if (configured != dev) {
        CKG(cudaFuncSetAttribute(gb2bd_chase_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmemGbTile));
        configured = dev;
      }
      CKG(cudaLaunchCooperativeKernel((const void*)gb2bd_chase_smem_kernel, dim3(G), dim3(kGbThreads), args,
                                      kSmemGbTile, s));
    } else {
      CKG(cudaLaunchCooperativeKernel((const void*)gb2bd_chase_kernel, dim3(G), dim3(kGbThreads), args, 0, s));
    }
  }
  {
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
    prof::count_launch();
    gb_band_out_kernel<<<blocks, 256, 0, s>>>((int)n, up, LB, ws.Bs, d, e);
    CKG(cudaGetLastError());
  }
  return 0;
}

size_t bdsv_workspace_bytes(int64_t n) {
  const size_t v = (sizeof(double) * (size_t)std::max<int64_t>(2 * n, 1) + 255) / 256 * 256;
  return 3 * v + sterf_workspace_bytes(std::max<int64_t>(2 * n, 1));
}

int bdsv_run(int64_t n, const double* d, const double* e, double* sig, void* work, cudaStream_t s) {
  if (n <= 0) return 0;
  const size_t v = (sizeof(double) * (size_t)(2 * n) + 255) / 256 * 256;
  char* base = static_cast<char*>(work);
  double* z = reinterpret_cast<double*>(base);
  double* o = reinterpret_cast<double*>(base + v);
  double* lam = reinterpret_cast<double*>(base + 2 * v);
  void* sw = base + 3 * v;
  const int blocks = (int)std::min<int64_t>((2 * n + 255) / 256, 1024);
  prof::count_launch();
  tgk_kernel<<<blocks, 256, 0, s>>>((int)n, d, e, z, o);
  CKG(cudaGetLastError());
  // only the upper half of the Golub-Kahan spectrum: eigenvalues n .. 2n - 1
  const int rc = sterf_range_run(2 * n, z, o, lam, n, n, sw, s);
  if (rc != 0) return rc;
  prof::count_launch();
  sv_out_kernel<<<blocks, 256, 0, s>>>((int)n, lam, sig);
  CKG(cudaGetLastError());
  return 0;
}

}  // namespace bandred
