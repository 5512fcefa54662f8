// Panel factorisation in FP64: Householder QR of a tall j x bk panel (Eq. updateA0 of
// Section 2.1; Eq. updateB of Section 3.1) or, through transposed addressing, the LQ
// factorisation of a wide bk x j row panel (Eq. updateC).  Produces, in one cooperative
// launch:
//   - the reflectors in the packed LAPACK layout (beta on the diagonal, v below it,
//     tau[0..bk)),
//   - Y: a contiguous copy of V with its unit diagonal and zeros above (j x bk),
//   - W = -Y T (j x bk), so that the panel's orthogonal factor is Q = I + W Y^T with the
//     compact-WY triangular factor T of the paper's reference implementation (Section 4.1).
//
// Design (one GPU, FP64 on the CUDA cores):
//   Each CTA keeps a contiguous slab of the panel's rows in shared memory.  For reflector
//   i the CTAs compute, over their rows below row i, the dot products of column i with
//   every panel column (column i itself gives ||x2||^2; earlier columns give the entries
//   Y^T y_i needed for T; later columns give v^T a_c for the in-panel update), add them
//   into accumulators in L2, publish row i, and meet at one grid-wide barrier.  After it
//   every CTA reads the same sums, derives the same beta, tau and coefficients, and
//   updates its own rows without further communication.  GB300 issues FP64 at two
//   operations per clock per SM, so the kernel keeps FP64 instructions to the FMAs the
//   method needs (no per-CTA re-summation of partials, hoisted scalings).
//   W's column i follows from the recurrence W(:, i) = -tau_i (y_i + W(:, 0:i) Y(:, 0:i)^T y_i),
//   which equals -Y T with T built column by column as in the compact-WY definition.
#include <cmath>

#include "panel_common.cuh"
#include "prof.h"

namespace bandred {

namespace {

using namespace panel_detail;

__global__ void __launch_bounds__(kPanelThreads, 1) panel_qr_kernel(PanelParams p) {
  extern __shared__ double smem[];
  constexpr int NT = kPanelThreads;
  const int tid = threadIdx.x, lane = tid & 31;
  const int G = gridDim.x, g = blockIdx.x;
  const int bk = p.bk, Rp = p.Rp;
  const int rb = g * p.R;
  const int nr = max(0, min(p.R, p.j - rb));
  double* slab = smem;                        // bk columns x Rp rows
  double* dsum = slab + (size_t)bk * Rp;      // bk + 1 combined sums
  double* rowi = dsum + bk + 1;               // row i of the panel
  double* coef = rowi + bk;                   // z_c (c > i) and, for c < i, Y^T y_i
  double* coef2 = coef + bk;                  // -z_c * scal (c > i)
  double* gprev = coef2 + bk;                 // Y^T y of the previous reflector (for W)
  float* gprevf = reinterpret_cast<float*>(gprev + bk);  // the same in FP32 (bk floats)
  double* after = gprev + bk + (bk + 1) / 2;
  // This CTA's rows of W: in shared memory when they fit (FP32 when p.w_fp32), else in
  // the W output itself.
  const bool wf32 = p.w_in_smem && p.w_fp32;
  double* wl = p.w_in_smem ? after : p.W + rb;
  float* wlf = reinterpret_cast<float*>(after);
  const int64_t wld = p.w_in_smem ? Rp : p.ldy;
  __shared__ double s_beta, s_tau, s_scal, s_tau_prev;
  __shared__ double s_red[NT / 32];
  __shared__ int s_rescale, s_ok;

  if (p.rs == 1) {
    for (int idx = tid; idx < nr * bk; idx += NT) {
      const int r = idx % nr, c = idx / nr;
      slab[(size_t)c * Rp + r] = p.A[(int64_t)(rb + r) + (int64_t)c * p.cs];
    }
  } else {
    for (int idx = tid; idx < nr * bk; idx += NT) {
      const int c = idx % bk, r = idx / bk;
      slab[(size_t)c * Rp + r] = p.A[(int64_t)(rb + r) * p.rs + (int64_t)c * p.cs];
    }
  }
  __syncthreads();

  // Threads per column in the dot products (a power of two dividing 32).
  const int TPC = bk >= 128 ? 2 : (bk >= 64 ? 4 : 8);
  const int CPP = NT / TPC;  // columns per pass
  const int sub = tid % TPC;
  const size_t accsz = (size_t)(bk + 1) * kAccStride;
  unsigned int gen = 0;
  for (int i = 0; i < bk; ++i) {
    double* acc = p.acc + (size_t)(i % 3) * accsz;
    double* rowg = p.rowbuf + (size_t)(i & 1) * bk;
    const int lo = min(max(i + 1 - rb, 0), nr);
    const double* xi = slab + (size_t)i * Rp;
    const bool own_row = (i >= rb) && (i < rb + nr);
    if (g == 0) {  // clear the buffer of step i+1 (last read at step i-2, before barrier i-1)
      double* nxt = p.acc + (size_t)((i + 1) % 3) * accsz;
      for (int v = tid; v <= bk; v += NT) nxt[(size_t)v * kAccStride] = 0.0;
    }

    // Partial dot products of x2 = column i below row i with every panel column, added
    // into the L2 accumulators (two independent FMA chains per thread).
    for (int c0 = 0; c0 < bk; c0 += CPP) {
      const int c = c0 + tid / TPC;
      double s = 0.0, t = 0.0;
      if (c < bk) {
        const double* ac = slab + (size_t)c * Rp;
        int r = lo + sub;
        for (; r + TPC < nr; r += 2 * TPC) {
          s = fma(xi[r], ac[r], s);
          t = fma(xi[r + TPC], ac[r + TPC], t);
        }
        if (r < nr) s = fma(xi[r], ac[r], s);
      }
      s += t;
      for (int o = TPC / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (sub == 0 && c < bk) atomicAdd(&acc[(size_t)c * kAccStride], s);
    }
    // max |x2| by integer comparison of the bit patterns (no FP64 instruction): one warp
    if (tid < 32) {
      unsigned long long m = 0ull;
      for (int r = lo + lane; r < nr; r += 32) {
        const unsigned long long u = (unsigned long long)__double_as_longlong(xi[r]) & 0x7FFFFFFFFFFFFFFFull;
        m = u > m ? u : m;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v > m ? v : m;
      }
      if (lane == 0) atomicMax(reinterpret_cast<unsigned long long*>(&acc[(size_t)bk * kAccStride]), m);
    }
    if (own_row)
      for (int c = tid; c < bk; c += NT) __stcg(&rowg[c], slab[(size_t)c * Rp + (i - rb)]);
    __syncthreads();
    if (tid == 0) grid_arrive(p.gs);
    ++gen;
    // W column of the previous reflector: off the critical path, overlaps the barrier.
    if (i > 0) {
      if (wf32)
        w_column_f32(i - 1, (float)s_tau_prev, gprevf, slab, Rp, rb, nr, wlf);
      else
        w_column(i - 1, s_tau_prev, gprev, slab, Rp, rb, nr, wl, wld);
    }
    if (tid == 0) s_ok = grid_wait(p.gs, gen, p.extra, p.status, p.limit_ns) ? 1 : 0;
    __syncthreads();
    if (!s_ok) return;

    // Thread 0 reads the three numbers the reflector needs and derives it while warps
    // 1..7 fetch the remaining sums and row i (warp 0 does nothing else, so the two do
    // not serialise through divergence).
    if (tid == 0) {
      const double alpha = ldcg(&rowg[i]);
      const double ssq = ldcg(&acc[(size_t)i * kAccStride]);
      const double amax = ldcg(&acc[(size_t)bk * kAccStride]);
      const int rescale = (p.j - i > 1) && (amax > 0.0) && !(ssq < 0x1p1000 && amax > 0x1p-450);
      s_rescale = rescale || !(fabs(alpha) < 0x1p500);
      // Common path: h = ||[alpha; x2]|| = q / sqrt(q) with q = alpha^2 + ||x2||^2 (no
      // overflow: both terms are bounded here); tau = (beta - alpha) / beta = 1 + |alpha|/h
      // and scal = 1 / (alpha - beta) = sign(alpha) / (|alpha| + h).
      double tau = 0.0, beta = alpha, scal = 1.0;
      if (!s_rescale && p.j - i > 1 && ssq != 0.0) {
        const double q = fma(alpha, alpha, ssq);
        const double rq = rsqrt_newton(q);
        const double h = q * rq;
        const double aa = fabs(alpha);
        beta = (alpha >= 0.0) ? -h : h;
        tau = fma(aa, rq, 1.0);
        const double rs = rcp_newton(aa + h);
        scal = (alpha >= 0.0) ? rs : -rs;
      }
      s_beta = beta;
      s_tau = tau;
      s_scal = scal;
    } else if (tid >= 32) {
      for (int v = tid - 32; v <= bk; v += NT - 32) dsum[v] = ldcg(&acc[(size_t)v * kAccStride]);
      for (int c = tid - 32; c < bk; c += NT - 32) rowi[c] = ldcg(&rowg[c]);
    }
    __syncthreads();

    // Rare path: the plain sum of squares over/underflows (or |alpha| is huge): a scaled
    // second pass over x2 and the overflow-safe formulas.  Same decision in every CTA.
    if (s_rescale) {
      const double inv = dsum[bk] > 0.0 ? 1.0 / dsum[bk] : 0.0;
      double s = 0.0;
      for (int r = lo + tid; r < nr; r += NT) {
        const double t = xi[r] * inv;
        s = fma(t, t, s);
      }
      s = warp_sum(s);
      if (lane == 0) s_red[tid >> 5] = s;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int q = 0; q < NT / 32; ++q) t += s_red[q];
        __stcg(&p.part2[g], t);
      }
      if (!grid_barrier(p.gs, ++gen, p.extra, p.status, p.limit_ns)) return;
      if (tid < 32) {
        double t = 0.0;
        for (int q = lane; q < G; q += 32) t += ldcg(&p.part2[q]);
        t = warp_sum(t);
        if (lane == 0) {
          const double amax = dsum[bk];
          const bool rescaled = (p.j - i > 1) && (amax > 0.0) && !(dsum[i] < 0x1p1000 && amax > 0x1p-450);
          const double xnorm = rescaled ? amax * sqrt(t) : sqrt(dsum[i]);
          const double alpha = rowi[i];
          double tau = 0.0, beta = alpha, scal = 1.0;
          if (p.j - i > 1 && xnorm != 0.0) {
            const double h = hypot(alpha, xnorm);
            beta = (alpha >= 0.0) ? -h : h;
            tau = (beta - alpha) / beta;
            scal = 1.0 / (alpha - beta);
          }
          s_beta = beta;
          s_tau = tau;
          s_scal = scal;
        }
      }
      __syncthreads();
    }
    if (tid == 0 && g == 0) p.tau[i] = s_tau;

    const double tau = s_tau, scal = s_scal;
    // Coefficients and the in-panel update, one column per group of TPU threads:
    // z_c = tau v^T a_c, a_c -= z_c v (c > i); and (Y^T y_i)_c for c < i (for W).
    {
      const int TPU = bk >= 128 ? 2 : (bk >= 64 ? 4 : 8);
      for (int c0 = 0; c0 < bk; c0 += NT / TPU) {
        const int c = c0 + tid / TPU, rg = tid % TPU;
        if (c > i && c < bk) {
          const double z = tau * fma(scal, dsum[c], rowi[c]);
          if (tau != 0.0) {
            const double z2 = -z * scal;
            double* ac = slab + (size_t)c * Rp;
            for (int r = lo + rg; r < nr; r += TPU) ac[r] = fma(z2, xi[r], ac[r]);
            if (own_row && rg == 0) ac[i - rb] -= z;
          }
        } else if (c < i && rg == 0) {
          const double gv = fma(scal, dsum[c], rowi[c]);
          gprev[c] = gv;
          gprevf[c] = f64_to_f32_rz(gv);
        }
      }
    }
    __syncthreads();
    if (tau != 0.0)
      for (int r = lo + tid; r < nr; r += NT) slab[(size_t)i * Rp + r] *= scal;
    if (own_row && tid == 0) slab[(size_t)i * Rp + (i - rb)] = s_beta;
    if (tid == 0) s_tau_prev = tau;
    __syncthreads();
  }
  if (wf32)
    w_column_f32(bk - 1, (float)s_tau_prev, gprevf, slab, Rp, rb, nr, wlf);
  else
    w_column(bk - 1, s_tau_prev, gprev, slab, Rp, rb, nr, wl, wld);
  __syncthreads();

  if (wf32) {
    for (int idx = tid; idx < nr * bk; idx += NT) {
      const int r = idx % nr, c = idx / nr;
      p.W[rb + r + (int64_t)c * p.ldy] = tc::f32_to_f64(wlf[r + c * Rp]);
    }
  } else if (p.w_in_smem) {
    for (int idx = tid; idx < nr * bk; idx += NT) {
      const int r = idx % nr, c = idx / nr;
      p.W[rb + r + (int64_t)c * p.ldy] = wl[r + (int64_t)c * wld];
    }
  }

  // Write back: packed reflectors/R into the matrix, Y into the workspace.
  if (p.rs == 1) {
    for (int idx = tid; idx < nr * bk; idx += NT) {
      const int r = idx % nr, c = idx / nr;
      const double v = slab[(size_t)c * Rp + r];
      p.A[(int64_t)(rb + r) + (int64_t)c * p.cs] = v;
      const int gr = rb + r;
      p.Y[gr + (int64_t)c * p.ldy] = gr > c ? v : (gr == c ? 1.0 : 0.0);
    }
  } else {
    for (int idx = tid; idx < nr * bk; idx += NT) {
      const int c = idx % bk, r = idx / bk;
      p.A[(int64_t)(rb + r) * p.rs + (int64_t)c * p.cs] = slab[(size_t)c * Rp + r];
    }
    for (int idx = tid; idx < nr * bk; idx += NT) {
      const int r = idx % nr, c = idx / nr;
      const int gr = rb + r;
      p.Y[gr + (int64_t)c * p.ldy] = gr > c ? slab[(size_t)c * Rp + r] : (gr == c ? 1.0 : 0.0);
    }
  }
}

}  // namespace

size_t panel_smem_bytes(int bk, int Rp, bool w_in_smem) {
  return ((size_t)bk * Rp * (w_in_smem ? 2 : 1) + 5 * (size_t)bk + 1 + (bk + 1) / 2) * sizeof(double);
}

size_t panel_sync_bytes(int bk) { return 256 + 3 * (size_t)(bk + 1) * kAccStride * sizeof(double); }

int panel_geometry(int j, int bk, int max_ctas, int min_rows, int* G, int* R, int* Rp, bool* w_in_smem) {
  if (j <= 0 || bk <= 0) return -1;
  int g = (j + min_rows - 1) / min_rows;
  if (g > max_ctas) g = max_ctas;
  if (g < 1) g = 1;
  int r = (j + g - 1) / g;
  g = (j + r - 1) / r;  // every CTA owns at least one row
  int rp = r | 1;       // odd stride: conflict-free strided shared-memory access
  if (panel_smem_bytes(bk, rp, false) > 227 * 1024) return -2;
  *G = g;
  *R = r;
  *Rp = rp;
  *w_in_smem = panel_smem_bytes(bk, rp, true) <= 227 * 1024;
  return 0;
}

cudaError_t launch_panel(const PanelParams& prm, int G, cudaStream_t s) {
  static int configured_device = -1;
  static size_t max_dynamic = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_device != dev) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, panel_qr_kernel);
    if (e != cudaSuccess) return e;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    max_dynamic = (size_t)optin - fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(panel_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_dynamic);
    if (e != cudaSuccess) return e;
    configured_device = dev;
  }
  const size_t smem = panel_smem_bytes(prm.bk, prm.Rp, prm.w_in_smem);
  if (smem > max_dynamic) return cudaErrorInvalidValue;
  // barrier counters and the first accumulator buffer (contiguous, see PanelParams)
  cudaError_t e = cudaMemsetAsync(prm.gs, 0, panel_sync_bytes(prm.bk), s);
  if (e != cudaSuccess) return e;
  PanelParams p = prm;
  void* args[] = {&p};
  prof::count_launch();
  return cudaLaunchCooperativeKernel((const void*)panel_qr_kernel, dim3(G), dim3(kPanelThreads), args, smem, s);
}

}  // namespace bandred
