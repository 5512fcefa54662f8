// Panel factorisation by one thread-block cluster per panel (Eq. updateA0 of Section 2.1;
// Eqs. updateB and updateC of Section 3.1), for panels short enough that C <= 16 CTAs
// hold them: the small panels of the batched reductions and the last panels of a large
// one.  Computes what panel.cu computes (reflectors in place, tau, Y, W = -Y T) but the
// per-reflector sums travel through distributed shared memory: every CTA writes its
// partial sums into its own shared memory, the cluster meets at the hardware cluster
// barrier (arrive, then W of the previous reflector, then wait), and each CTA adds the
// C partials in rank order, so the result is deterministic and no grid-wide
// synchronisation or cooperative launch is needed.  A batch of panels is one launch:
// cluster y of the grid factors problem y.
#include <cooperative_groups.h>

#include "panel_common.cuh"
#include "prof.h"

namespace bandred {

namespace {

using namespace panel_detail;
namespace cg = cooperative_groups;

__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

__global__ void __launch_bounds__(kPanelThreads, 4)
    panel_cluster_kernel(PanelParams single, const PanelParams* probs) {
  extern __shared__ double smem[];
  constexpr int NT = kPanelThreads;
  cg::cluster_group cluster = cg::this_cluster();
  const PanelParams& p = probs ? probs[blockIdx.y] : single;
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int bk = p.bk;
  if (bk <= 0) return;  // inactive problem: the whole cluster leaves together
  const int tid = threadIdx.x, lane = tid & 31;
  const int R = p.R, Rp = p.Rp;
  const int rb = rank * R;
  const int nr = max(0, min(R, p.j - rb));
  double* slab = smem;                             // bk columns x Rp rows
  double* part = slab + (size_t)bk * Rp;           // 2 x (bk + 2): partial sums (+ amax bits)
  double* rowpub = part + 2 * (bk + 2);            // 2 x bk: row i, when this CTA owns it
  double* dsum = rowpub + 2 * bk;                  // bk + 1
  double* rowi = dsum + bk + 1;                    // bk
  double* gprev = rowi + bk;                       // bk
  float* gprevf = reinterpret_cast<float*>(gprev + bk);
  double* resc = gprev + bk + (bk + 1) / 2;        // bk: partial sums of the rare path's scaled pass
  double* after = resc + bk;
  const bool wf32 = p.w_fp32;
  // gram: W is formed after the panel (w_from_gram) from the T coefficients that rank 0
  // stores into p.G; no W recurrence inside the panel
  const bool gram = p.G != nullptr;
  double* wl = after;                              // W rows: FP64 or FP32, always in shared memory
  float* wlf = reinterpret_cast<float*>(after);
  __shared__ double s_beta, s_tau, s_scal, s_dscal, s_tau_prev;
  __shared__ int s_rescale;
  trace_start(p.trace);

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

  const int TPC = bk >= 128 ? 2 : (bk >= 64 ? 4 : 8);
  const int CPP = NT / TPC;
  const int sub = tid % TPC;
  const int pst = bk + 2;
  for (int i = 0; i < bk; ++i) {
    const int buf = i & 1;
    double* mypart = part + buf * pst;
    double* myrow = rowpub + buf * bk;
    const int lo = min(max(i + 1 - rb, 0), nr);
    const double* xi = slab + (size_t)i * Rp;
    const int owner = i / R;

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
      if (sub == 0 && c < bk) mypart[c] = s;
    }
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
      if (lane == 0) mypart[bk] = __longlong_as_double((long long)m);
    }
    if (rank == owner)
      for (int c = tid; c < bk; c += NT) myrow[c] = slab[(size_t)c * Rp + (i - rb)];
    __syncthreads();
    cluster_arrive();
    if (i > 0 && !gram) {
      if (wf32)
        w_column_f32(i - 1, (float)s_tau_prev, gprevf, slab, Rp, rb, nr, wlf);
      else
        w_column(i - 1, s_tau_prev, gprev, slab, Rp, rb, nr, wl, Rp);
    }
    cluster_wait();

    // Sums over the cluster in rank order (identical in every CTA).
    for (int v = tid; v <= bk; v += NT) {
      if (v < bk) {
        double s = 0.0;
        for (int q = 0; q < C; ++q) s += *cluster.map_shared_rank(&mypart[v], q);
        dsum[v] = s;
      } else {
        unsigned long long m = 0ull;
        for (int q = 0; q < C; ++q) {
          const unsigned long long u =
              (unsigned long long)__double_as_longlong(*cluster.map_shared_rank(&mypart[bk], q));
          m = u > m ? u : m;
        }
        dsum[bk] = __longlong_as_double((long long)m);
      }
    }
    for (int c = tid; c < bk; c += NT) rowi[c] = *cluster.map_shared_rank(&myrow[c], owner);
    __syncthreads();

    if (tid == 0) {
      const double alpha = rowi[i], ssq = dsum[i], amax = dsum[bk];
      const long long us = dbits(ssq), um = dbits(amax);  // amax >= 0 (an integer maximum)
      const int rescale = (p.j - i > 1) && (um > 0) && !(us >= 0 && us < kBits2p1000 && um > kBits2m450);
      s_rescale = rescale || !(abits(alpha) < kBits2p500);
      double tau = 0.0, beta = alpha, scal = 1.0;
      if (!s_rescale && p.j - i > 1 && (us << 1) != 0) {
        const double q = fma(alpha, alpha, ssq);
        const double rq = rsqrt_newton(q);
        const double h = q * rq;
        const double aa = fabs(alpha);
        const bool apos = nonneg(alpha);
        beta = neg_if(h, apos);
        tau = fma(aa, rq, 1.0);
        const double rs = rcp_newton(aa + h);
        scal = neg_if(rs, !apos);
      }
      s_beta = beta;
      s_tau = tau;
      s_scal = scal;
      s_dscal = scal;
    }
    // A sum outside the range where the plain formulas hold (not finite, or near the
    // overflow threshold) forces the scaled path too.
    int bad = 0;
    for (int v = tid; v < bk; v += NT) bad |= !(abits(dsum[v]) < kBits2p1000);
    const int force = __syncthreads_or(bad);
    // Rare path: column i scaled by the power of two 2^-e with 2^e <= max|x2| < 2^(e+1)
    // (exact); a second cluster reduction forms ||x2 2^-e||^2 and the dot products
    // (x2 2^-e)^T a_c, and the coefficients take scal 2^e for the dot terms.  Same
    // decision in every CTA of the cluster.
    if (s_rescale || force) {
      const double amax = dsum[bk];
      const int e = amax > 0.0 ? max(-1022, min(1022, ilogb(amax))) : 0;
      const double inv = ldexp(1.0, -e), sc = ldexp(1.0, e);
      for (int c0 = 0; c0 < bk; c0 += CPP) {
        const int c = c0 + tid / TPC;
        double sv = 0.0;
        if (c < bk) {
          const double* ac = slab + (size_t)c * Rp;
          for (int r = lo + sub; r < nr; r += TPC) {
            const double t = xi[r] * inv;
            sv = fma(t, c == i ? t : ac[r], sv);
          }
        }
        for (int o = TPC / 2; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
        if (sub == 0 && c < bk) resc[c] = sv;
      }
      cluster.sync();
      for (int v = tid; v < bk; v += NT) {
        double t = 0.0;
        for (int q = 0; q < C; ++q) t += *cluster.map_shared_rank(&resc[v], q);
        dsum[v] = t;
      }
      __syncthreads();
      if (tid == 0) {
        const double xnorm = amax > 0.0 ? sqrt(dsum[i]) * sc : 0.0;
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
        s_dscal = scal * sc;
      }
      __syncthreads();
    }
    if (tid == 0 && rank == 0) p.tau[i] = s_tau;
    const double tau = s_tau, scal = s_scal, dscal = s_dscal;
    const bool own_row = rank == owner;
    {
      const int TPU = bk >= 128 ? 2 : (bk >= 64 ? 4 : 8);
      for (int c0 = 0; c0 < bk; c0 += NT / TPU) {
        const int c = c0 + tid / TPU, rg = tid % TPU;
        if (c > i && c < bk) {
          const double z = tau * fma(dscal, dsum[c], rowi[c]);
          if (tau != 0.0) {
            const double z2 = -z * scal;
            double* ac = slab + (size_t)c * Rp;
            for (int r = lo + rg; r < nr; r += TPU) ac[r] = fma(z2, xi[r], ac[r]);
            if (own_row && rg == 0) ac[i - rb] -= z;
          }
        } else if (c < i && rg == 0) {
          const double gv = fma(dscal, dsum[c], rowi[c]);
          gprev[c] = gv;
          if (gram && rank == 0) p.G[c + (size_t)i * bk] = gv;
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
  if (!gram) {
    if (wf32)
      w_column_f32(bk - 1, (float)s_tau_prev, gprevf, slab, Rp, rb, nr, wlf);
    else
      w_column(bk - 1, s_tau_prev, gprev, slab, Rp, rb, nr, wl, Rp);
    __syncthreads();
    for (int idx = tid; idx < nr * bk; idx += NT) {
      const int r = idx % nr, c = idx / nr;
      p.W[rb + r + (int64_t)c * p.ldy] = wf32 ? tc::f32_to_f64(wlf[r + c * Rp]) : wl[r + (int64_t)c * Rp];
    }
  }
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
  cluster.sync();  // no CTA leaves while a peer may still read its shared memory
  trace_end(p.trace);
}

}  // namespace

size_t panel_cluster_smem_bytes(int bk, int Rp) {
  return ((size_t)bk * Rp * 2 + 2 * (size_t)(bk + 2) + 2 * (size_t)bk + (bk + 1) + 2 * (size_t)bk + (bk + 1) / 2 +
          (size_t)bk) *
         sizeof(double);
}

// Rows per CTA for a cluster of C CTAs over a j x bk panel (0 when it does not fit).
int panel_cluster_rows(int j, int bk, int C) {
  const int R = (j + C - 1) / C;
  if (panel_cluster_smem_bytes(bk, R | 1) > 220 * 1024) return 0;
  return R;
}

cudaError_t launch_panel_cluster(const PanelParams* single, const PanelParams* dev_probs, int nprob, int C, int Rp_max,
                                 int bk_max, cudaStream_t s) {
  static int configured_device = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_device != dev) {
    cudaError_t e = cudaFuncSetAttribute(panel_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(panel_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    if (e != cudaSuccess) return e;
    configured_device = dev;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, nprob, 1);
  cfg.blockDim = dim3(kPanelThreads, 1, 1);
  cfg.dynamicSmemBytes = panel_cluster_smem_bytes(bk_max, Rp_max);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  PanelParams none{};
  prof::count_launch();
  return cudaLaunchKernelEx(&cfg, panel_cluster_kernel, single ? *single : none, dev_probs);
}

}  // namespace bandred
