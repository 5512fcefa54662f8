// Panel factorisation in FP64 with up to four reflectors per grid-wide reduction: the same
// outputs as panel_qr_kernel (packed reflectors, tau, Y, W = -Y T; Eq. updateA0 of
// Section 2.1, Eqs. updateB and updateC of Section 3.1), with half its grid barriers.
//
// A step at column i takes the block of mt <= 4 columns a_0 .. a_{mt-1} (columns i ..
// i+mt-1).  Rows i .. i+mt-1 are the block's explicit rows; rows below them are the tail.
// One reduction gives, for every panel column c, the sums G(q, c) = t_q . t_c over the tail
// rows (t_x: the tail of column x) and the explicit rows of c.  Every Householder quantity
// of the block then follows from these numbers alone: after reflectors 0 .. k-1 a block
// column's tail is t_q + sum_p lam(q, p) t_p, so its norm and its inner products with any
// column are bilinear forms in G.  Reflector k is taken only while its tail norm keeps at
// least 1/8 of the sum of the squared norms it is formed from (the terms that cancel), so
// its relative error stays a small multiple of the unit roundoff; otherwise the step ends
// after k reflectors and the next reduction starts fresh.  A column c then moves by the
// block's compact-WY factor: w = V^T c (four independent dot products), z = T^T w,
// c -= V z, which on the tail rows is c_r += sum_p l(c, p) t_p[r].
#include <cmath>

#include "panel_common.cuh"
#include "prof.h"

namespace bandred {

namespace {

using namespace panel_detail;

constexpr int MB = 4;  // reflectors per reduction, at most

__global__ void __launch_bounds__(kPanelThreads, 1) panel_qr4_kernel(PanelParams p) {
  extern __shared__ double smem[];
  constexpr int NT = kPanelThreads;
  const int tid = threadIdx.x, lane = tid & 31;
  const int G = gridDim.x, g = blockIdx.x;
  const int bk = p.bk, Rp = p.Rp;
  const int rb = g * p.R;
  const int nr = max(0, min(p.R, p.j - rb));
  double* slab = smem;                                 // bk columns x Rp rows
  double* dsum = slab + (size_t)bk * Rp;               // G(q, c) at dsum[q bk + c]; max |tail of a_0| at MB bk
  double* top = dsum + MB * bk + 2;                    // explicit rows: top[s bk + c]
  double* gq = top + MB * bk;                          // y_c . y_{i+k} at gq[k bk + c] (for W)
  double* lcs = gq + MB * bk;                          // tail coefficients l(c, p) at lcs[c MB + p]
  float* gqf = reinterpret_cast<float*>(lcs + MB * bk);  // gq in FP32
  double* after = lcs + MB * bk + (MB * bk + 1) / 2;
  const bool wf32 = p.w_in_smem && p.w_fp32;
  double* wl = p.w_in_smem ? after : p.W + rb;
  float* wlf = reinterpret_cast<float*>(after);
  const int64_t wld = p.w_in_smem ? Rp : p.ldy;
  // the step's reflectors: beta, tau, scal; v_k on the explicit rows (s_v[k][s], s > k);
  // v_k's tail as a combination of the block tails (s_coef[k][p], p <= k); block column k
  // on the explicit rows at the time of reflector k (s_tb); the block's T factor (s_T)
  __shared__ double s_beta[MB], s_tau[MB], s_scal[MB], s_v[MB][MB], s_coef[MB][MB], s_tb[MB][MB], s_T[MB][MB];
  __shared__ double s_ptau[MB];
  __shared__ double s_amax, s_dfac;
  __shared__ int s_rescale, s_ok, s_meff;
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

  // W columns of the previous step's reflectors (all = false: warps 1..7, named barrier 1
  // between the columns, while thread 0 derives the next reflectors)
  auto pending_w = [&](int npend, int pi, bool all) {
    const int t0 = all ? 0 : 32, nth = all ? NT : NT - 32;
    for (int q = 0; q < npend; ++q) {
      if (q) {
        if (all)
          __syncthreads();
        else
          asm volatile("bar.sync 1, %0;" ::"r"(NT - 32) : "memory");
      }
      if (wf32)
        w_column_f32(pi + q, (float)s_ptau[q], gqf + q * bk, slab, Rp, rb, nr, wlf, t0, nth);
      else
        w_column(pi + q, s_ptau[q], gq + q * bk, slab, Rp, rb, nr, wl, wld, t0, nth);
    }
  };

  const int TPC = bk >= 128 ? 2 : (bk >= 64 ? 4 : 8);  // threads per column in the sums
  const int CPP = NT / TPC;
  const int sub = tid % TPC;
  const size_t accsz = panel_acc_entries(bk) * kAccStride;
  unsigned int gen = 0;
  int npend = 0, pend_i = 0;
  for (int i = 0, step = 0; i < bk; ++step) {
    int mt = min(MB, min(bk - i, p.j - i - 1));  // the tail must have rows
    if (mt < 1) mt = 1;
    double* acc = p.acc + (size_t)(step % 3) * accsz;
    double* rowg = p.rowbuf + (size_t)(step & 1) * MB * bk;
    const int lo = min(max(i + mt - rb, 0), nr);  // this CTA's first tail row
    const double* x0 = slab + (size_t)i * Rp;
    const double* x1 = slab + (size_t)(i + min(1, mt - 1)) * Rp;
    const double* x2 = slab + (size_t)(i + min(2, mt - 1)) * Rp;
    const double* x3 = slab + (size_t)(i + min(3, mt - 1)) * Rp;
    if (g == 0) {  // clear the buffer of the next step (last read two steps ago)
      double* nxt = p.acc + (size_t)((step + 1) % 3) * accsz;
      for (int v = tid; v < MB * bk + 2; v += NT) nxt[(size_t)v * kAccStride] = 0.0;
      for (int v = tid; v < bk; v += NT) nxt[(size_t)(kRescaleSlot * bk + 2 + v) * kAccStride] = 0.0;
    }

    // ---- tail sums of the block columns against every column, added into L2
    for (int c0 = 0; c0 < bk; c0 += CPP) {
      const int c = c0 + tid / TPC;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      if (c < bk) {
        const double* ac = slab + (size_t)c * Rp;
        if (mt == 4) {
          for (int r = lo + sub; r < nr; r += TPC) {
            const double v = ac[r];
            s0 = fma(x0[r], v, s0);
            s1 = fma(x1[r], v, s1);
            s2 = fma(x2[r], v, s2);
            s3 = fma(x3[r], v, s3);
          }
        } else {
          for (int r = lo + sub; r < nr; r += TPC) {
            const double v = ac[r];
            s0 = fma(x0[r], v, s0);
            if (mt > 1) s1 = fma(x1[r], v, s1);
            if (mt > 2) s2 = fma(x2[r], v, s2);
          }
        }
      }
      for (int o = TPC / 2; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s3 += __shfl_xor_sync(0xffffffffu, s3, o);
      }
      if (sub == 0 && c < bk) {
        atomicAdd(&acc[(size_t)c * kAccStride], s0);
        if (mt > 1) atomicAdd(&acc[(size_t)(bk + c) * kAccStride], s1);
        if (mt > 2) atomicAdd(&acc[(size_t)(2 * bk + c) * kAccStride], s2);
        if (mt > 3) atomicAdd(&acc[(size_t)(3 * bk + c) * kAccStride], s3);
      }
    }
    // max |tail of a_0| by integer comparison of the bit patterns: one warp
    if (tid < 32) {
      unsigned long long m = 0ull;
      for (int r = lo + lane; r < nr; r += 32) {
        const unsigned long long u = (unsigned long long)__double_as_longlong(x0[r]) & 0x7FFFFFFFFFFFFFFFull;
        m = u > m ? u : m;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v > m ? v : m;
      }
      if (lane == 0) atomicMax(reinterpret_cast<unsigned long long*>(&acc[(size_t)MB * bk * kAccStride]), m);
    }
    // explicit rows, published by the CTAs that own them
    for (int s = 0; s < mt; ++s)
      if (i + s >= rb && i + s < rb + nr)
        for (int c = tid; c < bk; c += NT) __stcg(&rowg[s * bk + c], slab[(size_t)c * Rp + (i + s - rb)]);
    __syncthreads();
    if (tid == 0) grid_arrive(p.gs);
    ++gen;
    if (tid == 0) s_ok = grid_wait(p.gs, gen, p.extra, p.status, p.limit_ns) ? 1 : 0;
    __syncthreads();
    if (!s_ok) return;

    // ---- thread 0 derives the block's reflectors; warps 1..7 fetch the sums and rows and
    // form the previous step's W columns
    if (tid == 0) {
      double tb[MB][MB], Gb[MB][MB], lam[MB][MB];
#pragma unroll
      for (int q = 0; q < MB; ++q)
#pragma unroll
        for (int s = 0; s < MB; ++s) {
          tb[q][s] = (q < mt && s < mt) ? ldcg(&rowg[s * bk + i + q]) : 0.0;
          Gb[q][s] = (q < mt && s < mt) ? ldcg(&acc[(size_t)(q * bk + i + s) * kAccStride]) : 0.0;
          lam[q][s] = 0.0;
        }
      const double amax_t = __longlong_as_double(
          (long long)__ldcg(reinterpret_cast<const unsigned long long*>(&acc[(size_t)MB * bk * kAccStride])));
      double amax = amax_t, ex = 0.0;
#pragma unroll
      for (int s = 1; s < MB; ++s)
        if (s < mt) {
          amax = fmax(amax, fabs(tb[0][s]));
          ex = fma(tb[0][s], tb[0][s], ex);
        }
      const double ssq = Gb[0][0] + ex;
      const int rescale = (p.j - i > 1) && (amax > 0.0) && !(ssq < 0x1p1000 && amax > 0x1p-450);
      s_rescale = rescale || !(fabs(tb[0][0]) < 0x1p500);
      s_amax = amax;
      s_dfac = 1.0;
#pragma unroll
      for (int k = 0; k < MB; ++k)
#pragma unroll
        for (int s = 0; s < MB; ++s) {
          s_v[k][s] = 0.0;
          s_coef[k][s] = 0.0;
          s_tb[k][s] = tb[k][s];
          s_T[k][s] = 0.0;
        }
      int meff = 0;
      if (!s_rescale) {
#pragma unroll
        for (int k = 0; k < MB; ++k) {
          if (k >= mt) break;
          double e[MB];
#pragma unroll
          for (int q = 0; q < MB; ++q) e[q] = lam[k][q] + (q == k ? 1.0 : 0.0);
          double n2t = 0.0, bound = 0.0;
#pragma unroll
          for (int q = 0; q < MB; ++q) {
            double row = 0.0;
#pragma unroll
            for (int r = 0; r < MB; ++r) row = fma(Gb[q][r], e[r], row);
            n2t = fma(e[q], row, n2t);
            bound = fma(e[q] * e[q], Gb[q][q], bound);
          }
          double xn2 = n2t;
#pragma unroll
          for (int s = 0; s < MB; ++s)
            if (s > k && s < mt) xn2 = fma(tb[k][s], tb[k][s], xn2);
          const double alpha = tb[k][k];
          if (k > 0 && !(n2t > 0.125 * bound && xn2 < 0x1p1000 && xn2 > 0x1p-900 && fabs(alpha) < 0x1p500)) break;
          // reflector k (beta = -sign(alpha) ||x||, tau = 1 + |alpha| / ||x||,
          // scal = 1 / (alpha - beta)); tau = 0 for an empty or zero x2
          double tau = 0.0, beta = alpha, scal = 1.0;
          if (p.j - (i + k) > 1 && xn2 != 0.0) {
            const double qv = fma(alpha, alpha, xn2);
            const double rq = rsqrt_newton(qv);
            const double h = qv * rq;
            const double aa = fabs(alpha);
            beta = (alpha >= 0.0) ? -h : h;
            tau = fma(aa, rq, 1.0);
            const double rs = rcp_newton(aa + h);
            scal = (alpha >= 0.0) ? rs : -rs;
          }
          s_beta[k] = beta;
          s_tau[k] = tau;
          s_scal[k] = scal;
#pragma unroll
          for (int s = 0; s < MB; ++s) {
            s_v[k][s] = (s > k && s < mt) ? scal * tb[k][s] : 0.0;
            s_coef[k][s] = scal * e[s];
            s_tb[k][s] = tb[k][s];
          }
          meff = k + 1;
          // y_{i+q} . y_{i+k} for q < k (the in-block entries of W's g vector) and column k
          // of the block's T factor: T(q, k) = -tau_k sum_{q <= r < k} T(q, r) g(r)
          double gb[MB];
#pragma unroll
          for (int q = 0; q < MB; ++q) {
            gb[q] = 0.0;
            if (q < k) {
              double d = s_v[q][k];
#pragma unroll
              for (int s = 0; s < MB; ++s)
                if (s > k) d = fma(s_v[q][s], s_v[k][s], d);
              double cg = 0.0;
#pragma unroll
              for (int a = 0; a < MB; ++a) {
                double row = 0.0;
#pragma unroll
                for (int b2 = 0; b2 < MB; ++b2) row = fma(Gb[a][b2], s_coef[k][b2], row);
                cg = fma(s_coef[q][a], row, cg);
              }
              gb[q] = d + cg;
              gq[k * bk + i + q] = gb[q];
              gqf[k * bk + i + q] = f64_to_f32_rz(gb[q]);
            }
          }
          s_T[k][k] = tau;
#pragma unroll
          for (int q = 0; q < MB; ++q)
            if (q < k) {
              double t = 0.0;
#pragma unroll
              for (int r = 0; r < MB; ++r)
                if (r >= q && r < k) t = fma(s_T[q][r], gb[r], t);
              s_T[q][k] = -tau * t;
            }
          // the block columns after k move by H_k
#pragma unroll
          for (int q = 0; q < MB; ++q) {
            if (q <= k || q >= mt) continue;
            double eq[MB];
#pragma unroll
            for (int r = 0; r < MB; ++r) eq[r] = lam[q][r] + (r == q ? 1.0 : 0.0);
            double d = tb[q][k];
#pragma unroll
            for (int s = 0; s < MB; ++s)
              if (s > k) d = fma(s_v[k][s], tb[q][s], d);
#pragma unroll
            for (int a = 0; a < MB; ++a) {
              double row = 0.0;
#pragma unroll
              for (int b2 = 0; b2 < MB; ++b2) row = fma(Gb[a][b2], eq[b2], row);
              d = fma(s_coef[k][a], row, d);
            }
            const double z = tau * d;
            tb[q][k] -= z;
#pragma unroll
            for (int s = 0; s < MB; ++s)
              if (s > k) tb[q][s] = fma(-z, s_v[k][s], tb[q][s]);
#pragma unroll
            for (int r = 0; r < MB; ++r) lam[q][r] = fma(-z, s_coef[k][r], lam[q][r]);
          }
        }
      }
      s_meff = meff;
    } else if (tid >= 32) {
      for (int v = tid - 32; v < mt * bk; v += NT - 32) {
        dsum[v] = ldcg(&acc[(size_t)v * kAccStride]);
        top[v] = ldcg(&rowg[v]);
      }
      pending_w(npend, pend_i, false);
    }
    // A tail sum outside the range where the plain formulas hold (not finite, or near the
    // overflow threshold) forces the scaled path too.
    int bad = 0;
    if (tid >= 32)
      for (int v = tid - 32; v < mt * bk; v += NT - 32) bad |= !(fabs(dsum[v]) < 0x1p1000);
    const int force = __syncthreads_or(bad);

    // Rare path: the plain sums of reflector 0 over/underflow (or |alpha| is huge).  Column
    // i is scaled by the power of two 2^-e with 2^e <= max|x2| < 2^(e+1) (exact), and a
    // second reduction forms the tail's ||x 2^-e||^2 and the tail dot products
    // (x 2^-e)^T a_c of every column; the dot terms then take the factor 2^e (s_dfac).
    // One reflector this step.
    if (s_rescale || force) {
      const int e = s_amax > 0.0 ? max(-1022, min(1022, ilogb(s_amax))) : 0;
      const double inv = ldexp(1.0, -e), sc = ldexp(1.0, e);
      double* resc = acc + (size_t)(kRescaleSlot * bk + 2) * kAccStride;
      for (int c0 = 0; c0 < bk; c0 += CPP) {
        const int c = c0 + tid / TPC;
        double sv = 0.0;
        if (c < bk) {
          const double* ac = slab + (size_t)c * Rp;
          for (int r = lo + sub; r < nr; r += TPC) {
            const double t = x0[r] * inv;
            sv = fma(t, c == i ? t : ac[r], sv);
          }
        }
        for (int o = TPC / 2; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
        if (sub == 0 && c < bk) atomicAdd(&resc[(size_t)c * kAccStride], sv);
      }
      if (!grid_barrier(p.gs, ++gen, p.extra, p.status, p.limit_ns)) return;
      for (int c = tid; c < bk; c += NT) dsum[c] = ldcg(&resc[(size_t)c * kAccStride]);
      __syncthreads();
      if (tid == 0) {
        double t = dsum[i];
        for (int sr = 1; sr < mt; ++sr) {
          const double u = top[sr * bk + i] * inv;
          t = fma(u, u, t);
        }
        const double xnorm = s_amax > 0.0 ? sqrt(t) * sc : 0.0;
        const double alpha = top[i];
        double tau = 0.0, beta = alpha, scal = 1.0;
        if (p.j - i > 1 && xnorm != 0.0) {
          const double h = hypot(alpha, xnorm);
          beta = (alpha >= 0.0) ? -h : h;
          tau = (beta - alpha) / beta;
          scal = 1.0 / (alpha - beta);
        }
        s_beta[0] = beta;
        s_tau[0] = tau;
        s_scal[0] = scal;
        for (int k = 0; k < MB; ++k)
          for (int sr = 0; sr < MB; ++sr) {
            s_v[k][sr] = (k == 0 && sr > 0 && sr < mt) ? scal * top[sr * bk + i] : 0.0;
            s_coef[k][sr] = (k == 0 && sr == 0) ? scal : 0.0;
            s_tb[k][sr] = (k == 0 && sr < mt) ? top[sr * bk + i] : 0.0;
            s_T[k][sr] = 0.0;
          }
        s_T[0][0] = tau;
        s_dfac = sc;
        s_meff = 1;
      }
      __syncthreads();
    }
    const int meff = s_meff;
    if (tid == 0 && g == 0)
      for (int k = 0; k < meff; ++k) p.tau[i + k] = s_tau[k];

    // ---- every column: w = V^T c (lane k of a group of four), z = T^T w; columns right of
    // the block get their explicit rows and tail coefficients, columns left of it the W dots
    const double dfac = s_dfac;
    for (int c0 = 0; c0 < bk; c0 += NT / MB) {
      const int c = c0 + tid / MB, t = tid % MB;
      const bool in = c < bk && !(c >= i && c < i + meff);
      double w = 0.0;
      if (in && t < meff) {
        w = top[t * bk + c];
#pragma unroll
        for (int s = 0; s < MB; ++s)
          if (s > t && s < mt) w = fma(s_v[t][s], top[s * bk + c], w);
#pragma unroll
        for (int q = 0; q < MB; ++q)
          if (q <= t) w = fma(q == 0 ? s_coef[t][0] * dfac : s_coef[t][q], dsum[q * bk + c], w);
      }
      if (in && c < i && t < meff) {
        gq[t * bk + c] = w;
        gqf[t * bk + c] = f64_to_f32_rz(w);
      }
      const int base = lane & ~(MB - 1);
      double wv[MB];
#pragma unroll
      for (int k = 0; k < MB; ++k) wv[k] = __shfl_sync(0xffffffffu, w, base + k);
      double z = 0.0;
#pragma unroll
      for (int q = 0; q < MB; ++q)
        if (q <= t && t < meff) z = fma(s_T[q][t], wv[q], z);
      double zv[MB];
#pragma unroll
      for (int k = 0; k < MB; ++k) zv[k] = __shfl_sync(0xffffffffu, z, base + k);
      if (in && c >= i + meff) {
        if (t < mt) {  // explicit row i + t
          double nt = top[t * bk + c];
#pragma unroll
          for (int k = 0; k < MB; ++k)
            if (k < meff && k <= t) nt = fma(-zv[k], k == t ? 1.0 : s_v[k][t], nt);
          if (i + t >= rb && i + t < rb + nr) slab[(size_t)c * Rp + (i + t - rb)] = nt;
        }
        double l = 0.0;
#pragma unroll
        for (int k = 0; k < MB; ++k)
          if (k < meff) l = fma(-zv[k], s_coef[k][t], l);
        lcs[c * MB + t] = l;
      }
    }
    __syncthreads();

    // ---- tail rows of the columns right of the block: c_r += sum_p l(c, p) t_p[r]
    {
      const int TPU = TPC;
      for (int c0 = 0; c0 < bk; c0 += NT / TPU) {
        const int c = c0 + tid / TPU, rg = tid % TPU;
        if (c >= i + meff && c < bk) {
          const double l0 = lcs[c * MB], l1 = lcs[c * MB + 1], l2 = lcs[c * MB + 2], l3 = lcs[c * MB + 3];
          double* ac = slab + (size_t)c * Rp;
          if (meff == 4) {
            for (int r = lo + rg; r < nr; r += TPU)
              ac[r] = fma(l3, x3[r], fma(l2, x2[r], fma(l1, x1[r], fma(l0, x0[r], ac[r]))));
          } else if (meff == 3) {
            for (int r = lo + rg; r < nr; r += TPU) ac[r] = fma(l2, x2[r], fma(l1, x1[r], fma(l0, x0[r], ac[r])));
          } else if (meff == 2) {
            for (int r = lo + rg; r < nr; r += TPU) ac[r] = fma(l1, x1[r], fma(l0, x0[r], ac[r]));
          } else {
            for (int r = lo + rg; r < nr; r += TPU) ac[r] = fma(l0, x0[r], ac[r]);
          }
        }
      }
    }
    __syncthreads();
    // ---- the block columns become v_0 .. v_{meff-1}: tails from the original block tails,
    // explicit rows from the reflectors (R above the diagonal, beta on it, v below)
    for (int r = lo + tid; r < nr; r += NT) {
      const double a0 = x0[r], a1 = x1[r], a2 = x2[r], a3 = x3[r];
      slab[(size_t)i * Rp + r] = s_coef[0][0] * a0;
      if (meff > 1) slab[(size_t)(i + 1) * Rp + r] = fma(s_coef[1][1], a1, s_coef[1][0] * a0);
      if (meff > 2) slab[(size_t)(i + 2) * Rp + r] = fma(s_coef[2][2], a2, fma(s_coef[2][1], a1, s_coef[2][0] * a0));
      if (meff > 3)
        slab[(size_t)(i + 3) * Rp + r] =
            fma(s_coef[3][3], a3, fma(s_coef[3][2], a2, fma(s_coef[3][1], a1, s_coef[3][0] * a0)));
    }
    if (tid < MB * MB) {
      const int k = tid / MB, s = tid % MB;
      if (k < meff && s < mt && i + s >= rb && i + s < rb + nr) {
        const double v = s < k ? s_tb[k][s] : (s == k ? s_beta[k] : s_v[k][s]);
        slab[(size_t)(i + k) * Rp + (i + s - rb)] = v;
      }
    }
    if (tid < MB) s_ptau[tid] = s_tau[tid];
    npend = meff;
    pend_i = i;
    i += meff;
    __syncthreads();
  }
  pending_w(npend, pend_i, true);
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

  // write back: packed reflectors/R into the matrix, Y into the workspace
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
  __syncthreads();
  trace_end(p.trace);
}

}  // namespace

size_t panel4_smem_bytes(int bk, int Rp, bool w_in_smem) {
  return ((size_t)bk * Rp * (w_in_smem ? 2 : 1) + 4 * (size_t)MB * bk + (MB * bk + 1) / 2 + 2) * sizeof(double);
}

cudaError_t launch_panel4(const PanelParams& prm, int G, cudaStream_t s) {
  static int configured_device = -1;
  static size_t max_dynamic = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_device != dev) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, panel_qr4_kernel);
    if (e != cudaSuccess) return e;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    max_dynamic = (size_t)optin - fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(panel_qr4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_dynamic);
    if (e != cudaSuccess) return e;
    configured_device = dev;
  }
  const size_t smem = panel4_smem_bytes(prm.bk, prm.Rp, prm.w_in_smem);
  if (smem > max_dynamic) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(prm.gs, 0, panel_sync_bytes(prm.bk), s);
  if (e != cudaSuccess) return e;
  PanelParams p = prm;
  void* args[] = {&p};
  prof::count_launch();
  return cudaLaunchCooperativeKernel((const void*)panel_qr4_kernel, dim3(G), dim3(kPanelThreads), args, smem, s);
}

}  // namespace bandred
