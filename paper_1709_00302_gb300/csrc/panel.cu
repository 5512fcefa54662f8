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
//   Reflectors are taken two per grid-wide reduction when the second one's norm can be
//   updated without cancellation (H_i is orthogonal, so the sums of column i + 1 against
//   the panel determine those of H_i applied to it): half the barriers, the same FMAs.
//   W's column i follows from the recurrence W(:, i) = -tau_i (y_i + W(:, 0:i) Y(:, 0:i)^T y_i),
//   which equals -Y T with T built column by column as in the compact-WY definition.
#include <cmath>

#include "launch.h"
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
  double* dsum = slab + (size_t)bk * Rp;      // 2 bk + 2 combined sums (S_a, max|x2|, S_b)
  double* rowi = dsum + 2 * bk + 2;           // row i of the panel (before the step)
  double* rowi1 = rowi + bk;                  // row i + 1 (paired steps)
  double* gq0 = rowi1 + bk;                   // Y^T y of the step's first reflector (for W)
  double* gq1 = gq0 + bk;                     // ... and of its second
  float* gqf0 = reinterpret_cast<float*>(gq1 + bk);  // the same in FP32 (bk floats each)
  float* gqf1 = gqf0 + bk;
  double* after = gq1 + 2 * bk;
  // This CTA's rows of W: in shared memory when they fit (FP32 when p.w_fp32), else in
  // the W output itself.
  const bool wf32 = p.w_in_smem && p.w_fp32;
  // gram: no W in the panel; CTA 0 stores the T coefficients (y_c^T y_i) into p.G instead
  const bool gram = p.G != nullptr;
  double* wl = p.w_in_smem ? after : p.W + rb;
  float* wlf = reinterpret_cast<float*>(after);
  const int64_t wld = p.w_in_smem ? Rp : p.ldy;
  __shared__ double s_beta, s_tau, s_scal, s_dscal, s_beta2, s_tau2, s_scal2, s_zb, s_Taa, s_Tab;
  __shared__ double s_ptau[2];
  __shared__ int s_rescale, s_ok, s_pair;
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

  // W columns of the previous step's reflectors (their T entries are in gq0 / gq1).
  // all = false: warps 1..7 only (named barrier 1 between the columns), while thread 0
  // waits at the grid barrier.
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
        w_column_f32(pi + q, (float)s_ptau[q], q ? gqf1 : gqf0, slab, Rp, rb, nr, wlf, t0, nth);
      else
        w_column(pi + q, s_ptau[q], q ? gq1 : gq0, slab, Rp, rb, nr, wl, wld, t0, nth);
    }
  };

  // Threads per column in the dot products (a power of two dividing 32).
  const int TPC = bk >= 128 ? 2 : (bk >= 64 ? 4 : 8);
  const int CPP = NT / TPC;  // columns per pass
  const int sub = tid % TPC;
  const size_t accsz = panel_acc_entries(bk) * kAccStride;
  unsigned int gen = 0;
  int npend = 0, pend_i = 0;
  // phase timing (diagnostic): CTA 0's thread 0 records clock64 at the points of a step
  auto stamp = [&](int step, int q) {
    if (p.phases && g == 0 && tid == 0 && step < p.phase_steps) p.phases[step * 8 + q] = clock64();
  };
  for (int i = 0, step = 0; i < bk; ++step) {
    stamp(step, 0);
    // A paired step computes reflectors i and i + 1 from one grid-wide reduction: the
    // sums over the rows below row i of column i and of column i + 1 against every
    // column; the second reflector's norm and coefficients follow from them and rows i,
    // i + 1 by the orthogonality of the first (see the pair branch below).
    const bool want_pair = (i + 1 < bk) && (p.j - i - 2 >= 1);
    double* acc = p.acc + (size_t)(step % 3) * accsz;
    double* rowg = p.rowbuf + (size_t)(step & 1) * 2 * bk;
    const int lo = min(max(i + 1 - rb, 0), nr);
    double* xa = slab + (size_t)i * Rp;
    double* xb = slab + (size_t)(want_pair ? i + 1 : i) * Rp;
    const bool own0 = (i >= rb) && (i < rb + nr);
    const bool own1 = (i + 1 >= rb) && (i + 1 < rb + nr);
    if (g == 0) {  // clear the buffer of the next step (last read two steps ago)
      double* nxt = p.acc + (size_t)((step + 1) % 3) * accsz;
      for (int v = tid; v < 2 * bk + 2; v += NT) nxt[(size_t)v * kAccStride] = 0.0;
      for (int v = tid; v < bk; v += NT) nxt[(size_t)(kRescaleSlot * bk + 2 + v) * kAccStride] = 0.0;
    }

    // Partial dot products over this CTA's rows below row i, added into L2 accumulators.
    for (int c0 = 0; c0 < bk; c0 += CPP) {
      const int c = c0 + tid / TPC;
      double sa = 0.0, ta = 0.0, sbv = 0.0, tbv = 0.0;
      if (c < bk) {
        const double* ac = slab + (size_t)c * Rp;
        int r = lo + sub;
        if (want_pair) {
          for (; r + TPC < nr; r += 2 * TPC) {
            const double v0 = ac[r], v1 = ac[r + TPC];
            sa = fma(xa[r], v0, sa);
            sbv = fma(xb[r], v0, sbv);
            ta = fma(xa[r + TPC], v1, ta);
            tbv = fma(xb[r + TPC], v1, tbv);
          }
          if (r < nr) {
            sa = fma(xa[r], ac[r], sa);
            sbv = fma(xb[r], ac[r], sbv);
          }
        } else {
          for (; r + TPC < nr; r += 2 * TPC) {
            sa = fma(xa[r], ac[r], sa);
            ta = fma(xa[r + TPC], ac[r + TPC], ta);
          }
          if (r < nr) sa = fma(xa[r], ac[r], sa);
        }
      }
      sa += ta;
      sbv += tbv;
      for (int o = TPC / 2; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        if (want_pair) sbv += __shfl_xor_sync(0xffffffffu, sbv, o);
      }
      if (sub == 0 && c < bk) {
        atomicAdd(&acc[(size_t)c * kAccStride], sa);
        if (want_pair) atomicAdd(&acc[(size_t)(bk + 1 + c) * kAccStride], sbv);
      }
    }
    stamp(step, 1);
    // max |x2| by integer comparison of the bit patterns (no FP64 instruction): one warp
    if (tid < 32) {
      unsigned long long m = 0ull;
      for (int r = lo + lane; r < nr; r += 32) {
        const unsigned long long u = (unsigned long long)__double_as_longlong(xa[r]) & 0x7FFFFFFFFFFFFFFFull;
        m = u > m ? u : m;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v > m ? v : m;
      }
      if (lane == 0) atomicMax(reinterpret_cast<unsigned long long*>(&acc[(size_t)bk * kAccStride]), m);
    }
    if (own0)
      for (int c = tid; c < bk; c += NT) __stcg(&rowg[c], slab[(size_t)c * Rp + (i - rb)]);
    if (want_pair && own1)
      for (int c = tid; c < bk; c += NT) __stcg(&rowg[bk + c], slab[(size_t)c * Rp + (i + 1 - rb)]);
    __syncthreads();
    stamp(step, 2);
    if (tid == 0) grid_arrive(p.gs);
    ++gen;
    // While thread 0 waits for the barrier, warps 1..7 form the W columns of the previous
    // step: the FP64 pipe is otherwise idle here, and kept off the scalar chain after it.
    if (tid == 0)
      s_ok = grid_wait(p.gs, gen, p.extra, p.status, p.limit_ns) ? 1 : 0;
    else if (tid >= 32 && !gram)
      pending_w(npend, pend_i, false);
    npend = 0;
    stamp(step, 3);
    __syncthreads();
    if (!s_ok) return;

    // Thread 0 derives the reflector(s) from a few sums while warps 1..7 fetch the rest.
    if (tid == 0) {
      // every sum and row entry thread 0 needs, loaded at once (one round trip to L2);
      // the pair's are read even when the step takes one reflector (valid addresses)
      const double alpha = ldcg(&rowg[i]);
      const double ssq = ldcg(&acc[(size_t)i * kAccStride]);
      const double amax = ldcg(&acc[(size_t)bk * kAccStride]);
      const double Sab = ldcg(&acc[(size_t)(i + 1) * kAccStride]);
      const double Sbb = ldcg(&acc[(size_t)(bk + 2 + i) * kAccStride]);
      const double bi = ldcg(&rowg[i + 1]), ai1 = ldcg(&rowg[bk + i]), bi1 = ldcg(&rowg[bk + i + 1]);
      const long long us = dbits(ssq), um = dbits(amax);  // amax >= 0 (an integer maximum)
      const int rescale = (p.j - i > 1) && (um > 0) && !(us >= 0 && us < kBits2p1000 && um > kBits2m450);
      s_rescale = rescale || !(abits(alpha) < kBits2p500);
      // Common path: h = ||[alpha; x2]|| = q / sqrt(q) with q = alpha^2 + ||x2||^2 (no
      // overflow: both terms are bounded here); tau = (beta - alpha) / beta = 1 + |alpha|/h
      // and scal = 1 / (alpha - beta) = sign(alpha) / (|alpha| + h).
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
      // Second reflector.  With a = column i, b = column i + 1 and sums over rows >= i + 1
      // (S_aa, S_ab, S_bb), H_i b = b - z_b v_i has z_b = tau (b_i + scal S_ab); below row
      // i + 1 its entries are b_r - zs a_r (zs = z_b scal), so their squared norm is
      //   n2 = T_bb - 2 zs T_ab + zs^2 T_aa,  T_xy = S_xy - x_{i+1} y_{i+1},
      // and the new diagonal entry is b_{i+1} - zs a_{i+1}.  The step is paired only when
      // n2 keeps at least 1/8 of S_bb + zs^2 S_aa (a bound on the terms that cancel), so
      // its relative error stays a small multiple of the unit roundoff; otherwise the
      // step takes reflector i alone and the next step starts from a fresh reduction.
      int pair = 0;
      if (want_pair && !s_rescale) {
        const double zb = tau * fma(scal, Sab, bi);
        const double zs = zb * scal;
        const double Taa = fma(-ai1, ai1, ssq), Tab = fma(-ai1, bi1, Sab), Tbb = fma(-bi1, bi1, Sbb);
        const double n2 = fma(zs * zs, Taa, fma(-2.0 * zs, Tab, Tbb));
        const double alpha2 = fma(-zs, ai1, bi1);
        const double bound = fma(zs * zs, ssq, Sbb);
        // n2 > bound / 8 (bound >= 0: the pattern of bound / 8 is bound's minus 3 in the
        // exponent; when that underflows, n2 > 2^-900 decides as the FP64 test would)
        const long long un2 = dbits(n2), ub = dbits(bound);
        if (un2 > kBits2m900 && un2 < kBits2p1000 && un2 > ub - (3LL << 52) && abits(alpha2) < kBits2p500) {
          const double q = fma(alpha2, alpha2, n2);
          const double rq = rsqrt_newton(q);
          const double h = q * rq;
          const double aa = fabs(alpha2);
          const bool apos = nonneg(alpha2);
          s_beta2 = neg_if(h, apos);
          s_tau2 = fma(aa, rq, 1.0);
          const double rs = rcp_newton(aa + h);
          s_scal2 = neg_if(rs, !apos);
          s_zb = zb;
          s_Taa = Taa;
          s_Tab = Tab;
          pair = 1;
        }
      }
      s_pair = pair;
    } else if (tid >= 32) {
      const int nsum = want_pair ? 2 * bk + 1 : bk + 1;
      for (int v = tid - 32; v < nsum; v += NT - 32) dsum[v] = ldcg(&acc[(size_t)v * kAccStride]);
      for (int c = tid - 32; c < bk; c += NT - 32) rowi[c] = ldcg(&rowg[c]);
      if (want_pair)
        for (int c = tid - 32; c < bk; c += NT - 32) rowi1[c] = ldcg(&rowg[bk + c]);
    }
    // A sum outside the range where the plain formulas hold (not finite, or near the
    // overflow threshold, as when some entries exceed 2^500) forces the scaled path too.
    int bad = 0;
    if (tid >= 32) {
      const int nsum = want_pair ? 2 * bk + 1 : bk + 1;
      for (int v = tid - 32; v < nsum; v += NT - 32) bad |= !(abits(dsum[v]) < kBits2p1000);
    }
    const int force = __syncthreads_or(bad);
    stamp(step, 4);

    // Rare path: the plain sums over/underflow (or |alpha| is huge).  Column i is scaled
    // by the power of two 2^-e with 2^e <= max|x2| < 2^(e+1) (exact), and a second
    // reduction forms ||x2 2^-e||^2 and the dot products (x2 2^-e)^T a_c of every column,
    // so no square or product leaves the range; the coefficients then take scal 2^e for
    // the dot terms.  One reflector this step.  Same decision in every CTA.
    if (s_rescale || force) {
      const double amax = dsum[bk];
      const int e = amax > 0.0 ? max(-1022, min(1022, ilogb(amax))) : 0;
      const double inv = ldexp(1.0, -e), sc = ldexp(1.0, e);
      double* resc = acc + (size_t)(kRescaleSlot * bk + 2) * kAccStride;
      for (int c0 = 0; c0 < bk; c0 += CPP) {
        const int c = c0 + tid / TPC;
        double sv = 0.0;
        if (c < bk) {
          const double* ac = slab + (size_t)c * Rp;
          for (int r = lo + sub; r < nr; r += TPC) {
            const double t = xa[r] * inv;
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
        s_pair = 0;
      }
      __syncthreads();
    }
    const bool paired = s_pair != 0;
    if (tid == 0 && g == 0) {
      p.tau[i] = s_tau;
      if (paired) p.tau[i + 1] = s_tau2;
    }

    const double tau = s_tau, scal = s_scal, dscal = s_dscal;
    const int TPU = bk >= 128 ? 2 : (bk >= 64 ? 4 : 8);
    if (!paired) {
      // Coefficients and the in-panel update, one column per group of TPU threads:
      // z_c = tau v^T a_c, a_c -= z_c v (c > i); and (Y^T y_i)_c for c < i (for W).
      for (int c0 = 0; c0 < bk; c0 += NT / TPU) {
        const int c = c0 + tid / TPU, rg = tid % TPU;
        if (c > i && c < bk) {
          const double z = tau * fma(dscal, dsum[c], rowi[c]);
          if (tau != 0.0) {
            const double z2 = -z * scal;
            double* ac = slab + (size_t)c * Rp;
            for (int r = lo + rg; r < nr; r += TPU) ac[r] = fma(z2, xa[r], ac[r]);
            if (own0 && rg == 0) ac[i - rb] -= z;
          }
        } else if (c < i && rg == 0) {
          const double gv = fma(dscal, dsum[c], rowi[c]);
          gq0[c] = gv;
          gqf0[c] = f64_to_f32_rz(gv);
          if (gram && g == 0) p.G[c + (size_t)i * bk] = gv;
        }
      }
      __syncthreads();
      stamp(step, 5);
      if (tau != 0.0)
        for (int r = lo + tid; r < nr; r += NT) xa[r] *= scal;
      if (own0 && tid == 0) xa[i - rb] = s_beta;
      if (tid == 0) s_ptau[0] = tau;
      npend = 1;
    } else {
      // Paired update.  For a column c > i + 1 the first reflector gives
      // z_c = tau (c_i + scal S_ac) and c'_{i+1} = c_{i+1} - z_c scal a_{i+1}; the second needs
      // (b')^T c' below row i + 1 = T_bc - z_c scal T_ab - zs T_ac + zs z_c scal T_aa, so
      // z'_c = tau2 (c'_{i+1} + scal2 (b')^T c') and below row i + 1
      //   c'' = c - (z_c scal - z'_c scal2 zs) a - z'_c scal2 b   (two FMAs per entry).
      const double tau2 = s_tau2, scal2 = s_scal2, zb = s_zb, Taa = s_Taa, Tab = s_Tab;
      const double zs = zb * scal;
      const double ai1 = rowi1[i], bi1 = rowi1[i + 1];
      const int lo2 = min(max(i + 2 - rb, 0), nr);
      for (int c0 = 0; c0 < bk; c0 += NT / TPU) {
        const int c = c0 + tid / TPU, rg = tid % TPU;
        if (c > i + 1 && c < bk) {
          const double z = tau * fma(scal, dsum[c], rowi[c]);
          const double zsc = z * scal;
          const double c1 = fma(-zsc, ai1, rowi1[c]);
          const double Tbc = fma(-bi1, rowi1[c], dsum[bk + 1 + c]);
          const double Tac = fma(-ai1, rowi1[c], dsum[c]);
          const double dot = fma(zs * zsc, Taa, fma(-zs, Tac, fma(-zsc, Tab, Tbc)));
          const double z2 = tau2 * fma(scal2, dot, c1);
          const double ca = fma(z2 * scal2, zs, -zsc);
          const double cb = -z2 * scal2;
          double* ac = slab + (size_t)c * Rp;
          for (int r = lo2 + rg; r < nr; r += TPU) ac[r] = fma(cb, xb[r], fma(ca, xa[r], ac[r]));
          if (rg == 0) {
            if (own0) ac[i - rb] -= z;
            if (own1) ac[i + 1 - rb] = c1 - z2;
          }
        } else if (c < i && rg == 0) {
          // y_c^T y_i and y_c^T y_{i+1} (y_c[i + 1] = row i + 1 of column c)
          const double g0 = fma(scal, dsum[c], rowi[c]);
          const double Tbq = fma(-rowi1[c], bi1, dsum[bk + 1 + c]);
          const double Taq = fma(-rowi1[c], ai1, dsum[c]);
          const double g1 = fma(scal2, fma(-zs, Taq, Tbq), rowi1[c]);
          gq0[c] = g0;
          gqf0[c] = f64_to_f32_rz(g0);
          gq1[c] = g1;
          gqf1[c] = f64_to_f32_rz(g1);
          if (gram && g == 0) {
            p.G[c + (size_t)i * bk] = g0;
            p.G[c + (size_t)(i + 1) * bk] = g1;
          }
        }
      }
      if (tid == 0) {  // y_i^T y_{i+1} = scal a_{i+1} + scal2 scal (T_ab - zs T_aa)
        const double gi = fma(scal2 * scal, fma(-zs, Taa, Tab), scal * ai1);
        gq1[i] = gi;
        gqf1[i] = f64_to_f32_rz(gi);
        if (gram && g == 0) p.G[i + (size_t)(i + 1) * bk] = gi;
        s_ptau[0] = tau;
        s_ptau[1] = tau2;
      }
      __syncthreads();
      stamp(step, 5);
      // columns i and i + 1 become v_i and v_{i+1}: rows below i + 1 hold scal a_r and
      // scal2 (b_r - zs a_r); row i + 1 holds scal a_{i+1} and beta2; row i holds beta and
      // b_i - z_b.
      for (int r = lo + tid; r < nr; r += NT) {
        const double ar = xa[r];
        xa[r] = ar * scal;
        xb[r] = (rb + r == i + 1) ? s_beta2 : fma(-zs, ar, xb[r]) * scal2;
      }
      if (own0 && tid == 0) {
        xa[i - rb] = s_beta;
        xb[i - rb] = rowi[i + 1] - zb;
      }
      npend = 2;
    }
    pend_i = i;
    i += paired ? 2 : 1;
    __syncthreads();
    stamp(step, 6);
  }
  if (!gram) pending_w(npend, pend_i, true);
  __syncthreads();
  if (gram) {
    // W is formed after the panel from G (w_from_gram)
  } else if (wf32) {
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
  __syncthreads();
  trace_end(p.trace);
}

}  // namespace

size_t panel_smem_bytes(int bk, int Rp, bool w_in_smem) {
  return ((size_t)bk * Rp * (w_in_smem ? 2 : 1) + 7 * (size_t)bk + 2) * sizeof(double);
}

// three rotating accumulator buffers of panel_acc_entries(bk) sums each
size_t panel_sync_bytes(int bk) { return 256 + 3 * panel_acc_entries(bk) * kAccStride * sizeof(double); }

int panel_geometry(int j, int bk, int max_ctas, int min_rows, int* G, int* R, int* Rp, bool* w_in_smem) {
  if (j <= 0 || bk <= 0) return -1;
  int g = (j + min_rows - 1) / min_rows;
  if (g > max_ctas) g = max_ctas;
  if (g < 1) g = 1;
  int r = (j + g - 1) / g;
  g = (j + r - 1) / r;  // every CTA owns at least one row
  int rp = r | 1;       // odd stride: conflict-free strided shared-memory access
  // the opt-in limit (227 KB) less a kilobyte for the kernel's static shared memory
  constexpr size_t kDynMax = 226 * 1024;
  if (panel_smem_bytes(bk, rp, false) > kDynMax) return -2;
  *G = g;
  *R = r;
  *Rp = rp;
  *w_in_smem = panel_smem_bytes(bk, rp, true) <= kDynMax;
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

namespace {

// One thread per row (kWgRows rows per block).  The strict upper triangle of G, tau and the
// block's rows of Y are staged in shared memory, and each row's entries of W stay there
// while the substitution runs (a global store followed by a load of the same address would
// wait for L2 on every term); four partial sums shorten the dependent FP64 chains.
constexpr int kWgRows = 32;
__global__ void w_from_gram_kernel(int j, int bk, const double* Y, const double* tau, const double* G, double* W,
                                   int64_t ldy, unsigned long long* trace) {
  extern __shared__ double wg_smem[];
  double* sTau = wg_smem;                     // bk
  double* sG = sTau + bk;                     // bk (bk - 1) / 2: column q at offset q (q - 1) / 2
  double* sW = sG + (size_t)bk * (bk - 1) / 2;  // bk x kWgRows: entry (q, t) at q kWgRows + t
  pdl_wait_and_release();
  trace_start(trace);
  const int t = threadIdx.x, r0 = blockIdx.x * kWgRows, r = r0 + t;
  for (int q = t; q < bk; q += blockDim.x) sTau[q] = tau[q];
  for (int q = 1; q < bk; ++q)
    for (int c = t; c < q; c += blockDim.x) sG[q * (q - 1) / 2 + c] = G[c + (size_t)q * bk];
  if (r < j)
    for (int q = 0; q < bk; ++q) sW[q * kWgRows + t] = Y[r + (int64_t)q * ldy];  // y_r, replaced by w_r
  __syncthreads();
  if (r < j) {
#pragma unroll 1
  for (int q = 0; q < bk; ++q) {
    const double* gq = sG + q * (q - 1) / 2;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int c = 0;
    for (; c + 3 < q; c += 4) {
      s0 = fma(sW[c * kWgRows + t], gq[c], s0);
      s1 = fma(sW[(c + 1) * kWgRows + t], gq[c + 1], s1);
      s2 = fma(sW[(c + 2) * kWgRows + t], gq[c + 2], s2);
      s3 = fma(sW[(c + 3) * kWgRows + t], gq[c + 3], s3);
    }
    for (; c < q; ++c) s0 = fma(sW[c * kWgRows + t], gq[c], s0);
    const double wq = -sTau[q] * (sW[q * kWgRows + t] + ((s0 + s1) + (s2 + s3)));
    sW[q * kWgRows + t] = wq;
    W[r + (int64_t)q * ldy] = wq;
  }
  }
  __syncthreads();
  trace_end(trace);
}

// Tn = -T of a factored panel from its Gram coefficients: T = U^{-1} with U = strict upper
// of Y^T Y (G) + diag(1 / tau).  Column c by back substitution T(c, c) = tau_c,
// T(r, c) = -tau_r sum_{p = r+1..c} G(r, p) T(p, c) for r = c - 1 .. 0 (a tau_r of 0 gives a
// zero row, the identity reflector), in right-looking order: once T(p, c) is known, every
// lane adds G(r, p) T(p, c) into the sums of its rows r < p, so the dependent chain per
// step is one multiply, one broadcast and one FMA.  On GB300 each FP64 warp instruction
// holds a sub-partition's FP64 unit for tens of cycles, so the kernel runs one column per
// CTA, whose threads stage the column's part of G in shared memory and whose first warp
// alone substitutes (one substituting warp per SM).
__global__ void t_from_gram_kernel(int bk, const double* tau, const double* G, double* Tn,
                                   unsigned long long* trace) {
  extern __shared__ double tg_smem[];  // G(0:c, 0:c+1), column p at p * bk; then tau
  pdl_wait_and_release();
  trace_start(trace);
  const int lane = threadIdx.x & 31, c = blockIdx.x;
  double* sTau = tg_smem + (size_t)bk * bk;
  // every thread of the CTA stages (many loads in flight); warp 0 alone substitutes
  for (int q = threadIdx.x; q < (c + 1) * bk; q += blockDim.x) {
    const int r = q % bk, p = q / bk;
    if (r < p) tg_smem[q] = G[q];
  }
  for (int r = threadIdx.x; r <= c; r += blockDim.x) sTau[r] = tau[r];
  __syncthreads();
  if (threadIdx.x >= 32) return;
  double acc[4] = {0.0, 0.0, 0.0, 0.0}, t[4] = {0.0, 0.0, 0.0, 0.0};  // rows lane + 32 u (bk <= 128)
  for (int p = c; p >= 0; --p) {
    const int q = p >> 5;
    const bool mine = (p & 31) == lane;
    double accp = 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (u == q) accp = acc[u];
    double tp = 0.0;
    if (mine) tp = p == c ? sTau[c] : -sTau[p] * accp;
    tp = __shfl_sync(0xffffffffu, tp, p & 31);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = lane + 32 * u;
      if (mine && u == q) t[u] = tp;
      if (r < p) acc[u] = fma(tg_smem[r + (size_t)p * bk], tp, acc[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int r = lane + 32 * u;
    if (r < bk) Tn[r + (size_t)c * bk] = r <= c ? -t[u] : 0.0;
  }
  trace_end(trace);
}

}  // namespace

cudaError_t launch_t_from_gram(int bk, const double* tau, const double* G, double* Tn, cudaStream_t s) {
  if (bk <= 0) return cudaSuccess;
  if (bk > 128) return cudaErrorInvalidValue;
  static int configured_device = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_device != dev) {
    cudaError_t e = cudaFuncSetAttribute(t_from_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)((128 * 128 + 128) * sizeof(double)));
    if (e != cudaSuccess) return e;
    configured_device = dev;
  }
  prof::TraceScope tr(prof::kTraceW, 0);
  unsigned long long* rec = prof::trace_take();
  prof::count_launch();
  return launch_pdl(t_from_gram_kernel, dim3(bk), dim3(256), ((size_t)bk * bk + bk) * sizeof(double), s, bk, tau, G,
                    Tn, rec);
}

cudaError_t launch_w_from_gram(int j, int bk, const double* Y, const double* tau, const double* G, double* W,
                               int64_t ldy, cudaStream_t s) {
  if (j <= 0 || bk <= 0) return cudaSuccess;
  if (bk > 128) return cudaErrorInvalidValue;
  static int configured_device = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_device != dev) {
    cudaError_t e = cudaFuncSetAttribute(w_from_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)((128 + 128 * 127 / 2 + 128 * kWgRows) * sizeof(double)));
    if (e != cudaSuccess) return e;
    configured_device = dev;
  }
  const size_t smem = ((size_t)bk + (size_t)bk * (bk - 1) / 2 + (size_t)bk * kWgRows) * sizeof(double);
  prof::TraceScope tr(prof::kTraceW, 0);
  unsigned long long* rec = prof::trace_take();
  prof::count_launch();
  return launch_pdl(w_from_gram_kernel, dim3((j + kWgRows - 1) / kWgRows), dim3(kWgRows), smem, s, j, bk, Y, tau, G,
                    W, ldy, rec);
}

}  // namespace bandred
