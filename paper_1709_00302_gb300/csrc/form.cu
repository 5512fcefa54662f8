// Forming the orthogonal factors of the reductions from their packed reflectors: Q of
// sy2sb (A = Q B Q^T, Section 2.1), U and V of ge2gb (A = U B V^T, Section 3.1; Q and P of
// the lower band form when m < n).  The reflectors H_c = I - tau_c v_c v_c^T are taken in
// groups of b consecutive ones, each in the compact-WY form of Section 4.1,
// H_c0 .. H_c0+bg-1 = I + W Y^T with Y the unit lower trapezoidal block of the v_c and
// W = -Y T; the product Q = H_0 H_1 ... is accumulated from the last group to the first,
// Q(o:N, o:N) += W (Y^T Q(o:N, o:N)), so that each group only touches the trailing block
// its reflectors act on (the rows of that block left of column o are still zero).
//
// W comes from Y without forming T: T^{-1} = strictly-upper(Y^T Y) + diag(1/tau), so each
// row w_r of W = -Y T solves w_r T^{-1} = -y_r, a forward substitution over the group's
// columns that runs independently per row:
//   w_r[q] = -tau_q (y_r[q] + sum_{p<q} w_r[p] (Y^T Y)(p, q)).
// The two large products run on the FP64 path or as Ozaki-scheme products.
#include <algorithm>
#include <cstdint>

#include "driver.h"
#include "kernels.h"
#include "ozaki.h"
#include "prof.h"

namespace bandred {
namespace {

constexpr size_t kAlignF = 256;
size_t alignf(size_t x) { return (x + kAlignF - 1) / kAlignF * kAlignF; }

// Q = I (N x N, column-major, ldq)
__global__ void identity_kernel(int N, double* Q, int64_t ldq) {
  const int64_t total = (int64_t)N * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % N), c = (int)(idx / N);
    Q[r + (int64_t)c * ldq] = r == c ? 1.0 : 0.0;
  }
}

// Y (j x bg, ld) of the group whose first reflector is c0 and first row o = c0 + shift:
// Y(t, q) = 0 above the diagonal, 1 on it, and below it the stored entries of v_{c0+q},
// which sit at P[(o + t) es + (c0 + q) cs].
__global__ void build_y_kernel(int j, int bg, const double* P, int64_t es, int64_t cs, int c0, int o, double* Y,
                               int64_t ld) {
  const int64_t total = (int64_t)j * bg;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(idx % j), q = (int)(idx / j);
    Y[t + (int64_t)q * ld] = t < q ? 0.0 : (t == q ? 1.0 : P[(int64_t)(o + t) * es + (int64_t)(c0 + q) * cs]);
  }
}

// W = -Y T by the per-row forward substitution above (G = Y^T Y, bg x bg, ldg = bg).
// One thread per row; the strict upper triangle of G and tau are staged in shared memory,
// and the row's earlier entries of W are read back from W itself (L1-resident).
constexpr int kMaxGroup = 64;
__global__ void w_from_y_kernel(int j, int bg, const double* Y, int64_t ld, const double* tau, const double* G,
                                double* W) {
  __shared__ double sG[kMaxGroup * (kMaxGroup - 1) / 2];  // column q at offset q (q - 1) / 2
  __shared__ double sTau[kMaxGroup];
  for (int q = threadIdx.x; q < bg; q += blockDim.x) sTau[q] = tau[q];
  for (int q = 1; q < bg; ++q)
    for (int p = threadIdx.x; p < q; p += blockDim.x) sG[q * (q - 1) / 2 + p] = G[p + (int64_t)q * bg];
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= j) return;
  double* wr = W + r;
#pragma unroll 1
  for (int q = 0; q < bg; ++q) {
    const double* gq = sG + q * (q - 1) / 2;
    double s0 = 0.0, s1 = 0.0;
    int p = 0;
    for (; p + 1 < q; p += 2) {
      s0 = fma(wr[(int64_t)p * ld], gq[p], s0);
      s1 = fma(wr[(int64_t)(p + 1) * ld], gq[p + 1], s1);
    }
    if (p < q) s0 = fma(wr[(int64_t)p * ld], gq[p], s0);
    wr[(int64_t)q * ld] = -sTau[q] * (Y[r + (int64_t)q * ld] + (s0 + s1));
  }
}

}  // namespace

// Sizes of the forming routine's workspace for an order-N factor and groups of b.
struct FormWs {
  double *Y, *W, *G, *Gp, *M;
  char* oz;
  char* ozr;
  size_t oz_cap;
  size_t bytes;
};

static FormWs carve_form(void* work, int N, int b, bool ozaki_path) {
  char* base = static_cast<char*>(work);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += alignf(bytes);
    return p;
  };
  FormWs ws{};
  const size_t nb = (size_t)std::max(N, 1) * b;
  ws.Y = reinterpret_cast<double*>(take(nb * sizeof(double)));
  ws.W = reinterpret_cast<double*>(take(nb * sizeof(double)));
  ws.G = reinterpret_cast<double*>(take((size_t)b * b * sizeof(double)));
  ws.Gp = reinterpret_cast<double*>(take((size_t)64 * b * b * sizeof(double)));  // split-K partials of G
  ws.M = reinterpret_cast<double*>(take(nb * sizeof(double)));
  if (ozaki_path) {
    const int n1 = std::max(N, 1);
    ws.oz_cap = ozaki::bytes(n1, b, n1, ozaki::choose_splits(n1, b, n1, 160));
    ws.oz = take(ws.oz_cap);
    ws.ozr = take(ozaki::bytes(n1, n1, b, 1, false));
  }
  ws.bytes = off + kAlignF;  // + one aligned word of status
  return ws;
}

size_t form_workspace_bytes(int64_t N, const Options& o) {
  const int b = std::min(o.b > 0 ? o.b : 64, kMaxGroup);
  return carve_form(nullptr, (int)N, b, o.precision != BANDRED_FP64).bytes;
}

#define CKF(call)                                                 \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return record_cuda_error(e_, #call);   \
  } while (0)

int form_run(int64_t N64, int64_t nref64, int64_t shift, const double* P, int64_t es, int64_t cs, const double* tau,
             double* Q, int64_t ldq, const Options& o, void* work, int* dev_status, cudaStream_t s) {
  const int N = (int)N64, nref = (int)std::max<int64_t>(0, std::min<int64_t>(nref64, N64 - shift));
  const int b = std::min(o.b > 0 ? o.b : 64, kMaxGroup);
  const bool oz = o.precision != BANDRED_FP64;
  FormWs ws = carve_form(work, N, b, oz);
  int* status = dev_status ? dev_status : reinterpret_cast<int*>(static_cast<char*>(work) + ws.bytes - kAlignF);
  CKF(cudaMemsetAsync(status, 0, sizeof(int), s));
  if (N <= 0) return 0;
  {
    const int blocks = (int)std::min<int64_t>(((int64_t)N * N + 255) / 256, 8192);
    prof::count_launch();
    identity_kernel<<<blocks, 256, 0, s>>>(N, Q, ldq);
    CKF(cudaGetLastError());
  }
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ld = std::max(N, 1);
  const int ngroups = (nref + b - 1) / b;
  for (int g = ngroups - 1; g >= 0; --g) {
    const int c0 = g * b, bg = std::min(b, nref - c0);
    const int r0 = c0 + (int)shift, j = N - r0;
    if (j <= 1 || bg <= 0) continue;
    double* Qs = Q + r0 + (int64_t)r0 * ldq;
    {
      const int blocks = (int)std::min<int64_t>(((int64_t)j * bg + 255) / 256, 4096);
      prof::count_launch();
      build_y_kernel<<<blocks, 256, 0, s>>>(j, bg, P, es, cs, c0, r0, ws.Y, ld);
      CKF(cudaGetLastError());
    }
    // G = Y^T Y (bg x bg), FP64 with split-K over the j rows
    const int sp = std::max(1, std::min(64, j / 512));
    CKF(gemm_f64(bg, bg, j, 1.0, MatView{ws.Y, ld, 1}, MatView{ws.Y, 1, ld}, 0.0, ws.G, bg, sp, ws.Gp, s));
    {
      prof::count_launch();
      w_from_y_kernel<<<(j + 127) / 128, 128, 0, s>>>(j, bg, ws.Y, ld, tau + c0, ws.G, ws.W);
      CKF(cudaGetLastError());
    }
    if (!oz) {
      // M = Y^T Qs (bg x j), then Qs += W M
      CKF(gemm_f64(bg, j, j, 1.0, MatView{ws.Y, ld, 1}, MatView{Qs, 1, ldq}, 0.0, ws.M, bg, 1, nullptr, s));
      CKF(gemm_f64(j, j, bg, 1.0, MatView{ws.W, 1, ld}, MatView{ws.M, 1, bg}, 1.0, Qs, ldq, 1, nullptr, s));
    } else {
      using ozaki::Operand;
      // M^T = Qs^T Y (j x bg; the large operand streamed), then Qs += W (M^T)^T
      const Operand qt{Qs, ldq, 1, j, nullptr, 0, 0, 0, j}, yt{ws.Y, ld, 1, j, nullptr, 0, 0, 0, bg};
      const int spz = ozaki::fit_splits(j, bg, j, ozaki::choose_splits(j, bg, j, sms), ws.oz_cap);
      CKF(ozaki::product(qt, yt, j, bg, j, 1.0, 0.0, ws.M, ld, ozaki::carve(ws.oz, j, bg, j, spz), spz, status,
                         o.limit_ns, s));
      const Operand wl{ws.W, ld, 0, bg, nullptr, 0, 0, 0, j}, mt{ws.M, ld, 0, bg, nullptr, 0, 0, 0, j};
      const ozaki::Bufs rb = ozaki::carve(ws.ozr, j, j, bg, 1);
      CKF(ozaki::prepare(wl, mt, rb, s));
      CKF(ozaki::rank_apply(j, j, bg, 1.0, Qs, ldq, 0, j, 0, rb, status, o.limit_ns, s));
    }
  }
  return 0;
}

}  // namespace bandred
