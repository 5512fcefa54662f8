// C entry points of the split-precision tensor-core engine on its own: a thin FP64 GEMM
// C = op(A) B (n <= 128) and a symmetric rank-2k update of a lower triangle.  The band
// reductions use the same kernels for Eqs. updateA2symm and updateA2syr2k.
#include <algorithm>
#include <cstdint>

#include "driver.h"
#include "ozaki.h"
#include "prof.h"
#include "split.h"

namespace {

using namespace bandred;

size_t al(size_t x) { return (x + 255) / 256 * 256; }

int gemm_splits(int M, int K, int sms) {
  const int tiles = (M + 127) / 128;
  const int nkb = (K + 31) / 32;
  int s = std::max(1, (2 * sms) / std::max(tiles, 1));
  s = std::min(s, std::max(1, nkb / 2));
  return std::min(s, 256);
}

int sms_now() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

bool valid_split_precision(int p) { return p == BANDRED_BF16X3 || p == BANDRED_BF16X6 || p == BANDRED_OZAKI; }

}  // namespace

extern "C" {

size_t bandred_gemm_split_workspace(int64_t m, int64_t n, int64_t k, int precision) {
  if (m < 0 || n < 1 || n > 128 || k < 0 || !valid_split_precision(precision)) return 0;
  if (precision == BANDRED_OZAKI) {
    const int sp = ozaki::choose_splits((int)m, (int)n, (int)k, sms_now());
    return ozaki::bytes((int)m, (int)n, (int)k, sp) + 256;
  }
  const int S = split::slices_of(precision);
  const int BN = split::stream_bn((int)n);
  const int splits = gemm_splits((int)m, (int)k, sms_now());
  return al(split::packed_bytes(BN, (int)std::max<int64_t>(k, 1), BN, 32, S)) +
         al((size_t)splits * std::max<int64_t>(m, 1) * n * 8) + 256;
}

int bandred_gemm_split(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, int transA, const double* B,
                       int64_t ldb, double* C, int64_t ldc, int precision, void* work, size_t work_bytes,
                       int* dev_status, cudaStream_t stream) {
  if (m < 0) return -1;
  if (n < 1 || n > 128) return -2;
  if (k < 0) return -3;
  if (m > 0 && k > 0 && !A) return -4;
  if (lda < std::max<int64_t>(1, transA ? k : m)) return -5;
  if (k > 0 && !B) return -7;
  if (ldb < std::max<int64_t>(1, k)) return -8;
  if (m > 0 && !C) return -9;
  if (ldc < std::max<int64_t>(1, m)) return -10;
  if (!valid_split_precision(precision)) return -11;
  if (!work || (reinterpret_cast<uintptr_t>(work) & 255u)) return -12;
  if (work_bytes < bandred_gemm_split_workspace(m, n, k, precision)) return -13;
  if (m == 0) return 0;
  if (precision == BANDRED_OZAKI) {
    if (dev_status && cudaMemsetAsync(dev_status, 0, sizeof(int), stream) != cudaSuccess) return BANDRED_ERR_CUDA;
    const int sp = ozaki::choose_splits((int)m, (int)n, (int)k, sms_now());
    const ozaki::Bufs b = ozaki::carve(work, (int)m, (int)n, (int)k, sp);
    const ozaki::Operand opA{A, lda, transA ? 1 : 0, (int)k, nullptr, 0, 0, 0, (int)m};
    const ozaki::Operand opB{B, ldb, 1, (int)k, nullptr, 0, 0, 0, (int)n};
    if (ozaki::product(opA, opB, (int)m, (int)n, (int)k, 1.0, 0.0, C, ldc, b, sp, dev_status, 2000ull * 1000000ull,
                       stream) != cudaSuccess)
      return BANDRED_ERR_CUDA;
    return 0;
  }
  const int S = split::slices_of(precision);
  const int BN = split::stream_bn((int)n);
  const int K = (int)std::max<int64_t>(k, 1);
  char* w = static_cast<char*>(work);
  __nv_bfloat16* blob = reinterpret_cast<__nv_bfloat16*>(w);
  const size_t blob_bytes = al(split::packed_bytes(BN, K, BN, 32, S));
  const int splits = gemm_splits((int)m, K, sms_now());
  double* P = reinterpret_cast<double*>(w + blob_bytes);
  int* status = dev_status;
  if (status && cudaMemsetAsync(status, 0, sizeof(int), stream) != cudaSuccess) return BANDRED_ERR_CUDA;

  split::PackParams pp{};
  pp.M1 = B;  // operand element (n_idx, k_idx) = B[k_idx + n_idx * ldb]
  pp.ld1 = ldb;
  pp.K1 = (int)k;
  pp.t1 = 1;
  pp.M2 = nullptr;
  pp.K2 = 0;
  pp.scale1 = pp.scale2 = 1.0;
  pp.R = (int)n;
  pp.TR = BN;
  pp.TK = 32;
  pp.nrb = 1;
  pp.nkb = (K + 31) / 32;
  pp.S = S;
  pp.out = blob;
  pp.status = status;
  if (split::pack(pp, stream) != cudaSuccess) return BANDRED_ERR_CUDA;

  split::StreamParams sp{};
  sp.A = A;
  sp.lda = lda;
  sp.mode = transA ? split::kModeTrans : split::kModePlain;
  sp.M = (int)m;
  sp.K = (int)k;
  sp.N = (int)n;
  sp.Bblob = blob;
  sp.nkb = pp.nkb;
  sp.stages_per_split = (pp.nkb + splits - 1) / splits;
  const int used = (pp.nkb + sp.stages_per_split - 1) / sp.stages_per_split;
  sp.P = P;
  sp.ldp = m;
  sp.split_stride = (int64_t)m * n;
  sp.status = status;
  sp.limit_ns = 2000ull * 1000000ull;
  if (split::stream_gemm(sp, S, std::max(used, 1), stream) != cudaSuccess) return BANDRED_ERR_CUDA;
  if (split::reduce((int)m, (int)n, std::max(used, 1), P, m, (int64_t)m * n, 1.0, 0.0, C, ldc, stream) !=
      cudaSuccess)
    return BANDRED_ERR_CUDA;
  return 0;
}

size_t bandred_syr2k_split_workspace(int64_t n, int64_t kb, int precision) {
  if (n < 0 || kb < 1 || !valid_split_precision(precision)) return 0;
  if (precision == BANDRED_OZAKI) return ozaki::bytes((int)n, (int)n, (int)(2 * kb), 1, false) + 256;
  const int S = split::slices_of(precision);
  const int Kr = (int)((2 * kb + 63) / 64 * 64);
  return 2 * al(split::packed_bytes((int)std::max<int64_t>(n, 1), Kr, 128, 64, S)) + 256;
}

int bandred_syr2k_split(int64_t n, int64_t kb, const double* X, int64_t ldx, const double* Y, int64_t ldy, double* C,
                        int64_t ldc, int precision, void* work, size_t work_bytes, int* dev_status,
                        cudaStream_t stream) {
  if (n < 0) return -1;
  if (kb < 1 || kb > 128) return -2;
  if (n > 0 && !X) return -3;
  if (ldx < std::max<int64_t>(1, n)) return -4;
  if (n > 0 && !Y) return -5;
  if (ldy < std::max<int64_t>(1, n)) return -6;
  if (n > 0 && !C) return -7;
  if (ldc < std::max<int64_t>(1, n)) return -8;
  if (!valid_split_precision(precision)) return -9;
  if (!work || (reinterpret_cast<uintptr_t>(work) & 255u)) return -10;
  if (work_bytes < bandred_syr2k_split_workspace(n, kb, precision)) return -11;
  if (n == 0) return 0;
  if (precision == BANDRED_OZAKI) {
    if (dev_status && cudaMemsetAsync(dev_status, 0, sizeof(int), stream) != cudaSuccess) return BANDRED_ERR_CUDA;
    const ozaki::Bufs b = ozaki::carve(work, (int)n, (int)n, (int)(2 * kb), 1);
    // [X 2^-sigma | Y 2^sigma] and [Y 2^sigma | X 2^-sigma]: the same product, with the two
    // halves of each row brought near one magnitude (the largest exponents of X and Y go
    // in the last 256 bytes of the workspace)
    int* sh = reinterpret_cast<int*>(static_cast<char*>(work) + ozaki::bytes((int)n, (int)n, (int)(2 * kb), 1, false));
    ozaki::Operand opA{X, ldx, 0, (int)kb, Y, ldy, 0, (int)kb, (int)n};  // [X | Y]
    ozaki::Operand opB{Y, ldy, 0, (int)kb, X, ldx, 0, (int)kb, (int)n};  // [Y | X]
    opA.sh = opB.sh = sh;
    opA.shsign = 1;
    opB.shsign = -1;
    if (ozaki::balance(opA, sh, stream) != cudaSuccess) return BANDRED_ERR_CUDA;
    if (ozaki::prepare(opA, opB, b, stream) != cudaSuccess) return BANDRED_ERR_CUDA;
    if (ozaki::rank_apply((int)n, (int)n, (int)(2 * kb), 1.0, C, ldc, 0, (int)n, 1, b, dev_status,
                          2000ull * 1000000ull, stream) != cudaSuccess)
      return BANDRED_ERR_CUDA;
    return 0;
  }
  const int S = split::slices_of(precision);
  const int Kr = (int)((2 * kb + 63) / 64 * 64);
  const size_t blob = al(split::packed_bytes((int)n, Kr, 128, 64, S));
  __nv_bfloat16* Ab = reinterpret_cast<__nv_bfloat16*>(work);
  __nv_bfloat16* Bb = reinterpret_cast<__nv_bfloat16*>(static_cast<char*>(work) + blob);
  if (dev_status && cudaMemsetAsync(dev_status, 0, sizeof(int), stream) != cudaSuccess) return BANDRED_ERR_CUDA;
  split::PackParams pp{};
  pp.M1 = X;
  pp.ld1 = ldx;
  pp.K1 = (int)kb;
  pp.t1 = 0;
  pp.M2 = Y;
  pp.ld2 = ldy;
  pp.K2 = (int)kb;
  pp.t2 = 0;
  pp.scale1 = pp.scale2 = 1.0;
  pp.R = (int)n;
  pp.TR = 128;
  pp.TK = 64;
  pp.nrb = (int)((n + 127) / 128);
  pp.nkb = Kr / 64;
  pp.S = S;
  pp.out = Ab;
  pp.status = dev_status;
  if (split::pack(pp, stream) != cudaSuccess) return BANDRED_ERR_CUDA;
  pp.M1 = Y;
  pp.ld1 = ldy;
  pp.M2 = X;
  pp.ld2 = ldx;
  pp.out = Bb;
  if (split::pack(pp, stream) != cudaSuccess) return BANDRED_ERR_CUDA;
  split::RankParams rp{};
  rp.Ablob = Ab;
  rp.Bblob = Bb;
  rp.Kr = Kr;
  rp.C = C;
  rp.ldc = ldc;
  rp.M = (int)n;
  rp.N = (int)n;
  rp.col0 = 0;
  rp.col1 = (int)n;
  rp.lower = 1;
  rp.tj0 = 0;
  rp.alpha = 1.0;
  rp.status = dev_status;
  rp.limit_ns = 2000ull * 1000000ull;
  const int T = (int)((n + 127) / 128);
  if (split::rank_update(rp, S, T, T, stream) != cudaSuccess) return BANDRED_ERR_CUDA;
  return 0;
}

}  // extern "C"
