// The extern "C" entry points declared in include/bandred.h: argument validation
// (LAPACK-style negative codes), workspace checks, device selection, and the allocating
// short forms.  The computation itself is in driver.cu and the kernels.
#include <algorithm>
#include <cstdint>
#include <cstring>

#include "driver.h"

using bandred::Options;

namespace {

bool aligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }

int ge2gb_check(int64_t m, int64_t n, int64_t w, const double* A, int64_t lda, const double* tauq,
                const double* taup, const bandred_opts* opts, Options* o) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (w < 1) return -3;
  if (n > 0 && !A) return -4;
  if (lda < (m > 1 ? m : 1)) return -5;
  // m >= n: n left and max(n - w, 0) right reflectors; m < n (lower band of the
  // transpose): max(m - w, 0) left and m right ones
  const int64_t nq = m >= n ? n : std::max<int64_t>(m - w, 0), np = m >= n ? std::max<int64_t>(n - w, 0) : m;
  if (nq > 0 && !tauq) return -6;
  if (np > 0 && !taup) return -7;
  if (std::max(m, n) > INT32_MAX / 2) return BANDRED_ERR_UNSUPPORTED;
  if (bandred::resolve_options(opts, w, o) != 0) return -8;
  return 0;
}

}  // namespace

int bandred::sy2sb_check(int64_t n, int64_t w, const double* A, int64_t lda, const double* tau,
                         const bandred_opts* opts, Options* o) {
  if (n < 0) return -1;
  if (w < 1) return -2;
  if (n > 0 && !A) return -3;
  if (lda < (n > 1 ? n : 1)) return -4;
  if (n - w > 0 && !tau) return -5;
  if (n > INT32_MAX / 2) return BANDRED_ERR_UNSUPPORTED;
  if (bandred::resolve_options(opts, w, o) != 0) return -6;
  return 0;
}

extern "C" {

void bandred_default_opts(bandred_opts* opts) {
  if (!opts) return;
  std::memset(opts, 0, sizeof(*opts));
  opts->b = 0;
  opts->lookahead = -1;
  opts->precision = BANDRED_FP64;
  opts->slices = 0;
}

const char* bandred_status_string(int code) {
  switch (code) {
    case 0: return "success";
    case BANDRED_DEV_TIMEOUT: return "device: a bounded wait timed out (results invalid)";
    case BANDRED_DEV_INVARIANT: return "device: internal consistency check failed";
    case BANDRED_DEV_RANGE: return "device: an entry is outside the range of the split-precision path";
    case BANDRED_ERR_CUDA: return "a CUDA runtime call failed";
    case BANDRED_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case BANDRED_ERR_UNSUPPORTED: return "size not supported by the kernels";
    case BANDRED_ERR_ALLOC: return "workspace allocation failed";
    case BANDRED_ERR_SCRATCH: return "problem too large for the fixed scratch of bandred_sy2sb_noalloc";
    default: break;
  }
  if (code < 0 && code > -100) return "invalid argument (-i = i-th argument)";
  return "unknown status";
}

const char* bandred_last_error(void) { return bandred::last_cuda_error(); }

size_t bandred_sy2sb_workspace(int64_t n, int64_t w, const bandred_opts* opts) {
  Options o;
  if (n < 0 || w < 1 || bandred::resolve_options(opts, w, &o) != 0) return 0;
  return bandred::sy2sb_workspace_bytes(n, w, o);
}

int bandred_sy2sb_ex(int64_t n, int64_t w, double* A, int64_t lda, double* tau, const bandred_opts* opts,
                     void* work, size_t work_bytes, int* dev_status, cudaStream_t stream) {
  Options o;
  int rc = bandred::sy2sb_check(n, w, A, lda, tau, opts, &o);
  if (rc) return rc;
  bandred::DeviceGuard dg;
  if (!dg.select(A)) return -3;
  if (!work || !aligned(work)) return -7;
  if (work_bytes < bandred::sy2sb_workspace_bytes(n, w, o)) return -8;
  return bandred::sy2sb_run(n, w, A, lda, tau, o, work, dev_status, stream);
}

int bandred_sy2sb(int64_t n, int64_t w, double* A, int64_t lda, double* tau, const bandred_opts* opts,
                  cudaStream_t stream) {
  Options o;
  int rc = bandred::sy2sb_check(n, w, A, lda, tau, opts, &o);
  if (rc) return rc;
  bandred::DeviceGuard dg;
  if (!dg.select(A)) return -3;
  const size_t bytes = bandred::sy2sb_workspace_bytes(n, w, o);
  void* work = nullptr;
  if (cudaError_t e = cudaMallocAsync(&work, bytes, stream); e != cudaSuccess) {
    bandred::record_cuda_error(e, "cudaMallocAsync");
    return BANDRED_ERR_ALLOC;
  }
  rc = bandred::sy2sb_run(n, w, A, lda, tau, o, work, nullptr, stream);
  int status = 0;
  // The run wrote its status into the workspace (dev_status == nullptr).
  if (rc == 0) {
    // The status word is the last piece of the workspace.
    const int* st = reinterpret_cast<const int*>(static_cast<char*>(work) + bytes - 256);
    if (cudaMemcpyAsync(&status, st, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
      rc = BANDRED_ERR_CUDA;
  }
  cudaFreeAsync(work, stream);
  if (cudaStreamSynchronize(stream) != cudaSuccess) return BANDRED_ERR_CUDA;
  return rc ? rc : status;
}

size_t bandred_ge2gb_workspace(int64_t m, int64_t n, int64_t w, const bandred_opts* opts) {
  Options o;
  if (m < 0 || n < 0 || w < 1 || bandred::resolve_options(opts, w, &o) != 0) return 0;
  return bandred::ge2gb_workspace_bytes(m, n, w, o);
}

int bandred_ge2gb_ex(int64_t m, int64_t n, int64_t w, double* A, int64_t lda, double* tauq, double* taup,
                     const bandred_opts* opts, void* work, size_t work_bytes, int* dev_status, cudaStream_t stream) {
  Options o;
  int rc = ge2gb_check(m, n, w, A, lda, tauq, taup, opts, &o);
  if (rc) return rc;
  bandred::DeviceGuard dg;
  if (!dg.select(A)) return -4;
  if (!work || !aligned(work)) return -9;
  if (work_bytes < bandred::ge2gb_workspace_bytes(m, n, w, o)) return -10;
  return bandred::ge2gb_run(m, n, w, A, lda, tauq, taup, o, work, dev_status, stream);
}

int bandred_ge2gb(int64_t m, int64_t n, int64_t w, double* A, int64_t lda, double* tauq, double* taup,
                  const bandred_opts* opts, cudaStream_t stream) {
  Options o;
  int rc = ge2gb_check(m, n, w, A, lda, tauq, taup, opts, &o);
  if (rc) return rc;
  bandred::DeviceGuard dg;
  if (!dg.select(A)) return -4;
  const size_t bytes = bandred::ge2gb_workspace_bytes(m, n, w, o);
  void* work = nullptr;
  if (cudaError_t e = cudaMallocAsync(&work, bytes, stream); e != cudaSuccess) {
    bandred::record_cuda_error(e, "cudaMallocAsync");
    return BANDRED_ERR_ALLOC;
  }
  rc = bandred::ge2gb_run(m, n, w, A, lda, tauq, taup, o, work, nullptr, stream);
  int status = 0;
  if (rc == 0) {
    const int* st = reinterpret_cast<const int*>(static_cast<char*>(work) + bytes - 256);
    if (cudaMemcpyAsync(&status, st, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
      rc = BANDRED_ERR_CUDA;
  }
  cudaFreeAsync(work, stream);
  if (cudaStreamSynchronize(stream) != cudaSuccess) return BANDRED_ERR_CUDA;
  return rc ? rc : status;
}

size_t bandred_form_workspace(int64_t N, const bandred_opts* opts) {
  Options o;
  if (N < 0 || bandred::resolve_options(opts, 1 << 20, &o) != 0) return 0;
  return bandred::form_workspace_bytes(N, o);
}

namespace {

// Shared checks and launch of the three forming entry points.
int form_call(int64_t N, int64_t nref, int64_t shift, const double* A, int64_t lda, int64_t need_lda, int64_t es,
              int64_t cs, const double* tau, double* Q, int64_t ldq, const bandred_opts* opts, void* work,
              size_t work_bytes, int* dev_status, cudaStream_t stream) {
  Options o;
  if (N > INT32_MAX / 2) return BANDRED_ERR_UNSUPPORTED;
  if (N > 0 && !A) return -3;
  if (lda < std::max<int64_t>(1, need_lda)) return -4;
  if (nref > 0 && !tau) return -5;
  if (N > 0 && !Q) return -6;
  if (ldq < std::max<int64_t>(1, N)) return -7;
  if (bandred::resolve_options(opts, 1 << 20, &o) != 0) return -8;
  if (!work || !aligned(work)) return -9;
  if (work_bytes < bandred::form_workspace_bytes(N, o)) return -10;
  bandred::DeviceGuard dg;
  if (N > 0 && !dg.select(Q)) return -6;
  return bandred::form_run(N, nref, shift, A, es, cs, tau, Q, ldq, o, work, dev_status, stream);
}

}  // namespace

int bandred_sy2sb_form_q(int64_t n, int64_t w, const double* A, int64_t lda, const double* tau, double* Q,
                         int64_t ldq, const bandred_opts* opts, void* work, size_t work_bytes, int* dev_status,
                         cudaStream_t stream) {
  if (n < 0) return -1;
  if (w < 1) return -2;
  return form_call(n, std::max<int64_t>(n - w, 0), w, A, lda, n, 1, lda, tau, Q, ldq, opts, work, work_bytes,
                   dev_status, stream);
}

int bandred_ge2gb_form(int64_t m, int64_t n, int64_t w, const double* A, int64_t lda, const double* tau, int side,
                       double* Q, int64_t ldq, const bandred_opts* opts, void* work, size_t work_bytes,
                       int* dev_status, cudaStream_t stream) {
  if (m < 0) return -1;
  if (n < 0 || w < 1) return -2;
  if (side != 0 && side != 1) return -5;
  const bool tall = m >= n;
  if (side == 0)  // U (m >= n: n reflectors on rows c..) or Q (m < n: m - w reflectors on rows c+w..)
    return form_call(m, tall ? n : std::max<int64_t>(m - w, 0), tall ? 0 : w, A, lda, m, 1, lda, tau, Q, ldq, opts,
                     work, work_bytes, dev_status, stream);
  // V (m >= n: n - w reflectors on columns c+w..) or P (m < n: m reflectors on columns c..)
  return form_call(n, tall ? std::max<int64_t>(n - w, 0) : m, tall ? w : 0, A, lda, m, lda, 1, tau, Q, ldq, opts,
                   work, work_bytes, dev_status, stream);
}

size_t bandred_ge2bb_workspace(int64_t m, int64_t n, int64_t w, const bandred_opts* opts) {
  Options o;
  if (m < 0 || n < 0 || w < 1 || bandred::resolve_options(opts, w, &o) != 0) return 0;
  return bandred::ge2bb_workspace_bytes(m, n, w, o);
}

int bandred_ge2bb_ex(int64_t m, int64_t n, int64_t w, double* A, int64_t lda, double* tauq, double* taup,
                     const bandred_opts* opts, void* work, size_t work_bytes, int* dev_status, cudaStream_t stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (w < 1) return -3;
  if (m > 0 && n > 0 && !A) return -4;
  if (lda < std::max<int64_t>(1, m)) return -5;
  const int64_t nlq = std::max<int64_t>(0, std::min(n, m - w)), nrq = std::max<int64_t>(0, std::min(m, n - w));
  if (nlq > 0 && !tauq) return -6;
  if (nrq > 0 && !taup) return -7;
  if (std::max(m, n) > INT32_MAX / 2) return BANDRED_ERR_UNSUPPORTED;
  Options o;
  if (bandred::resolve_options(opts, w, &o) != 0) return -8;
  if (!work || !aligned(work)) return -9;
  if (work_bytes < bandred::ge2bb_workspace_bytes(m, n, w, o)) return -10;
  bandred::DeviceGuard dg;
  if (m > 0 && n > 0 && !dg.select(A)) return -4;
  return bandred::ge2bb_run(m, n, w, A, lda, tauq, taup, o, work, dev_status, stream);
}

int bandred_ge2bb_form(int64_t m, int64_t n, int64_t w, const double* A, int64_t lda, const double* tau, int side,
                       double* Q, int64_t ldq, const bandred_opts* opts, void* work, size_t work_bytes,
                       int* dev_status, cudaStream_t stream) {
  if (m < 0) return -1;
  if (n < 0 || w < 1) return -2;
  if (side != 0 && side != 1) return -5;
  if (side == 0)  // U: reflector c acts on rows c+w .., v in column c below the band
    return form_call(m, std::max<int64_t>(0, std::min(n, m - w)), w, A, lda, m, 1, lda, tau, Q, ldq, opts, work,
                     work_bytes, dev_status, stream);
  // V: reflector c acts on columns c+w .., v in row c right of the band
  return form_call(n, std::max<int64_t>(0, std::min(m, n - w)), w, A, lda, m, lda, 1, tau, Q, ldq, opts, work,
                   work_bytes, dev_status, stream);
}

size_t bandred_sb2st_workspace(int64_t n, int64_t w) {
  if (n < 0 || w < 1 || w > 128) return 0;
  return bandred::sb2st_workspace_bytes(n, w);
}

int bandred_sb2st(int64_t n, int64_t w, const double* A, int64_t lda, double* d, double* e,
                  const bandred_opts* opts, void* work, size_t work_bytes, int* dev_status, cudaStream_t stream) {
  if (n < 0) return -1;
  if (w < 1) return -2;
  if (w > 128) return BANDRED_ERR_UNSUPPORTED;
  if (n > 0 && !A) return -3;
  if (lda < std::max<int64_t>(1, n)) return -4;
  if (n > 0 && !d) return -5;
  if (n > 1 && !e) return -6;
  if (n > INT32_MAX / 256) return BANDRED_ERR_UNSUPPORTED;
  Options o;
  if (bandred::resolve_options(opts, w, &o) != 0) return -7;
  if (!work || !aligned(work)) return -8;
  if (work_bytes < bandred::sb2st_workspace_bytes(n, w)) return -9;
  bandred::DeviceGuard dg;
  if (n > 0 && !dg.select(A)) return -3;
  return bandred::sb2st_run(n, w, A, lda, d, e, o.limit_ns, work, dev_status, stream);
}

size_t bandred_gb2bd_workspace(int64_t n, int64_t w) {
  return (n < 0 || w < 1 || w > 128) ? 0 : bandred::gb2bd_workspace_bytes(n, w);
}

int bandred_gb2bd(int64_t n, int64_t w, const double* A, int64_t lda, double* d, double* e,
                  const bandred_opts* opts, void* work, size_t work_bytes, int* dev_status, cudaStream_t stream) {
  if (n < 0) return -1;
  if (w < 1) return -2;
  if (w > 128) return BANDRED_ERR_UNSUPPORTED;
  if (n > 0 && !A) return -3;
  if (lda < std::max<int64_t>(1, n)) return -4;
  if (n > 0 && !d) return -5;
  if (n > 1 && !e) return -6;
  if (n > INT32_MAX / 512) return BANDRED_ERR_UNSUPPORTED;
  Options o;
  if (bandred::resolve_options(opts, w, &o) != 0) return -7;
  if (!work || !aligned(work)) return -8;
  if (work_bytes < bandred::gb2bd_workspace_bytes(n, w)) return -9;
  bandred::DeviceGuard dg;
  if (n > 0 && !dg.select(A)) return -3;
  return bandred::gb2bd_run(n, w, A, lda, d, e, o.limit_ns, work, dev_status, stream);
}

size_t bandred_bdsv_workspace(int64_t n) { return n < 0 ? 0 : bandred::bdsv_workspace_bytes(n); }

int bandred_bdsv(int64_t n, const double* d, const double* e, double* sigma, void* work, size_t work_bytes,
                 cudaStream_t stream) {
  if (n < 0) return -1;
  if (n > 0 && !d) return -2;
  if (n > 1 && !e) return -3;
  if (n > 0 && !sigma) return -4;
  if (n > INT32_MAX / 4) return BANDRED_ERR_UNSUPPORTED;
  if (!work || !aligned(work)) return -5;
  if (work_bytes < bandred::bdsv_workspace_bytes(n)) return -6;
  bandred::DeviceGuard dg;
  if (n > 0 && !dg.select(sigma)) return -4;
  return bandred::bdsv_run(n, d, e, sigma, work, stream);
}

size_t bandred_sterf_workspace(int64_t n) { return n < 0 ? 0 : bandred::sterf_workspace_bytes(n); }

int bandred_sterf(int64_t n, const double* d, const double* e, double* lam, void* work, size_t work_bytes,
                  cudaStream_t stream) {
  if (n < 0) return -1;
  if (n > 0 && !d) return -2;
  if (n > 1 && !e) return -3;
  if (n > 0 && !lam) return -4;
  if (n > INT32_MAX / 2) return BANDRED_ERR_UNSUPPORTED;
  if (!work || !aligned(work)) return -5;
  if (work_bytes < bandred::sterf_workspace_bytes(n)) return -6;
  bandred::DeviceGuard dg;
  if (n > 0 && !dg.select(lam)) return -4;
  return bandred::sterf_run(n, d, e, lam, work, stream);
}

}  // extern "C"
