// Internal interface between the C ABI (api.cu) and the host-side loops (driver.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/bandred.h"

namespace bandred {

struct Options {
  int b;
  int lookahead;
  int precision;
  int slices;
  int panel_ctas;
  unsigned long long limit_ns;
  int debug;
  int panel_group;  // reflectors per grid-wide reduction of the panel: 2 (default) or 4
  int depth;        // look-ahead depth: 1, or 2 (V1 with 3b <= w)
};

// Records a failed CUDA call (readable through bandred_last_error) and returns
// BANDRED_ERR_CUDA.
int record_cuda_error(cudaError_t e, const char* what);
const char* last_cuda_error();

// Validates and completes the caller's options for bandwidth w; returns 0 or -1.
int resolve_options(const bandred_opts* in, int64_t w, Options* o);

// Argument checks of bandred_sy2sb_ex / bandred_sy2sb_noalloc (everything but the
// workspace): 0, a negative argument index or BANDRED_ERR_UNSUPPORTED; fills *o.
int sy2sb_check(int64_t n, int64_t w, const double* A, int64_t lda, const double* tau, const bandred_opts* opts,
                Options* o);

// Makes the device that owns a pointer current while the guard lives, and gives the
// caller's current device back when it goes out of scope: the library may share the
// process with other CUDA users (PyTorch, for one) that keep their own current device.
class DeviceGuard {
 public:
  DeviceGuard() = default;
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
  // false when ptr is not device (or managed) memory; nullptr selects nothing
  bool select(const void* ptr) {
    if (!ptr) return true;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return false;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return false;
    if (cur == at.device) return true;
    if (cudaSetDevice(at.device) != cudaSuccess) return false;
    prev_ = cur;
    return true;
  }
  ~DeviceGuard() {
    if (prev_ >= 0) cudaSetDevice(prev_);
  }

 private:
  int prev_ = -1;
};

size_t sy2sb_workspace_bytes(int64_t n, int64_t w, const Options& o);
int sy2sb_run(int64_t n, int64_t w, double* A, int64_t lda, double* tau, const Options& o, void* work,
              int* dev_status, cudaStream_t s);

size_t ge2gb_workspace_bytes(int64_t m, int64_t n, int64_t w, const Options& o);
size_t ge2bb_workspace_bytes(int64_t m, int64_t n, int64_t w, const Options& o);
// Second stage: band -> tridiagonal (bulge chasing) and the tridiagonal's eigenvalues.
size_t sb2st_workspace_bytes(int64_t n, int64_t w);
int sb2st_run(int64_t n, int64_t w, const double* A, int64_t lda, double* d, double* e, unsigned long long limit_ns,
              void* work, int* dev_status, cudaStream_t s);
size_t sterf_workspace_bytes(int64_t n);
int sterf_run(int64_t n, const double* d, const double* e, double* lam, void* work, cudaStream_t s);
// eigenvalues k0 .. k0 + count - 1 (ascending) of (d, e) into lam[0 .. count)
int sterf_range_run(int64_t n, const double* d, const double* e, double* lam, int64_t k0, int64_t count, void* work,
                    cudaStream_t s);
size_t gb2bd_workspace_bytes(int64_t n, int64_t w);
int gb2bd_run(int64_t n, int64_t w, const double* A, int64_t lda, double* d, double* e, unsigned long long limit_ns,
              void* work, int* dev_status, cudaStream_t s);
size_t bdsv_workspace_bytes(int64_t n);
int bdsv_run(int64_t n, const double* d, const double* e, double* sig, void* work, cudaStream_t s);
int ge2bb_run(int64_t m, int64_t n, int64_t w, double* A, int64_t lda, double* tauq, double* taup, const Options& o,
              void* work, int* dev_status, cudaStream_t s);
int ge2gb_run(int64_t m, int64_t n, int64_t w, double* A, int64_t lda, double* tauq, double* taup,
              const Options& o, void* work, int* dev_status, cudaStream_t s);

// Orthogonal factor of N x N from packed reflectors (form.cu): Q = H_0 .. H_{nref-1},
// H_c acting on indices c + shift .. N-1, v_c's stored entries at P[(c + shift + 1 + t) es
// + c cs].  FP64 products for BANDRED_FP64, Ozaki-scheme products otherwise.
size_t form_workspace_bytes(int64_t N, const Options& o);
int form_run(int64_t N, int64_t nref, int64_t shift, const double* P, int64_t es, int64_t cs, const double* tau,
             double* Q, int64_t ldq, const Options& o, void* work, int* dev_status, cudaStream_t s);

// Batched reductions (batched.cu).  mode 1 = plan (upload the schedule's tables), 2 = run.
int sy2sb_batched(int count, const int64_t* n, const int64_t* w, double* const* A, const int64_t* lda,
                  double* const* tau, const Options& o, void* work, size_t work_bytes, int* dev_status,
                  cudaStream_t s, int mode);
size_t sy2sb_batched_workspace(int count, const int64_t* n, const int64_t* w, const Options& o);
int ge2gb_batched(int count, const int64_t* m, const int64_t* n, const int64_t* w, double* const* A,
                  const int64_t* lda, double* const* tauq, double* const* taup, const Options& o, void* work,
                  size_t work_bytes, int* dev_status, cudaStream_t s, int mode);
size_t ge2gb_batched_workspace(int count, const int64_t* m, const int64_t* n, const int64_t* w, const Options& o);

}  // namespace bandred
