// bandred_sy2sb_noalloc: the symmetric band reduction for callers that cannot allocate
// device memory.
//
// Some callers may not call cudaMalloc (or any allocator) at the point where they need
// the reduction: code running inside a stream that is being captured, where an
// allocation would break or serialise the capture; real-time or embedded hosts whose
// memory budget is fixed up front; plug-ins living in a process whose allocator belongs
// to someone else.  This entry point gives them the same computation as
// bandred_sy2sb_ex with its workspace taken from a fixed scratch array that the library
// declares at file scope on the device.  The array (BANDRED_NOALLOC_SCRATCH_BYTES bytes)
// is reserved on every GPU that loads the library and stays reserved until the process
// exits; no call allocates or frees anything.
//
// Host code cannot use the array's name as a device address (it names a host-side
// stand-in), so the first call on each device looks the real address up with
// cudaGetSymbolAddress while that device is current and keeps it for later calls.
#include <cstdint>
#include <mutex>

#include "driver.h"

namespace {

constexpr size_t kScratchBytes = BANDRED_NOALLOC_SCRATCH_BYTES;

// The shared scratch: every call on a device uses the same bytes.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[64] = {};

// Device address of the scratch on the current device (looked up once per device).
void* scratch_address(int* rc) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    *rc = bandred::record_cuda_error(e == cudaSuccess ? cudaErrorInvalidDevice : e, "cudaGetDevice");
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      *rc = bandred::record_cuda_error(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                                       "cudaGetSymbolAddress(g_noalloc_scratch)");
      return nullptr;
    }
    g_scratch_addr[dev] = p;
  }
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" int bandred_sy2sb_noalloc(int64_t n, int64_t w, double* A, int64_t lda, double* tau,
                                     const bandred_opts* opts, int* dev_status, cudaStream_t stream) {
  bandred::Options o;
  const int chk = bandred::sy2sb_check(n, w, A, lda, tau, opts, &o);
  if (chk) return chk;
  bandred::DeviceGuard dg;  // the device of A while the call runs; the caller's device afterwards
  if (n > 0 && !dg.select(A)) return -3;
  if (bandred::sy2sb_workspace_bytes(n, w, o) > kScratchBytes) return BANDRED_ERR_SCRATCH;
  int rc = 0;
  void* scratch = scratch_address(&rc);
  if (!scratch) return rc;
  return bandred::sy2sb_run(n, w, A, lda, tau, o, scratch, dev_status, stream);
}
