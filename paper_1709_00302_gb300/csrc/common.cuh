// Device helpers shared by the band-reduction kernels: bounded waits, reductions,
// cache-bypassing loads and the workspace/status conventions.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/bandred.h"

namespace bandred {

// Counters used by the grid-wide barrier of a cooperative launch.  Zeroed by the host
// (cudaMemsetAsync) before every launch that uses them.
struct GridSync {
  unsigned int count;   // arrivals, monotonically increasing within one launch
  unsigned int abort;   // set by the first CTA whose wait timed out
  unsigned int pad[30];
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier with a time limit.  Every CTA of the (co-resident, cooperative)
// grid calls it with the same `generation` (1, 2, 3, ...).  `extra` extra arrivals are
// awaited (0 in normal use; a positive value makes the wait unsatisfiable, which is how
// the tests exercise the timeout path).  Returns false when the wait timed out or
// another CTA aborted; the caller must then return without touching shared results.
// Ordering: the CTA's writes before the call happen before its release-add (bar.sync,
// then a gpu-scope release by thread 0); the acquire-load that sees the final count makes
// every other CTA's writes visible to this CTA after the closing bar.sync.
__device__ __forceinline__ bool grid_barrier(GridSync* gs, unsigned int generation, unsigned int extra,
                                             int* status, unsigned long long limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    red_release_add(&gs->count, 1u);
    const unsigned int target = generation * (gridDim.x + extra);
    unsigned long long t0 = 0;
    unsigned int spins = 0;
    while (true) {
      if (ld_acquire_gpu(&gs->count) >= target) break;
      if ((++spins & 15u) == 0u) {
        if (ld_acquire_gpu(&gs->abort) != 0u) { ok = 0; break; }
        const unsigned long long t = global_ns();
        if (t0 == 0) t0 = t;
        else if (t - t0 > limit_ns) {
          atomicExch(&gs->abort, 1u);
          if (status) atomicCAS(status, 0, BANDRED_DEV_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The two halves of grid_barrier, for CTAs that overlap independent work with the wait:
// grid_arrive (thread 0 only, after a __syncthreads that follows the writes to publish)
// and grid_wait (thread 0 only; the caller follows it with a __syncthreads).
__device__ __forceinline__ void grid_arrive(GridSync* gs) { red_release_add(&gs->count, 1u); }

__device__ __forceinline__ bool grid_wait(GridSync* gs, unsigned int generation, unsigned int extra, int* status,
                                          unsigned long long limit_ns) {
  const unsigned int target = generation * (gridDim.x + extra);
  unsigned long long t0 = 0;
  unsigned int spins = 0;
  while (true) {
    if (ld_acquire_gpu(&gs->count) >= target) return true;
    if ((++spins & 15u) == 0u) {
      if (ld_acquire_gpu(&gs->abort) != 0u) return false;
      const unsigned long long t = global_ns();
      if (t0 == 0) t0 = t;
      else if (t - t0 > limit_ns) {
        atomicExch(&gs->abort, 1u);
        if (status) atomicCAS(status, 0, BANDRED_DEV_TIMEOUT);
        return false;
      }
    }
  }
}

// Device trace stamps (see prof.h): the earliest start and the latest end over the CTAs
// of a launch, the end stored complemented so that both take an atomic minimum.
__device__ __forceinline__ void trace_start(unsigned long long* rec) {
  if (rec && threadIdx.x == 0) atomicMin(rec, global_ns());
}
__device__ __forceinline__ void trace_end(unsigned long long* rec) {
  if (rec && threadIdx.x == 0) atomicMin(rec + 1, ~global_ns());
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Loads of data written by other CTAs during the same launch: skip L1.
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

// Programmatic dependent launch.  A kernel launched with launch_pdl (launch.h) may start
// while the kernel before it in the stream is still running.  Every thread calls this
// once, after the prologue that touches only parameters, shared and tensor memory, and
// before its first access to global memory that an earlier kernel writes: the wait
// returns once the previous grid has completed and its writes are visible, and the
// release then lets the next kernel of the stream begin its own launch.  Without the
// launch attribute both instructions return at once.
__device__ __forceinline__ void pdl_wait_and_release() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

}  // namespace bandred
