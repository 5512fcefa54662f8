// Host side of programmatic dependent launch: the kernel may begin (launch, shared- and
// tensor-memory set-up) while the previous kernel of the stream finishes, and waits in
// pdl_wait_and_release (common.cuh) before it reads that kernel's results.  Every kernel
// launched through launch_pdl must call pdl_wait_and_release before such reads.
#pragma once
#include <cuda_runtime.h>

namespace bandred {

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace bandred
