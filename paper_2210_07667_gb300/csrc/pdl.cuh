// Programmatic dependent launch.  A kernel started with launch_pdl may be
// scheduled before the kernel ahead of it on the stream has finished: it calls
// pdl_wait() before its first access to global memory, which returns once
// every preceding kernel has completed and its writes are visible.  This
// hides part of the launch latency between the short kernels of one call.
// pdl_trigger() would let the next kernel launch before this one ends; the
// kernels here do not call it: waiting CTAs of the next kernel then share
// the SMs with the running one, and a call's Tucker operators ran 16% slower
// that way (7% faster without it than with plain launches).
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace phiks {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace phiks
