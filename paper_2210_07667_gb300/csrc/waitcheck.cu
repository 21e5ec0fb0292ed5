// A check of the failure path that every tensor-core kernel of the library
// takes when one of its bounded mbarrier waits gives up: one CTA allocates
// TMEM, waits on an mbarrier that nothing arrives at (so the wait must run
// out after limit_ns), records the failure in the plan's status word as those
// kernels do, frees its TMEM and returns.  The host then reads the status
// (phiks_device_status: PHIKS_ERR_TIMEOUT) and the context stays usable.
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "tcgen05.cuh"

namespace phiks {
namespace {

using namespace ptx;

constexpr int kWaitCheckSite = 21;  // the code the status word receives

__global__ void __launch_bounds__(64) wait_check_kernel(int* status, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(32)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_slot;
  // phase 0 of a barrier with one expected arrival and none made: the wait
  // can only end by its limit
  if (threadIdx.x == 0) (void)mbar_wait_for(&bar, 0, status, kWaitCheckSite, limit_ns);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(32)
                 : "memory");
  }
}

}  // namespace

cudaError_t launch_wait_check(int* status, uint64_t limit_ns, cudaStream_t st) {
  count_launch();
  wait_check_kernel<<<1, 64, 0, st>>>(status, limit_ns);
  return cudaGetLastError();
}

}  // namespace phiks
