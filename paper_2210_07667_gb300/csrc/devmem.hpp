// Device memory of the library.  Every device allocation and release goes
// through these four calls so that the number of live allocations can be
// read back and a test can make the k-th allocation fail (include/phiks.h:
// phiks_debug_fail_alloc, phiks_debug_live_allocations), which exercises the
// out-of-memory paths without exhausting a GPU.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace phiks {

cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t st);
// Both accept nullptr (no-op).  dev_free may synchronise (cudaFree);
// dev_free_async releases in stream order on `st`.
void dev_free(void* p);
void dev_free_async(void* p, cudaStream_t st);

}  // namespace phiks
