// swe_alloc.h -- every device allocation of the library goes through
// dev_malloc / dev_malloc_async.  A test hook (swe_debug_fail_alloc in
// include/swe.h) makes the n-th next allocation fail as if the device were
// out of memory, so that each error path runs without exhausting a GPU.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace swe {

// True if the allocation about to be made is the one chosen to fail
// (defined in swe_api.cu; thread-safe).
bool alloc_should_fail();

inline cudaError_t dev_malloc(void **p, size_t bytes) {
  if (alloc_should_fail()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

inline cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st) {
  if (alloc_should_fail()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocAsync(p, bytes, st);
}

}  // namespace swe
