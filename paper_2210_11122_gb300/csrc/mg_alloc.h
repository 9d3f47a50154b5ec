// mg_alloc.h -- every device and pinned-host allocation of the engine goes through these wrappers, which
// count the live allocations (mg_diag_live_allocs) and can be told to fail the n-th next allocation
// (mg_diag_fail_alloc): the host-side fault injector of the allocation-failure tests.  A failed
// allocation returns cudaErrorMemoryAllocation with *p = nullptr, as cudaMalloc does.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace mg {

cudaError_t alloc_raw(void** p, size_t bytes, bool host);
cudaError_t free_raw(void* p, bool host);

template <class T>
inline cudaError_t dev_alloc(T** p, size_t bytes) { return alloc_raw(reinterpret_cast<void**>(p), bytes, false); }
template <class T>
inline cudaError_t host_alloc(T** p, size_t bytes) { return alloc_raw(reinterpret_cast<void**>(p), bytes, true); }
inline cudaError_t dev_free(const void* p) { return free_raw(const_cast<void*>(p), false); }
inline cudaError_t host_free(const void* p) { return free_raw(const_cast<void*>(p), true); }

}  // namespace mg
