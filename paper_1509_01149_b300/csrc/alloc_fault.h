// Host-side fault injection for the allocation paths of mppi_create and mppi_server_create,
// so that their out-of-memory handling can be tested without exhausting a GPU: once armed
// with n (mppi_debug_fail_allocations), the allocation after n successful ones through
// dev_malloc / host_alloc fails with cudaErrorMemoryAllocation without calling CUDA, once.
#pragma once
#include <atomic>
#include <cuda_runtime.h>

namespace mppi {

extern std::atomic<int> g_alloc_fail_countdown;  // -1: off

inline bool alloc_should_fail() {
  int v = g_alloc_fail_countdown.load(std::memory_order_relaxed);
  while (v >= 0) {
    if (g_alloc_fail_countdown.compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) return v == 0;
  }
  return false;
}

template <class T>
cudaError_t dev_malloc(T **p, size_t bytes) {
  if (alloc_should_fail()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(reinterpret_cast<void **>(p), bytes);
}

template <class T>
cudaError_t host_alloc(T **p, size_t bytes, unsigned int flags) {
  if (alloc_should_fail()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaHostAlloc(reinterpret_cast<void **>(p), bytes, flags);
}

}  // namespace mppi
