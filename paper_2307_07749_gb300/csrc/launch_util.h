// launch_util.h - host helpers shared by the kernel launchers: the dynamic shared-memory limit of
// a kernel, set once per device.
#pragma once
#include <atomic>
#include <cuda_runtime.h>

namespace bltt {

template <typename K>
static inline cudaError_t set_smem(K kern, size_t bytes) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// cudaFuncSetAttribute acts on the current device only, so each caller records, per device (bit d
// of a mask), that its attributes are set.  Setting them twice is harmless, so two threads racing
// on a first call only repeat the work; devices beyond 63 set them on every call.
template <class F>
static inline cudaError_t once_per_device(std::atomic<unsigned long long>& mask, F&& f) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
  if (bit && (mask.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = f();
  if (e == cudaSuccess && bit) mask.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

}  // namespace bltt
