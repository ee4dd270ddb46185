// launch_config.h -- per-device launch set-up of the persistent kernels.
//
// A persistent kernel is launched with as many CTAs as the current device
// keeps resident; kernels with more than 48 KB of dynamic shared memory also
// need that size set as a function attribute, once per device. Both are kept
// per (kernel, device) under a lock, so the first launch on each device sets
// up its own state and concurrent first launches from several threads do not
// race.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

namespace synth {

// CTAs of `kernel` (threads per CTA, dynamic shared memory smem bytes) that
// the current device keeps resident at once, at least one per SM; sets the
// shared-memory attribute on first use on the device.
inline cudaError_t resident_grid(const void* kernel, int threads, int smem, int* grid) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(kernel, dev);
  const auto it = cache.find(key);
  if (it != cache.end()) {
    *grid = it->second;
    return cudaSuccess;
  }
  if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
      cudaSuccess)
    return e;
  int sms = 0, per_sm = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem)) !=
      cudaSuccess)
    return e;
  const int g = sms * (per_sm > 0 ? per_sm : 1);
  cache.emplace(key, g);
  *grid = g;
  return cudaSuccess;
}

}  // namespace synth
