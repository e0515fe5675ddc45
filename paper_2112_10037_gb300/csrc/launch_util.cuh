// Host helpers for kernel launches: per-kernel shared-memory opt-in and
// occupancy, cached after the first query.
#pragma once

#include <mutex>
#include <unordered_map>

#include "internal.cuh"

namespace sg {

struct KernelInfo {
  int blocks_per_sm = 0;
};

// Blocks of `kernel` that fit on one SM with `threads` threads and `smem`
// bytes of dynamic shared memory (opting in above 48 KB).  0 on error.
template <typename Kern>
int kernel_blocks_per_sm(Kern kernel, int threads, size_t smem) {
  static std::mutex mu;
  static std::unordered_map<unsigned long long, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long key = ((unsigned long long)(uintptr_t)(const void*)kernel) ^
                                 ((unsigned long long)smem << 40) ^ ((unsigned long long)dev << 58) ^
                                 (unsigned long long)threads;
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) n = 0;
  std::lock_guard<std::mutex> g(mu);
  cache[key] = n;
  return n;
}

// Grid for a grid-stride kernel: enough blocks for `units` (rows per block
// given), capped at the number that are resident at once.
inline int persistent_grid(long long units, int units_per_block, int nsm, int per_sm) {
  long long want = units >= 0 ? (units + units_per_block - 1) / units_per_block : (long long)nsm * per_sm;
  long long cap = (long long)nsm * (per_sm > 0 ? per_sm : 1);
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return (int)want;
}

}  // namespace sg
