// Host-side setup of a kernel's shared-memory attributes, shared by every
// kernel file.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <mutex>

namespace cov {

// Raises `fn`'s dynamic shared-memory limit on the current device to at least
// `smem` bytes before a launch with that much (needed above 48 KB), and with
// `max_carveout` asks for the largest shared-memory carveout on its first use
// there. A table of (kernel, device, limit set), guarded by a mutex, makes
// later calls issue no CUDA call; safe from several host threads and across
// devices.
inline cudaError_t ensure_dyn_smem(const void *fn, size_t smem, bool max_carveout) {
  struct Entry {
    const void *fn;
    int dev;
    size_t smem;
  };
  static Entry table[512];
  static int used = 0;
  static std::mutex mu;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  int slot = -1;
  for (int i = 0; i < used; ++i)
    if (table[i].fn == fn && table[i].dev == dev) {
      if (table[i].smem >= smem) return cudaSuccess;
      slot = i;
      break;
    }
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (slot < 0 && max_carveout) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  if (slot < 0 && used < 512) slot = used++;
  if (slot >= 0) table[slot] = {fn, dev, smem};
  return cudaSuccess;
}

}  // namespace cov
