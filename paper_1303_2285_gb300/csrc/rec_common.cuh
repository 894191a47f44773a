// Host and device helpers shared by the kernel files of the combination path.
#pragma once

#include <cuda_runtime.h>

#include <utility>

#include "cov_device.cuh"
#include "cov_internal.h"

namespace cov {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // bounded waits: 2 s

// Programmatic dependent launch: a kernel launched with the
// programmatic-serialization attribute may start while the previous kernel in
// the stream is still running; griddepcontrol.wait then blocks until that
// kernel has completed and its writes are visible.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

template <typename... KArgs, typename... Args>
static cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t s, bool pdl, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Raises a kernel's dynamic shared-memory limit once per device and size
// (host-side cache, so repeated calls issue no attribute call).
struct SmemAttrEntry {
  const void *fn;
  int dev;
  size_t smem;
};

template <typename K> static cudaError_t ensure_smem_attr(K kern, size_t smem) {
  static SmemAttrEntry table[256];
  static int used = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const void *fn = (const void *)kern;
  int slot = -1;
  for (int i = 0; i < used; ++i)
    if (table[i].fn == fn && table[i].dev == dev) {
      if (table[i].smem >= smem) return cudaSuccess;
      slot = i;
      break;
    }
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (slot < 0) {
    // Same shared-memory carveout for every kernel of the path, so that the
    // SMs are not reconfigured between consecutive kernels.
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  if (slot < 0 && used < 256) slot = used++;
  if (slot >= 0) table[slot] = {fn, dev, smem};
  return cudaSuccess;
}

}  // namespace cov
