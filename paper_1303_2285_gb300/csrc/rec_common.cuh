// Host and device helpers shared by the kernel files of the combination path.
#pragma once

#include <cuda_runtime.h>

#include <utility>

#include "cov_device.cuh"
#include "cov_internal.h"
#include "smem_attr.h"

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

// Raises a kernel's dynamic shared-memory limit once per device and size and
// gives every kernel of the path the same (largest) shared-memory carveout, so
// that the SMs are not reconfigured between consecutive kernels.
template <typename K> static cudaError_t ensure_smem_attr(K kern, size_t smem) {
  return ensure_dyn_smem((const void *)kern, smem, true);
}

}  // namespace cov
