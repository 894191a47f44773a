// Self-test of the library's failure detection (not part of the estimate):
// one warp waits, through the same bounded mbarrier wait the pipelined
// product kernel uses, on a barrier that nothing arrives on. The wait gives
// up after the caller's limit and the kernel records COV_ETIMEOUT in the
// workspace status word, then returns: no trap, no fault, the context stays
// usable.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cov.h"
#include "cov_device.cuh"
#include "cov_internal.h"

namespace cov {

__global__ void __launch_bounds__(32) k_selftest_timeout(unsigned *status,
                                                         unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  // phase 0 never completes: the expected arrival never comes
  const bool ok = mbar_wait(&bar, 0, limit_ns);
  __syncwarp();
  if (!ok && threadIdx.x == 0) atomicCAS(status, kDevOk, kDevTimeout);
}

}  // namespace cov

extern "C" cov_status cov_selftest_timeout(void *workspace, size_t ws_bytes, uint32_t limit_us,
                                           cov_stream_t stream) {
  if (limit_us < 1 || limit_us > 1000000) return COV_EINVAL;
  if (!workspace || ws_bytes < 4 || ((uintptr_t)workspace & 255) != 0) return COV_EWORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(workspace, 0, 4, s) != cudaSuccess) return COV_ECUDA;
  cov::k_selftest_timeout<<<1, 32, 0, s>>>((unsigned *)workspace,
                                           (unsigned long long)limit_us * 1000ull);
  return cudaGetLastError() == cudaSuccess ? COV_OK : COV_ECUDA;
}
