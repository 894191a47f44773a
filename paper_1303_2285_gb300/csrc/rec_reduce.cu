// Kernels 3 and 4 of the combination path: the reductions that finish the
// box sums, and the seed-and-walk writer of R (see cov_internal.h).
#include <cuda_runtime.h>

#include "cov_launch.h"
#include "rec_reduce.cuh"

namespace cov {

// Kernel 3, CTA form: one CTA per combination of the shard (reduce_combo_cta).
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_reduce_cta(const RecParams p) {
  extern __shared__ __align__(16) unsigned char smem_k3[];
  pdl_launch_dependents();
  pdl_wait();  // the product and fringe-row kernels' partials
  reduce_combo_cta<T>(p, p.u_lo + (int)blockIdx.x, (T *)smem_k3);
}

// Kernel 4: one CTA per block (bj, bj + dc) of R.
template <typename T>
__global__ void __launch_bounds__(256) k_walk_write(const RecParams p) {
  extern __shared__ __align__(16) unsigned char smem_k4[];
  int dc, bj;
  walk_block_of(p, blockIdx.x, dc, bj);
  pdl_wait();  // RV and CV of the reduction kernel
  walk_block<T>(p, dc, bj, smem_k4);
}

template <typename T>
static cudaError_t launch_walk_t(const RecParams &p, cudaStream_t s, bool pdl) {
  int nblk = 0;  // blocks (bj, bj + dc) of the shard's column lags
  for (int dc = p.dc_lo; dc < p.dc_hi; ++dc) nblk += p.Q - dc;
  const size_t smem = walk_smem_bytes<T>(p.P, p.NFR);
  auto kern = k_walk_write<T>;
  cudaError_t e = ensure_smem_attr(kern, smem);
  if (e != cudaSuccess) return e;
  return launch_k(kern, dim3(nblk), dim3(256), smem, s, pdl, p);
}

template <typename T>
static cudaError_t launch_reduce_cta_t(const RecParams &p, cudaStream_t s, bool pdl) {
  const int blocks = p.u_hi - p.u_lo;
  if (blocks <= 0) return cudaSuccess;
  const size_t smem = reduce_cta_smem_bytes<T>(p);
  auto kern = k_reduce_cta<T>;
  const cudaError_t e = ensure_smem_attr(kern, smem);
  if (e != cudaSuccess) return e;
  return launch_k(kern, dim3((unsigned)blocks), dim3(kRedThreads), smem, s, pdl, p);
}

cudaError_t launch_reduce(const RecParams &p, bool fp64, cudaStream_t s, bool pdl) {
  // one CTA per combination (reduce_combo_cta); the warp-task form
  // (reduce_task) serves the fused kernel
  return fp64 ? launch_reduce_cta_t<double>(p, s, pdl) : launch_reduce_cta_t<float>(p, s, pdl);
}

cudaError_t launch_walk(const RecParams &p, bool fp64, cudaStream_t s, bool pdl) {
  return fp64 ? launch_walk_t<double>(p, s, pdl) : launch_walk_t<float>(p, s, pdl);
}

}  // namespace cov
