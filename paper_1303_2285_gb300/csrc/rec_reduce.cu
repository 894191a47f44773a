// Kernels 3 and 4 of the combination path: the reductions that finish the
// box sums, and the seed-and-walk writer of R (see cov_internal.h).
#include <cuda_runtime.h>

#include "cov_launch.h"
#include "rec_reduce.cuh"

namespace cov {

// Kernel 3: one warp per reduction task (reduce_task).
template <typename T, int QMAX>
__global__ void __launch_bounds__(128) k_reduce(const RecParams p) {
  pdl_launch_dependents();
  pdl_wait();  // the product and fringe-row kernels' partials
  const int w = (int)blockIdx.x * 4 + (int)(threadIdx.x >> 5);
  if (w < reduce_tasks(p)) reduce_task<T, QMAX>(p, w, threadIdx.x & 31);
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

template <typename T, int QMAX>
static cudaError_t launch_reduce_q(const RecParams &p, cudaStream_t s, bool pdl) {
  const int blocks = (reduce_tasks(p) + 3) / 4;  // 4 warps a block
  const cudaError_t e = ensure_smem_attr(k_reduce<T, QMAX>, 0);
  if (e != cudaSuccess) return e;
  return launch_k(k_reduce<T, QMAX>, dim3((unsigned)blocks), dim3(128), 0, s, pdl, p);
}

// QMAX >= Q: the register count of the box-row task's running sums
template <typename T>
static cudaError_t launch_reduce_t(const RecParams &p, cudaStream_t s, bool pdl) {
  if (p.Q <= 8) return launch_reduce_q<T, 8>(p, s, pdl);
  if (p.Q <= 16) return launch_reduce_q<T, 16>(p, s, pdl);
  return launch_reduce_q<T, 32>(p, s, pdl);
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

cudaError_t launch_reduce(const RecParams &p, bool fp64, cudaStream_t s, bool pdl) {
  return fp64 ? launch_reduce_t<double>(p, s, pdl) : launch_reduce_t<float>(p, s, pdl);
}

cudaError_t launch_walk(const RecParams &p, bool fp64, cudaStream_t s, bool pdl) {
  return fp64 ? launch_walk_t<double>(p, s, pdl) : launch_walk_t<float>(p, s, pdl);
}

}  // namespace cov
