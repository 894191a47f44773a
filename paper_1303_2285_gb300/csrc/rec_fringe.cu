// Kernel 2 of the combination path: the products of the fringe rows with the
// inner columns (see cov_internal.h for the split of the work).
//
// A CTA takes one side (top or bottom fringe rows), one chunk of CWF inner
// columns and a block of FPB (fringe row n, row lag dr) pairs (one thread
// each; FP32 256, FP64 32 with narrower chunks, so that the slow FP64 pipe
// of every SM gets work). The strip of A
// those pairs touch (the 2P-2 rows next to the side, CWF+QMAX-1 columns) is
// staged in shared memory with cp.async (zero outside A). A thread owns one
// pair: it walks the chunk's columns in blocks of RC, keeps RC values
// a = A[n][m] in registers, streams b = A[n+dr][m+k], and accumulates the
// product of every column lag dc in its own register, so the chunk's sums for
// the pair's Q combinations need no cross-thread reduction. Every product is
// formed once.
#include <cuda_runtime.h>

#include "cov_launch.h"
#include "rec_fringe.cuh"

namespace cov {

template <typename T, int QMAX, int RC>
__global__ void __launch_bounds__(256) k_fringe_rows(const RecParams p) {
  using C2 = typename C2t<T>::type;
  extern __shared__ __align__(16) unsigned char smem_k2[];
  C2 *S = (C2 *)smem_k2;
  pdl_launch_dependents();
  const int npairs = (p.P - 1) * (2 * p.P - 1);
  const int nblk = (npairs + (int)blockDim.x - 1) / (int)blockDim.x;
  int bid = blockIdx.x;
  const int pb = bid % nblk;
  bid /= nblk;
  const int cc = bid % p.NCH, side = bid / p.NCH;
  fringe_stage<T>(p, S, side, cc);
  __syncthreads();
  const int t = pb * (int)blockDim.x + threadIdx.x;
  if (t < npairs) fringe_pair<T, QMAX, RC>(p, S, side, cc, t);
  // The next kernels read this kernel's and the product kernel's output: do
  // not complete before the product kernel has.
  pdl_wait();
}

template <typename T, int QMAX>
static cudaError_t launch_fringe_q(const RecParams &p, cudaStream_t s, bool pdl) {
  auto kern = k_fringe_rows<T, QMAX, 8>;
  const int npairs = (p.P - 1) * (2 * p.P - 1);
  const long long grid = 2LL * p.NCH * ((npairs + p.FPB - 1) / p.FPB);
  const size_t smem = (size_t)(2 * p.P - 2) * p.FPITCH * sizeof(typename C2t<T>::type);
  cudaError_t e = ensure_smem_attr(kern, smem);
  if (e != cudaSuccess) return e;
  return launch_k(kern, dim3((unsigned)grid), dim3((unsigned)p.FPB), smem, s, pdl, p);
}

cudaError_t launch_fringe(const RecParams &p, bool fp64, cudaStream_t s, bool pdl) {
  if (p.NFR <= 0 || p.NCH <= 0) return cudaSuccess;
  switch (p.QMAXF) {
    case 4: return fp64 ? launch_fringe_q<double, 4>(p, s, pdl) : launch_fringe_q<float, 4>(p, s, pdl);
    case 8: return fp64 ? launch_fringe_q<double, 8>(p, s, pdl) : launch_fringe_q<float, 8>(p, s, pdl);
    case 16: return fp64 ? launch_fringe_q<double, 16>(p, s, pdl) : launch_fringe_q<float, 16>(p, s, pdl);
    case 32: return fp64 ? launch_fringe_q<double, 32>(p, s, pdl) : launch_fringe_q<float, 32>(p, s, pdl);
  }
  return cudaErrorInvalidValue;
}

}  // namespace cov
