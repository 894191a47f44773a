// Kernel 2 of the combination path: the products of the fringe rows with the
// inner columns (see cov_internal.h for the split of the work).
//
// A CTA takes one side (top or bottom fringe rows), one chunk of CWF inner
// columns and a block of 256 (fringe row n, row lag dr) pairs. The strip of A
// those pairs touch (the 2P-2 rows next to the side, CWF+QMAX-1 columns) is
// staged in shared memory with cp.async (zero outside A). A thread owns one
// pair: it walks the chunk's columns in blocks of RC, keeps RC values
// a = A[n][m] in registers, streams b = A[n+dr][m+k], and accumulates the
// product of every column lag dc in its own register, so the chunk's sums for
// the pair's Q combinations need no cross-thread reduction. Every product is
// formed once.
#include <cuda_runtime.h>

#include "cov_launch.h"
#include "rec_common.cuh"

namespace cov {

template <typename T, int QMAX, int RC>
__global__ void __launch_bounds__(256) k_fringe_rows(const RecParams p) {
  using C2 = typename C2t<T>::type;
  extern __shared__ __align__(16) unsigned char smem_k2[];
  C2 *S = (C2 *)smem_k2;
  pdl_launch_dependents();
  const int P = p.P, Q = p.Q, N = p.N, M = p.M;
  const int npairs = (P - 1) * (2 * P - 1);
  const int nblk = (npairs + 255) / 256;
  int bid = blockIdx.x;
  const int pb = bid % nblk;
  bid /= nblk;
  const int cc = bid % p.NCH, side = bid / p.NCH;
  const int c0 = (Q - 1) + cc * p.CWF;  // first inner column of the chunk
  const int c_end = (c0 + p.CWF) < (M - Q + 1) ? (c0 + p.CWF) : (M - Q + 1);
  const int row0 = side == 0 ? 0 : N - 2 * P + 2;  // first staged row
  const int SR = 2 * P - 2, SP = p.FPITCH;
  const C2 *A = (const C2 *)p.A;
  for (int e = threadIdx.x; e < SR * SP; e += blockDim.x) {
    const int r = e / SP, c = e - r * SP;
    const int gr = row0 + r, gc = c0 + c;
    const bool ok = gr >= 0 && gr < N && gc < M;
    const C2 *src = ok ? A + (long long)gr * p.lda + gc : A;
    if (sizeof(C2) == 8)
      cp_async_8(S + e, src, ok);
    else
      cp_async_16(S + e, src, ok);
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();

  const int t = pb * 256 + threadIdx.x;
  if (t < npairs) {
    const int r = t % (P - 1), dr = t / (P - 1) - (P - 1);
    const int n = side == 0 ? r : (N - P + 1) + r;
    const int fr = side * (P - 1) + r;
    const int nb = n + dr;
    C2 acc[QMAX];
#pragma unroll
    for (int k = 0; k < QMAX; ++k) acc[k] = czero<C2>();
    if (nb >= 0 && nb < N) {
      const C2 *Sa = S + (n - row0) * SP;
      const C2 *Sb = S + (nb - row0) * SP;
      const int ncols = c_end - c0;
      for (int m0 = 0; m0 < ncols; m0 += RC) {
        C2 a[RC];
#pragma unroll
        for (int j = 0; j < RC; ++j) a[j] = (m0 + j < ncols) ? Sa[m0 + j] : czero<C2>();
#pragma unroll
        for (int k = 0; k < RC + QMAX - 1; ++k) {
          const C2 b = Sb[m0 + k];
#pragma unroll
          for (int j = 0; j < RC; ++j) {
            const int dc = k - j;
            if (dc >= 0 && dc < QMAX) cmac_conj(acc[dc], a[j], b);
          }
        }
      }
    }
    C2 *out = (C2 *)p.sin_part;
#pragma unroll
    for (int dc = 0; dc < QMAX; ++dc) {
      if (dc < p.dc_lo || dc >= p.dc_hi || (dc == 0 && dr < 0)) continue;
      const int D = combo_index(P, dr, dc);
      out[((long long)D * p.NFR + fr) * p.NCH + cc] = acc[dc];
    }
  }
  // The next kernels read this kernel's and the product kernel's output: do
  // not complete before the product kernel has.
  pdl_wait();
}

template <typename T, int QMAX>
static cudaError_t launch_fringe_q(const RecParams &p, cudaStream_t s, bool pdl) {
  auto kern = k_fringe_rows<T, QMAX, 8>;
  const int npairs = (p.P - 1) * (2 * p.P - 1);
  const long long grid = 2LL * p.NCH * ((npairs + 255) / 256);
  const size_t smem = (size_t)(2 * p.P - 2) * p.FPITCH * sizeof(typename C2t<T>::type);
  cudaError_t e = ensure_smem_attr(kern, smem);
  if (e != cudaSuccess) return e;
  return launch_k(kern, dim3((unsigned)grid), dim3(256), smem, s, pdl, p);
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
