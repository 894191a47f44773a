// The plain per-element path: each element of R as a direct FP64 sum over all
// K window positions (Eq. 2.2 evaluated element by element, the
// straightforward serial algorithm of Section 2.4 with one thread per
// element). It repeats every product and is the comparison baseline of the
// combination path.
#include <cuda_runtime.h>

#include "cov_device.cuh"
#include "cov_launch.h"

namespace cov {

template <typename C2>
__global__ void __launch_bounds__(256) k_direct(const DirectParams p) {
  if (blockIdx.y > blockIdx.x) return;  // tile entirely below the diagonal
  const int D = p.P * p.Q;
  const int a = blockIdx.y * 16 + threadIdx.y;
  const int b = blockIdx.x * 16 + threadIdx.x;
  if (a >= D || b >= D || b < a) return;
  const int ia = a % p.P, ja = a / p.P, ib = b % p.P, jb = b / p.P;
  const C2 *A = (const C2 *)p.A;
  double re = 0.0, im = 0.0;
  for (int pp = 0; pp + p.P <= p.N; ++pp) {
    const C2 *ra = A + (long long)(pp + ia) * p.lda + ja;
    const C2 *rb = A + (long long)(pp + ib) * p.lda + jb;
    for (int q = 0; q + p.Q <= p.M; ++q) {
      const C2 xa = ra[q], xb = rb[q];
      const double ar = (double)xa.x, ai = (double)xa.y;
      const double br = (double)xb.x, bi = (double)xb.y;
      re = __fma_rn(ar, br, re);
      re = __fma_rn(ai, bi, re);
      im = __fma_rn(ai, br, im);
      im = __fma_rn(-ar, bi, im);
    }
  }
  if (p.mean) {
    re = re / (double)p.K;
    im = im / (double)p.K;
  }
  if (a == b) im = 0.0;
  C2 *R = (C2 *)p.R;
  C2 o;
  o.x = (decltype(o.x))re;
  o.y = (decltype(o.y))im;
  R[(long long)a * D + b] = o;
  o.y = -o.y;
  if (a == b) o.y = 0;
  R[(long long)b * D + a] = o;
}

cudaError_t launch_direct(const DirectParams &p, bool c128, cudaStream_t s) {
  const int D = p.P * p.Q;
  const dim3 block(16, 16);
  const dim3 grid((D + 15) / 16, (D + 15) / 16);
  if (c128)
    k_direct<double2><<<grid, block, 0, s>>>(p);
  else
    k_direct<float2><<<grid, block, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace cov
