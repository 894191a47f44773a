// Minimum-variance (Capon) spectra of a batch of estimates: the downstream
// use of R that Section 2.3 cites (DeGraaf's MVM SAR imaging on the
// covariance matrices of overlapping apertures; the Capon estimator).
// For each matrix R_k (D x D, Hermitian) with diagonal loading
// d_k = loading * trace(R_k) / D and each steering vector a_f,
//     P_k(f) = 1 / (a_f^H (R_k + d_k I)^{-1} a_f) = 1 / ||L_k^{-1} a_f||^2,
// where L_k L_k^H = R_k + d_k I is the Cholesky factorisation.
//
// One CTA per matrix: the lower triangle of R_k + d_k I is staged in shared
// memory and factorised in place (right-looking: per column k the pivot, the
// column scaled by it, then the trailing lower triangle updated by every
// thread of the CTA); the steering vectors are then solved in chunks of 32
// (one per lane) by forward substitution in column form, the rows of each
// update spread over the eight warps. FP32 arithmetic; a non-positive pivot
// marks the matrix's spectrum NaN.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/cov.h"

namespace cov {

constexpr int kCaponThreads = 256;
constexpr int kCaponMaxD = 128;
constexpr int kCaponChunk = 32;  // steering vectors per pass

__host__ __device__ inline size_t capon_smem_bytes(int D) {
  // L: D x (D + 1) complex (odd row pitch), y: D x 32 complex, pivots' flag
  return ((size_t)D * (D + 1) + (size_t)D * kCaponChunk) * sizeof(float2) + 16;
}

__global__ void __launch_bounds__(kCaponThreads) k_capon(const float2 *__restrict__ Rall, int D,
                                                         const float2 *__restrict__ steer, int F,
                                                         float loading, float *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_c[];
  const int LD = D + 1;
  float2 *L = (float2 *)smem_c;            // [D][D+1], lower triangle used
  float2 *Y = L + (size_t)D * LD;          // [D][32]
  int *bad = (int *)(Y + (size_t)D * kCaponChunk);
  const float2 *R = Rall + (size_t)blockIdx.x * D * D;
  const int tid = threadIdx.x;
  // ---- stage the lower triangle and the loading ---------------------------
  for (int e = tid; e < D * D; e += kCaponThreads) {
    const int i = e / D, j = e - (e / D) * D;
    if (j <= i) L[i * LD + j] = R[e];
  }
  if (tid == 0) *bad = 0;
  __syncthreads();
  __shared__ float delta_s;
  if (tid < 32) {
    float tr = 0.f;
    for (int i = tid; i < D; i += 32) tr += L[i * LD + i].x;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if (tid == 0) delta_s = loading * tr / (float)D;
  }
  __syncthreads();
  for (int i = tid; i < D; i += kCaponThreads) {
    L[i * LD + i].x += delta_s;
    L[i * LD + i].y = 0.f;
  }
  __syncthreads();
  // ---- Cholesky, right-looking ---------------------------------------------
  for (int k = 0; k < D; ++k) {
    // pivot and column k below it
    const float piv = L[k * LD + k].x;
    if (!(piv > 0.f)) {  // not positive (or NaN): the matrix is not positive definite
      if (tid == 0) *bad = 1;
      break;  // uniform: every thread read the same pivot
    }
    const float d = sqrtf(piv), rd = 1.0f / d;
    __syncthreads();  // every thread has read the pivot before it is overwritten
    if (tid == 0) L[k * LD + k] = make_float2(d, 0.f);
    for (int i = k + 1 + tid; i < D; i += kCaponThreads) {
      float2 v = L[i * LD + k];
      v.x *= rd;
      v.y *= rd;
      L[i * LD + k] = v;
    }
    __syncthreads();
    // trailing update of the lower triangle: L[i][j] -= L[i][k] conj(L[j][k]),
    // k < j <= i; thread (ty, tx) of a 16 x 16 grid takes rows k+1+ty, +16, ...
    // and, in each, the columns k+1+tx, +16, ... up to the diagonal
    {
      const int ty = tid >> 4, tx = tid & 15;
      for (int i = k + 1 + ty; i < D; i += 16) {
        const float2 a = L[i * LD + k];
        float2 *Li = L + i * LD;
        for (int j = k + 1 + tx; j <= i; j += 16) {
          const float2 b = L[j * LD + k];
          float2 v = Li[j];
          v.x -= a.x * b.x + a.y * b.y;
          v.y -= a.y * b.x - a.x * b.y;
          Li[j] = v;
        }
      }
    }
    __syncthreads();
  }
  __syncthreads();
  const bool failed = *bad != 0;
  // ---- forward substitution for the steering vectors, 32 at a time --------
  // column form: y_j = b_j / L[j][j], then b_i -= L[i][j] y_j for i > j,
  // the 32 vectors of a chunk on the lanes and the rows i over the 8 warps
  const int fv = tid & 31, g = tid >> 5;
  for (int f0 = 0; f0 < F; f0 += kCaponChunk) {
    const int f = f0 + fv;
    const bool fok = f < F;
    const float2 *a = steer + (size_t)(fok ? f : 0) * D;
    for (int i = g; i < D; i += kCaponThreads / 32)
      Y[i * kCaponChunk + fv] = fok ? a[i] : make_float2(0.f, 0.f);
    __syncthreads();
    float nrm = 0.f;
    for (int j = 0; j < D && !failed; ++j) {
      if (g == 0) {
        const float rl = 1.0f / L[j * LD + j].x;
        float2 y = Y[j * kCaponChunk + fv];
        y.x *= rl;
        y.y *= rl;
        Y[j * kCaponChunk + fv] = y;
        nrm += y.x * y.x + y.y * y.y;
      }
      __syncthreads();
      const float2 y = Y[j * kCaponChunk + fv];
      for (int i = j + 1 + g; i < D; i += kCaponThreads / 32) {
        const float2 l = L[i * LD + j];
        float2 b = Y[i * kCaponChunk + fv];
        b.x -= l.x * y.x - l.y * y.y;
        b.y -= l.x * y.y + l.y * y.x;
        Y[i * kCaponChunk + fv] = b;
      }
      __syncthreads();
    }
    if (g == 0 && fok) out[(size_t)blockIdx.x * F + f] = failed ? nanf("") : 1.0f / nrm;
    __syncthreads();  // Y is reused by the next chunk
  }
}

}  // namespace cov

extern "C" cov_status cov_capon_spectrum(const void *R, int count, int D, const void *steer, int F,
                                         float loading, float *out, cov_stream_t stream) {
  if (!R || !steer || !out || count < 1 || count > (1 << 30) || D < 1 || D > cov::kCaponMaxD ||
      F < 1 || !(loading >= 0.f))
    return COV_EINVAL;
  if (((uintptr_t)R & 7) || ((uintptr_t)steer & 7) || ((uintptr_t)out & 3)) return COV_EINVAL;
  const size_t smem = cov::capon_smem_bytes(D);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(cov::k_capon, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess) {
    cudaGetLastError();
    return COV_ECUDA;
  }
  cov::k_capon<<<count, cov::kCaponThreads, smem, (cudaStream_t)stream>>>(
      (const float2 *)R, D, (const float2 *)steer, F, loading, out);
  return cudaGetLastError() == cudaSuccess ? COV_OK : COV_ECUDA;
}
