// Device code of the fringe-row stage of the combination path: the products
// of the fringe rows with the inner columns (see cov_internal.h for the split
// of the work), shared by the stand-alone kernel and the fused kernel.
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
#pragma once

#include <cuda_runtime.h>

#include "rec_common.cuh"

namespace cov {

// Stages the strip of A that chunk cc of side `side` reads (rows
// [row0, row0 + 2P - 2), FPITCH columns from the chunk's first column; zero
// outside A, including the rows above A that the bottom side's strip starts
// with where N < 2P-2) with cp.async by all threads of the CTA, and waits for
// the calling thread's copies. The caller synchronises the CTA before
// reading.
template <typename T>
__device__ __forceinline__ void fringe_stage(const RecParams &p, typename C2t<T>::type *S, int side,
                                             int cc) {
  using C2 = typename C2t<T>::type;
  const int P = p.P, Q = p.Q, N = p.N, M = p.M;
  const int c0 = (Q - 1) + cc * p.CWF;
  const int row0 = side == 0 ? 0 : N - 2 * P + 2;
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
}

// Pair t = (fringe row, row lag) of chunk cc of side `side`, from the staged
// strip S: the chunk's sums of the pair's products for every column lag of
// the shard, written to sin_part.
template <typename T, int QMAX, int RC>
__device__ __forceinline__ void fringe_pair(const RecParams &p, const typename C2t<T>::type *S,
                                            int side, int cc, int t) {
  using C2 = typename C2t<T>::type;
  const int P = p.P, N = p.N, M = p.M, Q = p.Q;
  const int c0 = (Q - 1) + cc * p.CWF;
  const int c_end = (c0 + p.CWF) < (M - Q + 1) ? (c0 + p.CWF) : (M - Q + 1);
  const int row0 = side == 0 ? 0 : N - 2 * P + 2;
  const int SP = p.FPITCH;
  const int r = t % (P - 1), dr = t / (P - 1) - (P - 1);
  const int fr = side * (P - 1) + r;
  if (fr >= p.NFR) return;  // N < 2P-1: the bottom side has N-P+1 rows
  const int n = fringe_row(P, p.n_inner, fr);
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
    out[((long long)D * p.NCH + cc) * p.NFR + fr] = acc[dc];
  }
}

}  // namespace cov
