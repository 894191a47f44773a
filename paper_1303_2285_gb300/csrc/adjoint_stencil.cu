// Stencil form of the adjoint (not in the paper; it reuses the paper's
// combination structure, Sections 3.1-3.3, for the derivative of Eq. 2.2).
//
// With H = (G + G^H)/K (G + G^H for the plain sum) the dense adjoint is
//   dA[n][m] = sum over windows w = (p, q) holding (n, m) of (H x_w)[a],
//   a = (n - p) + P (m - q).
// Writing b = a + Delta, Delta = (dr, dc) a combination (both signs), gives
// x_w[b] = A[n + dr][m + dc] for every such window, so
//   dA[n][m] = sum over Delta of T_Delta(n, m) * A[n + dr][m + dc],
//   T_Delta(n, m) = sum of H[a][a + Delta] over the a that some valid window
//                   places on (n, m) and with a + Delta inside the window.
// The admissible a form the rectangle i_a in I(n), j_a in J(m) with
// I(n) = [max(0, n - (N-P)), min(P-1, n)], so T depends on (n, m) only through
// a row class (2P-1 of them: the P-1 top fringe rows, the inner rows, the P-1
// bottom fringe rows) and a column class (2Q-1). Kernel 1 tabulates
// T[class][Delta] from prefix and suffix sums of H along each Delta; kernel 2
// applies the inner-class stencil (a 2-D correlation with (2P-1)(2Q-1)
// weights) to the inner rows and columns from a staged tile of A; kernel 3
// takes the fringe elements one by one; blockIdx.y indexes a batch of
// equal-shape members with fixed strides. Every element of dA has one writer;
// no atomics. Work: (2P-1)(2Q-1) complex MACs per element instead of (PQ)^2
// per window.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cov.h"
#include "cov_device.cuh"
#include "cov_internal.h"
#include "smem_attr.h"

namespace cov {

constexpr int kStTR = 32;  // output tile of the inner stencil: 32 rows x 32 columns,
constexpr int kStTC = 32;  // four consecutive rows a thread

struct StParams {
  const float2 *A;
  const float2 *G;
  float2 *T;   // [NRC * NCC][ND]
  float2 *dA;  // N x M, leading dimension M
  long long lda;
  int N, M, P, Q, Hn, W;
  long long K;
  int mean, NRC, NCC, ND;
  // batch member blockIdx.y: element strides between members
  long long sA, sG, sdA, sT;
};

// The parameters of batch member blockIdx.y.
__device__ __forceinline__ StParams member(const StParams &p0) {
  StParams p = p0;
  const long long b = blockIdx.y;
  p.A += b * p.sA;
  p.G += b * p.sG;
  p.dA += b * p.sdA;
  p.T += b * p.sT;
  return p;
}

// class -> admissible range of the window offset (rows; columns alike)
__device__ __forceinline__ void class_range(int c, int P, int &lo, int &hi) {
  if (c < P - 1) {
    lo = 0;
    hi = c;
  } else if (c == P - 1) {
    lo = 0;
    hi = P - 1;
  } else {
    lo = c - P + 1;
    hi = P - 1;
  }
}
__device__ __forceinline__ int row_class(int n, int P, int Hn) {
  return n < P - 1 ? n : (n < Hn ? P - 1 : P + (n - Hn));
}

// T[(rc * NCC + cc) * ND + Delta], Delta = (dr + P - 1) + (2P - 1)(dc + Q - 1).
// One warp per Delta, kStWW warps a CTA. The admissible offsets of a class
// are a prefix (top classes), the full range (inner class) or a suffix
// (bottom classes) of [0, P-1] (columns alike), so every entry is a sum of
// column prefix or suffix sums over a prefix or suffix of the columns: no
// differences, no cancellation. h[i][j] = H[(i,j)][(i+dr, j+dc)], zero where
// (i+dr, j+dc) leaves the window. The mean's 1/K is a multiplication by the
// FP32 reciprocal (within 1.5 ulp of the quotient).
constexpr int kStWW = 8;

__global__ void __launch_bounds__(kStWW * 32) k_adjs_weights(const StParams p0) {
  const StParams p = member(p0);
  extern __shared__ __align__(16) unsigned char smem_w[];
  const int P = p.P, Q = p.Q, D = P * Q;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int di = blockIdx.x * kStWW + warp;
  if (di >= p.ND) return;  // whole warps; no CTA barrier below
  float2 *pre = (float2 *)smem_w + (size_t)warp * 2 * D;  // [Q][P]: sum_{i <= r} h[i][j]
  float2 *suf = pre + D;                                    // [Q][P]: sum_{i >= r} h[i][j]
  const int dr = di % (2 * P - 1) - (P - 1), dc = di / (2 * P - 1) - (Q - 1);
  for (int e = lane; e < D; e += 32) {
    const int i = e % P, j = e / P;
    float2 h = make_float2(0.f, 0.f);
    if (i + dr >= 0 && i + dr < P && j + dc >= 0 && j + dc < Q) {
      const int a = i + P * j, b = (i + dr) + P * (j + dc);
      const float2 g1 = __ldg(p.G + (long long)a * D + b), g2 = __ldg(p.G + (long long)b * D + a);
      h = make_float2(g1.x + g2.x, g1.y - g2.y);  // H[a][b] = G[a][b] + conj(G[b][a])
    }
    pre[e] = h;
    suf[e] = h;
  }
  __syncwarp();
  for (int j = lane; j < Q; j += 32) {
    for (int i = 1; i < P; ++i) {
      pre[j * P + i].x += pre[j * P + i - 1].x;
      pre[j * P + i].y += pre[j * P + i - 1].y;
    }
    for (int i = P - 2; i >= 0; --i) {
      suf[j * P + i].x += suf[j * P + i + 1].x;
      suf[j * P + i].y += suf[j * P + i + 1].y;
    }
  }
  __syncwarp();
  const float inv = p.mean ? 1.0f / (float)p.K : 1.0f;
  for (int rc = lane; rc < p.NRC; rc += 32) {
    // v[j]: the row class's range summed in column j
    const float2 *src = rc <= P - 1 ? pre + rc : suf + (rc - P + 1);
    float2 *out = p.T + (long long)rc * p.NCC * p.ND + di;
    float2 acc = make_float2(0.f, 0.f);
    for (int j = 0; j < Q; ++j) {  // column classes 0..Q-1: prefixes j' <= cc
      acc.x += src[j * P].x;
      acc.y += src[j * P].y;
      out[(long long)j * p.ND] = make_float2(acc.x * inv, acc.y * inv);
    }
    acc = make_float2(0.f, 0.f);
    for (int j = Q - 1; j >= 1; --j) {  // classes Q..2Q-2: suffixes j' >= cc - Q + 1
      acc.x += src[j * P].x;
      acc.y += src[j * P].y;
      out[(long long)(Q - 1 + j) * p.ND] = make_float2(acc.x * inv, acc.y * inv);
    }
  }
}

// Inner rows [P-1, Hn-1] x inner columns [Q-1, W-1]: one 32 x 32 tile per
// CTA, the tile of A with its (P-1, Q-1) halo and the inner-class weights in
// shared memory. Thread (ty, tx) computes rows 4ty .. 4ty+3 of column tx:
// for each dc it slides a window of four A values down the column, so each
// shared-memory load of A feeds four complex MACs (one per row).
__device__ __forceinline__ void cmac4(float2 (&acc)[4], float2 w, float2 x0, float2 x1, float2 x2,
                                      float2 x3) {
  const float2 x[4] = {x0, x1, x2, x3};
#pragma unroll
  for (int k = 0; k < 4; ++k) {  // acc += w * x
    acc[k].x = fma_rn(w.x, x[k].x, acc[k].x);
    acc[k].x = fma_rn(-w.y, x[k].y, acc[k].x);
    acc[k].y = fma_rn(w.x, x[k].y, acc[k].y);
    acc[k].y = fma_rn(w.y, x[k].x, acc[k].y);
  }
}

__global__ void __launch_bounds__(256) k_adjs_inner(const StParams p0) {
  const StParams p = member(p0);
  extern __shared__ __align__(16) unsigned char smem_st[];
  const int P = p.P, Q = p.Q, DR = 2 * P - 1;
  const int SW = kStTC + 2 * Q - 2, SH = kStTR + 2 * P - 2;
  float2 *As = (float2 *)smem_st;  // [SH][SW]
  float2 *Ws = As + SH * SW;       // [ND]
  const int n_in = p.Hn - (P - 1), m_in = p.W - (Q - 1);
  const int tiles_x = (m_in + kStTC - 1) / kStTC;
  const int n0 = (P - 1) + (blockIdx.x / tiles_x) * kStTR;
  const int m0 = (Q - 1) + (blockIdx.x % tiles_x) * kStTC;
  const float2 *Tin = p.T + (long long)((P - 1) * p.NCC + (Q - 1)) * p.ND;
  for (int e = threadIdx.x; e < p.ND; e += blockDim.x) Ws[e] = __ldg(Tin + e);
  for (int e = threadIdx.x; e < SH * SW; e += blockDim.x) {
    const int r = e / SW, c = e - r * SW;
    const int gr = n0 - (P - 1) + r, gc = m0 - (Q - 1) + c;
    As[e] = (gr < p.N && gc < p.M) ? __ldg(p.A + (long long)gr * p.lda + gc) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float2 acc[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) acc[k] = make_float2(0.f, 0.f);
  for (int dc = 0; dc < 2 * Q - 1; ++dc) {
    const float2 *wv = Ws + dc * DR;
    const float2 *col = As + (4 * ty) * SW + tx + dc;  // row 4ty of the window at dr = 0
    float2 a0 = col[0], a1 = col[SW], a2 = col[2 * SW];
    int dr = 0;
    // rows used at lag dr: 4ty+dr .. 4ty+dr+3 (at most 4ty+2P+1 < SH)
    for (; dr + 4 <= DR; dr += 4) {
      const float2 a3 = col[(dr + 3) * SW];
      cmac4(acc, wv[dr], a0, a1, a2, a3);
      const float2 a4 = col[(dr + 4) * SW];
      cmac4(acc, wv[dr + 1], a1, a2, a3, a4);
      const float2 a5 = col[(dr + 5) * SW];
      cmac4(acc, wv[dr + 2], a2, a3, a4, a5);
      const float2 a6 = col[(dr + 6) * SW];
      cmac4(acc, wv[dr + 3], a3, a4, a5, a6);
      a0 = a4;
      a1 = a5;
      a2 = a6;
    }
    for (; dr < DR; ++dr) {
      const float2 a3 = col[(dr + 3) * SW];
      cmac4(acc, wv[dr], a0, a1, a2, a3);
      a0 = a1;
      a1 = a2;
      a2 = a3;
    }
  }
  const int m = m0 + tx;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int n = n0 + 4 * ty + k;
    if (n - (P - 1) < n_in && m - (Q - 1) < m_in) p.dA[(long long)n * p.M + m] = acc[k];
  }
}

// Fringe elements (outside the inner box), one warp each: lanes take the
// column lags (coalesced loads of A), a loop takes the row lags (a lane's
// weights are consecutive in the table, four to a 32-byte sector), weights of
// the element's row and column class from the table, then a warp sum.
__global__ void __launch_bounds__(256) k_adjs_fringe(const StParams p0, long long n_fringe) {
  const StParams p = member(p0);
  const long long idx = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (idx >= n_fringe) return;
  const int P = p.P, Q = p.Q, N = p.N, M = p.M;
  // enumerate: the P-1 top rows and P-1 bottom rows (all columns), then the
  // inner rows' Q-1 left and Q-1 right columns
  const long long top = (long long)(P - 1) * M;
  int n, m;
  if (idx < 2 * top) {
    const long long r = idx / M;
    m = (int)(idx - r * M);
    n = r < P - 1 ? (int)r : (int)(p.Hn + (r - (P - 1)));
  } else {
    const long long k = idx - 2 * top;
    const int nf = 2 * (Q - 1);
    n = (P - 1) + (int)(k / nf);
    const int c = (int)(k % nf);
    m = c < Q - 1 ? c : p.W + (c - (Q - 1));
  }
  const int rc = row_class(n, P, p.Hn), cc = row_class(m, Q, p.W);
  const float2 *Tc = p.T + (long long)(rc * p.NCC + cc) * p.ND;
  float sr = 0.f, si = 0.f;
  // lanes over the column lags (coalesced A rows), a loop over the row lags
  for (int c0 = 0; c0 < 2 * Q - 1; c0 += 32) {
    const int dci = c0 + lane, mm = m + dci - (Q - 1);
    const bool cok = dci < 2 * Q - 1 && mm >= 0 && mm < M;
    for (int dri = 0; dri < 2 * P - 1; ++dri) {
      const int nn = n + dri - (P - 1);
      if (nn < 0 || nn >= N) continue;  // uniform over the warp
      if (!cok) continue;
      const float2 w = __ldg(Tc + dri + (2 * P - 1) * dci);
      const float2 a = __ldg(p.A + (long long)nn * p.lda + mm);
      sr = fma_rn(w.x, a.x, sr);
      sr = fma_rn(-w.y, a.y, sr);
      si = fma_rn(w.x, a.y, si);
      si = fma_rn(w.y, a.x, si);
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) p.dA[(long long)n * p.M + m] = make_float2(sr, si);
}

bool stencil_adjoint_ok(long long N, long long M, int P, int Q) {
  const long long ND = (2LL * P - 1) * (2LL * Q - 1);
  return N >= 2LL * P - 1 && M >= 2LL * Q - 1 && ND <= 2048;
}

size_t stencil_adjoint_workspace(int P, int Q, int batch) {
  const size_t ND = (size_t)(2 * P - 1) * (2 * Q - 1);
  return kWsHeader + (((size_t)batch * ND * ND * sizeof(float2) + 255) & ~(size_t)255);
}

cudaError_t launch_stencil_adjoint(const void *A, const void *G, long long N, long long M, int P,
                                   int Q, int mean, void *dA, void *workspace, cudaStream_t s,
                                   int batch, long long sA, long long sG, long long sdA) {
  StParams p;
  p.A = (const float2 *)A;
  p.G = (const float2 *)G;
  p.T = (float2 *)((char *)workspace + kWsHeader);
  p.dA = (float2 *)dA;
  p.lda = M;
  p.N = (int)N;
  p.M = (int)M;
  p.P = P;
  p.Q = Q;
  p.Hn = (int)(N - P + 1);
  p.W = (int)(M - Q + 1);
  p.K = (long long)p.Hn * p.W;
  p.mean = mean;
  p.NRC = 2 * P - 1;
  p.NCC = 2 * Q - 1;
  p.ND = p.NRC * p.NCC;
  p.sA = sA;
  p.sG = sG;
  p.sdA = sdA;
  p.sT = (long long)p.ND * p.NRC * p.NCC;
  const size_t wsm = (size_t)kStWW * 2 * P * Q * sizeof(float2);
  cudaError_t e;
  e = ensure_dyn_smem((const void *)k_adjs_weights, wsm, false);
  if (e != cudaSuccess) return e;
  k_adjs_weights<<<dim3((unsigned)((p.ND + kStWW - 1) / kStWW), (unsigned)batch), kStWW * 32, wsm,
                   s>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n_in = p.Hn - (P - 1), m_in = p.W - (Q - 1);
  const long long tiles =
      (long long)((n_in + kStTR - 1) / kStTR) * ((m_in + kStTC - 1) / kStTC);
  const size_t smem =
      ((size_t)(kStTR + 2 * P - 2) * (kStTC + 2 * Q - 2) + (size_t)p.ND) * sizeof(float2);
  e = ensure_dyn_smem((const void *)k_adjs_inner, smem, false);
  if (e != cudaSuccess) return e;
  k_adjs_inner<<<dim3((unsigned)tiles, (unsigned)batch), 256, smem, s>>>(p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const long long n_fringe = 2LL * (P - 1) * M + (long long)n_in * 2 * (Q - 1);
  if (n_fringe > 0)
    k_adjs_fringe<<<dim3((unsigned)((n_fringe + 7) / 8), (unsigned)batch), 256, 0, s>>>(p, n_fringe);
  return cudaGetLastError();
}

}  // namespace cov
