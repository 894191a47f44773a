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
// applies the one-class runs of the fringe (fringe rows over inner columns,
// inner rows over fringe columns) from staged strips of A; kernel 4 takes the
// corner elements one by one; blockIdx.y indexes a batch of
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

constexpr int kStRPT = 8;             // consecutive output rows a thread of the inner stencil
constexpr int kStTR = 8 * kStRPT;     // its output tile: 8 warps x kStRPT rows
constexpr int kStTC = 32;             // x 32 columns

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
// One warp per Delta, kStWW warps a CTA (the CTA's outputs are staged and
// written lag-contiguous). The admissible offsets of a class
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
  const int d0 = blockIdx.x * kStWW, di = d0 + warp;
  const int NCP = p.NRC * p.NCC;
  float2 *pre = (float2 *)smem_w + (size_t)warp * 2 * D;  // [Q][P]: sum_{i <= r} h[i][j]
  float2 *suf = pre + D;                                    // [Q][P]: sum_{i >= r} h[i][j]
  float2 *ob = (float2 *)smem_w + (size_t)kStWW * 2 * D;   // [class pair][warp]: the CTA's outputs
  if (di < p.ND) {
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
      float2 *out = ob + (size_t)rc * p.NCC * kStWW + warp;
      float2 acc = make_float2(0.f, 0.f);
      for (int j = 0; j < Q; ++j) {  // column classes 0..Q-1: prefixes j' <= cc
        acc.x += src[j * P].x;
        acc.y += src[j * P].y;
        out[j * kStWW] = make_float2(acc.x * inv, acc.y * inv);
      }
      acc = make_float2(0.f, 0.f);
      for (int j = Q - 1; j >= 1; --j) {  // classes Q..2Q-2: suffixes j' >= cc - Q + 1
        acc.x += src[j * P].x;
        acc.y += src[j * P].y;
        out[(Q - 1 + j) * kStWW] = make_float2(acc.x * inv, acc.y * inv);
      }
    }
  }
  __syncthreads();
  // the CTA's eight consecutive lags of every class pair, contiguous in T
  const int nw = p.ND - d0 < kStWW ? p.ND - d0 : kStWW;
  for (int e = threadIdx.x; e < NCP * kStWW; e += blockDim.x) {
    const int cp = e / kStWW, w = e - cp * kStWW;
    if (w < nw) p.T[(long long)cp * p.ND + d0 + w] = ob[e];
  }
}

// Inner rows [P-1, Hn-1] x inner columns [Q-1, W-1]: one 32 x 32 tile per
// CTA, the tile of A with its (P-1, Q-1) halo and the inner-class weights
// (pre-paired for packed FP32x2 FMA) in shared memory; each A value is
// swapped once in registers, when it enters the window. Thread (ty, tx) computes rows 4ty ..
// 4ty+3 of column tx: for each dc it slides a window of four A values down
// the column, so each shared-memory load of A feeds four complex MACs (one
// per row).
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

// Packed FP32x2 form of acc += w * x for four consecutive rows: with the
// weight pre-paired as wxx = (wr, wr), wyy = (-wi, wi) and each A value x =
// (xr, xi) held both as loaded and swapped (xs = (xi, xr), formed once),
//   acc += wxx * x + wyy * xs = (wr xr - wi xi, wr xi + wi xr),
// two fma.rn.f32x2 per complex MAC.
__device__ __forceinline__ void cmac4_f2(unsigned long long (&acc)[4], unsigned long long wxx,
                                         unsigned long long wyy, const unsigned long long (&x)[4],
                                         const unsigned long long (&xs)[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    ffma2(acc[k], wxx, x[k]);
    ffma2(acc[k], wyy, xs[k]);
  }
}

__global__ void __launch_bounds__(256) k_adjs_inner(const StParams p0) {
  const StParams p = member(p0);
  extern __shared__ __align__(16) unsigned char smem_st[];
  const int P = p.P, Q = p.Q, DR = 2 * P - 1;
  const int SW = kStTC + 2 * Q - 2, SH = kStTR + 2 * P - 2;
  ulonglong2 *Ws = (ulonglong2 *)smem_st;                        // [ND]: (wxx, wyy)
  unsigned long long *As = (unsigned long long *)(Ws + p.ND);   // [SH][SW] (re, im)
  const int n_in = p.Hn - (P - 1), m_in = p.W - (Q - 1);
  const int tiles_x = (m_in + kStTC - 1) / kStTC;
  const int n0 = (P - 1) + (blockIdx.x / tiles_x) * kStTR;
  const int m0 = (Q - 1) + (blockIdx.x % tiles_x) * kStTC;
  const float2 *Tin = p.T + (long long)((P - 1) * p.NCC + (Q - 1)) * p.ND;
  for (int e = threadIdx.x; e < p.ND; e += blockDim.x) {
    const float2 w = __ldg(Tin + e);
    Ws[e] = make_ulonglong2(pk2(w.x, w.x), pk2(-w.y, w.y));
  }
  for (int e = threadIdx.x; e < SH * SW; e += blockDim.x) {
    const int r = e / SW, c = e - r * SW;
    const int gr = n0 - (P - 1) + r, gc = m0 - (Q - 1) + c;
    const float2 v =
        (gr < p.N && gc < p.M) ? __ldg(p.A + (long long)gr * p.lda + gc) : make_float2(0.f, 0.f);
    As[e] = pk2(v.x, v.y);
  }
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  constexpr int RPT = kStRPT;
  unsigned long long acc[RPT];
#pragma unroll
  for (int k = 0; k < RPT; ++k) acc[k] = 0ull;
  for (int dc = 0; dc < 2 * Q - 1; ++dc) {
    const ulonglong2 *wv = Ws + dc * DR;
    const int base = (RPT * ty) * SW + tx + dc;  // row RPT*ty of the window at dr = 0
    const unsigned long long *col = As + base;
    unsigned long long x[RPT - 1], xs[RPT - 1];
#pragma unroll
    for (int u = 0; u < RPT - 1; ++u) {
      x[u] = col[u * SW];
      xs[u] = swap2(x[u]);
    }
    // rows used at lag dr: RPT*ty+dr .. RPT*ty+dr+RPT-1 (at most
    // 8*RPT+2P-3 < SH); four lags per round, so that the window rotates by
    // register renaming
    int dr = 0;
    for (; dr + 4 <= DR; dr += 4) {
      unsigned long long y[RPT + 3], ys[RPT + 3];
#pragma unroll
      for (int u = 0; u < RPT - 1; ++u) {
        y[u] = x[u];
        ys[u] = xs[u];
      }
#pragma unroll
      for (int u = RPT - 1; u < RPT + 3; ++u) {
        y[u] = col[(dr + u) * SW];
        ys[u] = swap2(y[u]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const ulonglong2 w = wv[dr + u];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
          ffma2(acc[k], w.x, y[u + k]);
          ffma2(acc[k], w.y, ys[u + k]);
        }
      }
#pragma unroll
      for (int u = 0; u < RPT - 1; ++u) {
        x[u] = y[u + 4];
        xs[u] = ys[u + 4];
      }
    }
    for (; dr < DR; ++dr) {
      const unsigned long long xl = col[(dr + RPT - 1) * SW], xls = swap2(xl);
      const ulonglong2 w = wv[dr];
#pragma unroll
      for (int k = 0; k < RPT - 1; ++k) {
        ffma2(acc[k], w.x, x[k]);
        ffma2(acc[k], w.y, xs[k]);
      }
      ffma2(acc[RPT - 1], w.x, xl);
      ffma2(acc[RPT - 1], w.y, xls);
#pragma unroll
      for (int k = 0; k < RPT - 2; ++k) {
        x[k] = x[k + 1];
        xs[k] = xs[k + 1];
      }
      x[RPT - 2] = xl;
      xs[RPT - 2] = xls;
    }
  }
  const int m = m0 + tx;
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int n = n0 + RPT * ty + k;
    if (n - (P - 1) < n_in && m - (Q - 1) < m_in) p.dA[(long long)n * p.M + m] = upk2(acc[k]);
  }
}

// Corner elements (a fringe row and a fringe column, so the row and the column
// class both vary from element to element), one warp each: lanes take the
// column lags (coalesced loads of A), a loop takes the row lags (a lane's
// weights are consecutive in the table, four to a 32-byte sector), weights of
// the element's row and column class from the table, then a warp sum.
__global__ void __launch_bounds__(256) k_adjs_fringe(const StParams p0, long long n_fringe) {
  const StParams p = member(p0);
  const long long idx = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (idx >= n_fringe) return;
  const int P = p.P, Q = p.Q, N = p.N, M = p.M;
  // enumerate the corners: fringe rows (P-1 top, P-1 bottom) x fringe
  // columns (Q-1 left, Q-1 right)
  const int nfc = 2 * (Q - 1);
  const int fr = (int)(idx / nfc), fc = (int)(idx % nfc);
  const int n = fr < P - 1 ? fr : p.Hn + (fr - (P - 1));
  const int m = fc < Q - 1 ? fc : p.W + (fc - (Q - 1));
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

// Fringe elements in runs of one class: the top and bottom fringe rows over
// the inner columns (each row one class, a horizontal run) and the inner rows
// over the left and right fringe columns (each column one class, a vertical
// run). A CTA takes four runs of one side (a warp each) over 128 elements of
// the run direction (four consecutive elements a lane). The strip of A it
// needs is staged in shared memory with the run direction contiguous (a
// vertical run's strip transposed), zero outside A, and one padding slot after every four elements, so that the
// lanes' loads, four elements apart, fall in different banks; each run's class
// table, pre-paired for packed FP32x2 FMA (as the inner stencil), is staged
// too. A lane keeps a sliding window of four A values along the run, so each
// shared-memory load of A feeds four complex MACs with the same weight. The
// corner elements (fringe row and fringe column) go to k_adjs_fringe.
constexpr int kStRunLen = 128;   // elements of a run per CTA: four a lane
constexpr int kStRuns = 4;       // runs (warps) per CTA

__host__ __device__ inline int band_padded(int i) { return i + (i >> 2); }
// staged strip: (runs + 2 across-halo) rows of (run length + 2 along-halo)
// elements, padded
__host__ __device__ inline size_t band_smem_bytes(int P, int Q) {
  const int ah = 2 * P - 2, ch = 2 * Q - 2;
  const int a = (kStRuns + ah) * (band_padded(kStRunLen + ch) + 1);
  const int b = (kStRuns + ch) * (band_padded(kStRunLen + ah) + 1);
  const size_t nd = (size_t)(2 * P - 1) * (2 * Q - 1);
  // the strip and each run's pre-paired weights
  return (size_t)(a > b ? a : b) * sizeof(float2) + kStRuns * nd * sizeof(ulonglong2);
}

template <bool HORIZ>
__global__ void __launch_bounds__(kStRuns * 32) k_adjs_band(const StParams p0) {
  const StParams p = member(p0);
  extern __shared__ __align__(16) unsigned char smem_b[];
  const int P = p.P, Q = p.Q, DR = 2 * P - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // "across" = the runs' direction of separation (rows for horizontal runs),
  // "along" = the run direction
  const int HA = HORIZ ? P - 1 : Q - 1;   // across halo = lag reach across
  const int HB = HORIZ ? Q - 1 : P - 1;   // along halo
  const int DA = 2 * HA + 1, DB = 2 * HB + 1;
  const int nrun = HORIZ ? P - 1 : Q - 1;
  const int ngrp = (nrun + kStRuns - 1) / kStRuns;
  const int len = HORIZ ? p.W - (Q - 1) : p.Hn - (P - 1);
  const int ntile = (len + kStRunLen - 1) / kStRunLen;
  int b = blockIdx.x;
  const int tile = b % ntile;
  b /= ntile;
  const int grp = b % ngrp, side = b / ngrp;
  const int r0 = grp * kStRuns;                         // first run of the CTA within its side
  const int t0 = HB + tile * kStRunLen;                 // first element along the runs
  const int lim = HORIZ ? p.Hn : p.W;                   // first bottom / right fringe index
  const int acr0 = (side == 0 ? r0 : lim + r0) - HA;    // first staged across index
  const int alo0 = t0 - HB;                             // first staged along index
  const int SA = kStRuns + 2 * HA;                      // staged across lines
  const int SB = kStRunLen + 2 * HB;                    // staged along elements
  const int SBp = band_padded(SB) + 1;                  // padded line pitch
  const int NA = HORIZ ? p.N : p.M, NB = HORIZ ? p.M : p.N;
  ulonglong2 *Wt = (ulonglong2 *)smem_b;                                  // [runs][ND]
  unsigned long long *As = (unsigned long long *)(Wt + kStRuns * p.ND);   // [SA][SBp]
  for (int e = threadIdx.x; e < SA * SB; e += blockDim.x) {
    const int x = e / SB, y = e - x * SB;  // along fastest: coalesced rows for horizontal runs
    const int ga = acr0 + x, gb = alo0 + y;
    const int gr = HORIZ ? ga : gb, gc = HORIZ ? gb : ga;
    const float2 v = (ga >= 0 && ga < NA && gb >= 0 && gb < NB)
                         ? __ldg(p.A + (long long)gr * p.lda + gc)
                         : make_float2(0.f, 0.f);
    As[x * SBp + band_padded(y)] = pk2(v.x, v.y);
  }
  // each run's class table, pre-paired, in the order (across lag, along lag)
  for (int w = 0; w < kStRuns; ++w) {
    const int rr = r0 + w;
    if (rr >= nrun) break;
    const int cls = side == 0 ? rr : (HORIZ ? P : Q) + rr;
    const float2 *Tc = HORIZ ? p.T + (long long)(cls * p.NCC + (Q - 1)) * p.ND
                             : p.T + (long long)((P - 1) * p.NCC + cls) * p.ND;
    for (int e = threadIdx.x; e < p.ND; e += blockDim.x) {
      // e = da * DB + db; table index dri + DR * dci
      const int da = e / DB, db = e - da * DB;
      const float2 wv = __ldg(Tc + (HORIZ ? da + DR * db : db + DR * da));
      Wt[w * p.ND + e] = make_ulonglong2(pk2(wv.x, wv.x), pk2(-wv.y, wv.y));
    }
  }
  __syncthreads();
  const int r = r0 + warp;
  if (r >= nrun) return;
  const int pos = side == 0 ? r : lim + r;  // the run's row (column)
  const ulonglong2 *wt = Wt + warp * p.ND;
  unsigned long long acc[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) acc[k] = 0ull;
  const int e0 = 4 * lane;  // the lane's first element along the run, within the tile
  for (int da = 0; da < DA; ++da) {
    const int lo = (pos + da - HA - acr0) * SBp;
    const unsigned long long *line = As + lo;
    const ulonglong2 *wv = wt + da * DB;
    // element e0 + k at along lag db is staged element e0 + k + db
    unsigned long long x[3], xs[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      x[u] = line[band_padded(e0 + u)];
      xs[u] = swap2(x[u]);
    }
    int db = 0;
    for (; db + 4 <= DB; db += 4) {
      unsigned long long y[7], ys[7];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        y[u] = x[u];
        ys[u] = xs[u];
      }
#pragma unroll
      for (int u = 3; u < 7; ++u) {
        y[u] = line[band_padded(e0 + db + u)];
        ys[u] = swap2(y[u]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const ulonglong2 w = wv[db + u];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          ffma2(acc[k], w.x, y[u + k]);
          ffma2(acc[k], w.y, ys[u + k]);
        }
      }
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        x[u] = y[u + 4];
        xs[u] = ys[u + 4];
      }
    }
    for (; db < DB; ++db) {
      const unsigned long long x3 = line[band_padded(e0 + db + 3)], xs3 = swap2(x3);
      const unsigned long long xx[4] = {x[0], x[1], x[2], x3}, xxs[4] = {xs[0], xs[1], xs[2], xs3};
      const ulonglong2 w = wv[db];
      cmac4_f2(acc, w.x, w.y, xx, xxs);
      x[0] = x[1];
      x[1] = x[2];
      x[2] = x3;
      xs[0] = xs[1];
      xs[1] = xs[2];
      xs[2] = xs3;
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int t = e0 + k;
    if (t < kStRunLen && tile * kStRunLen + t < len) {
      const int n = HORIZ ? pos : t0 + t, m = HORIZ ? t0 + t : pos;
      p.dA[(long long)n * p.M + m] = upk2(acc[k]);
    }
  }
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
  const size_t wsm = ((size_t)kStWW * 2 * P * Q + (size_t)kStWW * p.NRC * p.NCC) * sizeof(float2);
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
  const size_t smem = (size_t)p.ND * sizeof(ulonglong2) +
                      (size_t)(kStTR + 2 * P - 2) * (kStTC + 2 * Q - 2) * sizeof(float2);
  e = ensure_dyn_smem((const void *)k_adjs_inner, smem, false);
  if (e != cudaSuccess) return e;
  k_adjs_inner<<<dim3((unsigned)tiles, (unsigned)batch), 256, smem, s>>>(p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the fringe runs: two sides x groups of four runs x tiles of 128 elements
  const size_t bsm = band_smem_bytes(P, Q);
  if (P > 1 && m_in > 0) {
    e = ensure_dyn_smem((const void *)k_adjs_band<true>, bsm, false);
    if (e != cudaSuccess) return e;
    const long long blocks =
        2LL * ((P - 1 + kStRuns - 1) / kStRuns) * ((m_in + kStRunLen - 1) / kStRunLen);
    k_adjs_band<true><<<dim3((unsigned)blocks, (unsigned)batch), kStRuns * 32, bsm, s>>>(p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (Q > 1 && n_in > 0) {
    e = ensure_dyn_smem((const void *)k_adjs_band<false>, bsm, false);
    if (e != cudaSuccess) return e;
    const long long blocks =
        2LL * ((Q - 1 + kStRuns - 1) / kStRuns) * ((n_in + kStRunLen - 1) / kStRunLen);
    k_adjs_band<false><<<dim3((unsigned)blocks, (unsigned)batch), kStRuns * 32, bsm, s>>>(p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const long long n_corner = 4LL * (P - 1) * (Q - 1);
  if (n_corner > 0)
    k_adjs_fringe<<<dim3((unsigned)((n_corner + 7) / 8), (unsigned)batch), 256, 0, s>>>(p, n_corner);
  return cudaGetLastError();
}

}  // namespace cov
