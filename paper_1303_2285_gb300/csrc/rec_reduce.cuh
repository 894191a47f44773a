// Device code of the reduction and walk stages of the combination path (see
// cov_internal.h), shared by the stand-alone kernels and the fused kernel.
#pragma once

#include <cuda_runtime.h>

#include "rec_common.cuh"

namespace cov {

// ---------------------------------------------------------------------------
// Reductions that finish the box sums, one warp per task.
//  - per combination D: core = sum of the core partials, the fringe-column
//    sums CS over inner rows, and CV[D][j] = core + the fringe-column sums
//    inside the box of column offset j (suffix scan over the left fringe
//    columns, prefix scan over the right ones);
//  - per D, one lane per fringe row fr: S_in = sum of the row's partials,
//    the row's own fringe-column products (each formed once) and the box-row
//    sums RV[D][j][fr] = S_in + the fringe-column products inside the box.
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
// inclusive scan over lanes k <= lane
template <typename T> __device__ __forceinline__ T scan_incl(T x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}
// inclusive scan over lanes k >= lane
template <typename T> __device__ __forceinline__ T scan_suffix(T x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_down_sync(0xffffffffu, x, o);
    if (lane + o < 32) x += y;
  }
  return x;
}

// Warp task: CV[D][j] for every column offset j of combination D = the sum
// of its core partials plus the fringe-column sums (over the inner rows)
// inside the box of column offset j (suffix scan over the left fringe
// columns, prefix scan over the right ones).
template <typename T>
__device__ __forceinline__ void reduce_combo_warp(const RecParams &p, int D, int lane) {
  using C2 = typename C2t<T>::type;
  const int P = p.P, Q = p.Q;
  int dr, dc;
  combo_of(P, D, dr, dc);
  Neu<T> cr, ci;
  const long long nparts = (long long)p.n_rb * p.n_cb;
  const C2 *cp = (const C2 *)p.core_part + (long long)D * nparts;
  for (long long k0 = lane; k0 < nparts; k0 += 8 * 32) {
    C2 x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = (k0 + 32 * u < nparts) ? cp[k0 + 32 * u] : czero<C2>();
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      cr.add(x[u].x);
      ci.add(x[u].y);
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const T s1 = __shfl_xor_sync(0xffffffffu, cr.s, o), c1 = __shfl_xor_sync(0xffffffffu, cr.c, o);
    const T s2 = __shfl_xor_sync(0xffffffffu, ci.s, o), c2 = __shfl_xor_sync(0xffffffffu, ci.c, o);
    cr.merge(s1, c1);
    ci.merge(s2, c2);
  }
  // lane k < Q-1: fringe columns m = k (left) and m = W + k (right), each
  // summed over the row blocks
  T lr = 0, li = 0, rr = 0, ri = 0;
  if (lane < Q - 1) {
    // partials [D][rb][fc]: lane's left column fc = lane, right fc = Q-1+lane
    const C2 *csl = (const C2 *)p.colsum_part + (long long)D * p.n_rb * p.NFC + lane;
    const C2 *csr = csl + (Q - 1);
    Neu<T> a, b, c, d;
    for (int rb0 = 0; rb0 < p.n_rb; rb0 += 4) {
      C2 x[4], y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        x[u] = rb0 + u < p.n_rb ? csl[(long long)(rb0 + u) * p.NFC] : czero<C2>();
        y[u] = rb0 + u < p.n_rb ? csr[(long long)(rb0 + u) * p.NFC] : czero<C2>();
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a.add(x[u].x);
        b.add(x[u].y);
        c.add(y[u].x);
        d.add(y[u].y);
      }
    }
    lr = a.value();
    li = b.value();
    rr = c.value();
    ri = d.value();
  }
  const T lsr = scan_suffix(lr, lane), lsi = scan_suffix(li, lane);
  T rpr = scan_incl(rr, lane), rpi = scan_incl(ri, lane);
  rpr = __shfl_up_sync(0xffffffffu, rpr, 1);  // exclusive
  rpi = __shfl_up_sync(0xffffffffu, rpi, 1);
  if (lane == 0) rpr = rpi = T(0);
  const int J = Q - dc;
  if (lane < J) {
    Neu<T> vr = cr, vi = ci;
    vr.add(lane < Q - 1 ? lsr : T(0));
    vi.add(lane < Q - 1 ? lsi : T(0));
    vr.add(rpr);
    vi.add(rpi);
    C2 o;
    o.x = vr.value();
    o.y = vi.value();
    ((C2 *)p.colval)[(long long)D * Q + lane] = o;
  }
}

// Warp task: the box-row sums RV[D][j][fr] of every fringe row fr of
// combination D, one lane per fringe row (no cross-lane traffic): S_in = the
// sum of the row's chunk partials (sin_part is [D][chunk][fr], so the lanes'
// loads are contiguous), plus the row's own fringe-column products (each
// formed once) inside the box of column offset j: a suffix over the left
// fringe columns k >= j and a prefix over the right ones k < j, both running
// sums in registers. The lane's J = Q - dc outputs are stored per j, lanes
// again contiguous.
template <typename T, int QMAX>
__device__ __forceinline__ void reduce_rows_warp(const RecParams &p, int D, int lane) {
  using C2 = typename C2t<T>::type;
  const int P = p.P, Q = p.Q, W = p.M - p.Q + 1, NFR = p.NFR, NCH = p.NCH;
  int dr, dc;
  combo_of(P, D, dr, dc);
  const int J = Q - dc;
  const C2 *A = (const C2 *)p.A;
  const C2 *sin_d = (const C2 *)p.sin_part + (long long)D * NCH * NFR;
  C2 *rv = (C2 *)p.rowval + (long long)D * Q * NFR;
  for (int fr = lane; fr < NFR; fr += 32) {
    const int n = fr < P - 1 ? fr : (p.N - P + 1) + (fr - (P - 1));
    const bool rowok = n + dr >= 0 && n + dr < p.N;
    // S_in: four interleaved partial sums over the chunks, 16 loads in
    // flight per round
    T sr[4] = {T(0), T(0), T(0), T(0)}, si[4] = {T(0), T(0), T(0), T(0)};
    const C2 *sp = sin_d + fr;
    for (int cc = 0; cc < NCH; cc += 16) {
      C2 x[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) x[u] = cc + u < NCH ? sp[(long long)(cc + u) * NFR] : czero<C2>();
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        sr[u & 3] += x[u].x;
        si[u & 3] += x[u].y;
      }
    }
    const T s_r = (sr[0] + sr[1]) + (sr[2] + sr[3]);
    const T s_i = (si[0] + si[1]) + (si[2] + si[3]);
    // out[j] = suffix of the left fringe-column products (k >= j)
    T outr[QMAX], outi[QMAX];
    {
      const C2 *An = A + (long long)n * p.lda;
      const C2 *Ab = A + (long long)(n + dr) * p.lda + dc;
      C2 acc = czero<C2>();
#pragma unroll
      for (int k = QMAX - 1; k >= 0; --k) {
        if (rowok && k < Q - 1) cmac_conj(acc, __ldg(An + k), __ldg(Ab + k));
        outr[k] = acc.x;
        outi[k] = acc.y;
      }
    }
    // + prefix of the right fringe-column products (k < j), then store
    {
      const C2 *An = A + (long long)n * p.lda + W;
      const C2 *Ab = A + (long long)(n + dr) * p.lda + W + dc;
      C2 acc = czero<C2>();
#pragma unroll
      for (int j = 0; j < QMAX; ++j) {
        if (j < J) {
          C2 o;
          o.x = s_r + outr[j] + acc.x;
          o.y = s_i + outi[j] + acc.y;
          rv[(long long)j * NFR + fr] = o;
        }
        if (rowok && j < Q - 1 && W + j + dc < p.M) cmac_conj(acc, __ldg(An + j), __ldg(Ab + j));
      }
    }
  }
}

// Reduction warp task w of the shard: [0, n_own) the combinations' CV, then
// [n_own, 2 n_own) their RV.
__host__ __device__ __forceinline__ int reduce_tasks(const RecParams &p) {
  return 2 * (p.u_hi - p.u_lo);
}
template <typename T, int QMAX>
__device__ __forceinline__ void reduce_task(const RecParams &p, int w, int lane) {
  const int n_own = p.u_hi - p.u_lo;
  if (w < n_own)
    reduce_combo_warp<T>(p, p.u_lo + w, lane);
  else
    reduce_rows_warp<T, QMAX>(p, p.u_lo + (w - n_own), lane);
}

// ---------------------------------------------------------------------------
// Block task: the P x P block (bj, bj+dc) of R, which the combinations
// (dr, dc) own entirely (Fig. 3). The block's box-row sums RV and column
// values CV are first staged in shared memory. A thread then takes one
// diagonal segment of one combination (L outputs at most): it seeds with the
// direct sum over the box, walks down the diagonal (subtract the leaving top
// fringe row, add the entering bottom fringe row; compensated), divides by K
// and stages the block; the block and its conjugate mirror are then written
// row by row (coalesced).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void walk_block(const RecParams &p, int dc, int bj, unsigned char *smem) {
  using C2 = typename C2t<T>::type;
  const int P = p.P, D2 = 2 * P - 1, PP = P + 1, NFR = p.NFR;
  C2 *B = (C2 *)smem;                    // [P][P+1]
  C2 *RVs = B + P * PP;                  // [2P-1][NFR]
  C2 *CVs = RVs + D2 * NFR;              // [2P-1]
  const C2 *rowval = (const C2 *)p.rowval;
  const C2 *colval = (const C2 *)p.colval;
  // stage: every thread issues all of its loads before storing any
  {
    constexpr int U = 16;  // (2P-1)(2P-2) <= 63*62 < 16*256 <= U*blockDim
    C2 v[U];
    const int total = D2 * NFR;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = threadIdx.x + u * (int)blockDim.x;
      v[u] = czero<C2>();
      if (idx < total) {
        const int di = idx / NFR, f = idx - di * NFR, dr = di - (P - 1);
        if (!(dc == 0 && dr < 0))
          v[u] = rowval[((long long)combo_index(P, dr, dc) * p.Q + bj) * NFR + f];
      }
    }
    C2 cvv = czero<C2>();
    if (threadIdx.x < D2) {
      const int dr = threadIdx.x - (P - 1);
      if (!(dc == 0 && dr < 0)) cvv = colval[(long long)combo_index(P, dr, dc) * p.Q + bj];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = threadIdx.x + u * (int)blockDim.x;
      if (idx < total) RVs[idx] = v[u];
    }
    if (threadIdx.x < D2) CVs[threadIdx.x] = cvv;
  }
  __syncthreads();
  const int nchunk = (P + p.L - 1) / p.L;
  for (int t = threadIdx.x; t < D2 * nchunk; t += blockDim.x) {
    const int dr = t % D2 - (P - 1), c = t / D2;
    if (dc == 0 && dr < 0) continue;
    const int adr = dr < 0 ? -dr : dr;
    const int I = P - adr, i0 = dr < 0 ? -dr : 0;
    const int is = i0 + c * p.L;
    if (is >= i0 + I) continue;
    const int ie = (i0 + I) < (is + p.L) ? (i0 + I) : (is + p.L);
    const C2 *RV = RVs + (dr + P - 1) * NFR;
    const C2 cv = CVs[dr + P - 1];
    // seed: the direct sum over the box of output (is, bj): the top fringe
    // rows n in [is, P-2] and the bottom fringe rows N-P+1+k, k < is, i.e.
    // the staged entries RV[is .. is+P-2], one contiguous range; two
    // interleaved compensated sums (independent chains), merged
    Neu<T> orr, oii, o2r, o2i;
    orr.add(cv.x);
    oii.add(cv.y);
    {
      const int ue = is + P - 1;
      int u = is;
      for (; u + 2 <= ue; u += 2) {
        const C2 a = RV[u], b = RV[u + 1];
        orr.add(a.x);
        oii.add(a.y);
        o2r.add(b.x);
        o2i.add(b.y);
      }
      if (u < ue) {
        orr.add(RV[u].x);
        oii.add(RV[u].y);
      }
      orr.merge(o2r.s, o2r.c);
      oii.merge(o2i.s, o2i.c);
    }
    for (int i = is; i < ie; ++i) {
      T re = orr.value(), im = oii.value();
      if (p.mean) {
        if (p.div_double) {
          re = (T)((double)re / (double)p.K);
          im = (T)((double)im / (double)p.K);
        } else {
          re = re / (T)p.K;
          im = im / (T)p.K;
        }
      }
      if (dr == 0 && dc == 0) im = T(0);
      C2 o;
      o.x = re;
      o.y = im;
      B[i * PP + i + dr] = o;
      if (i + 1 < ie) {  // walk: row i leaves the box, row i+N-P+1 enters
        orr.add(-RV[i].x);
        oii.add(-RV[i].y);
        orr.add(RV[P - 1 + i].x);
        oii.add(RV[P - 1 + i].y);
      }
    }
  }
  __syncthreads();
  const long long DD = (long long)P * p.Q;
  C2 *R = (C2 *)p.R;
  const long long ra = (long long)P * bj, cb = (long long)P * (bj + dc);
  if (dc > 0) {
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
      const int i = e / P, ii = e - i * P;
      R[(ra + i) * DD + cb + ii] = B[i * PP + ii];
    }
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
      const int ii = e / P, i = e - ii * P;
      C2 v = B[i * PP + ii];
      v.y = -v.y;
      R[(cb + ii) * DD + ra + i] = v;
    }
  } else {
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
      const int i = e / P, ii = e - i * P;
      C2 v;
      if (ii >= i) {
        v = B[i * PP + ii];
      } else {
        v = B[ii * PP + i];
        v.y = -v.y;
      }
      if (i == ii) v.y = T(0);
      R[(ra + i) * DD + ra + ii] = v;
    }
  }
}

// Blocks (bj, bj + dc) of the shard's column lags, in launch order.
__device__ __forceinline__ void walk_block_of(const RecParams &p, int b, int &dc, int &bj) {
  dc = p.dc_lo;
  while (b >= p.Q - dc) {
    b -= p.Q - dc;
    ++dc;
  }
  bj = b;
}

// Size of walk_block's shared memory.
template <typename T> __host__ __device__ constexpr size_t walk_smem_bytes(int P, int NFR) {
  return ((size_t)P * (P + 1) + (size_t)(2 * P - 1) * (NFR + 1)) * sizeof(typename C2t<T>::type);
}

}  // namespace cov
