// Kernels 3 and 4 of the combination path: the reductions that finish the
// box sums, and the seed-and-walk writer of R (see cov_internal.h).
#include <cuda_runtime.h>

#include "cov_launch.h"
#include "rec_common.cuh"

namespace cov {

// ---------------------------------------------------------------------------
// Kernel 3: reductions that finish the box sums, one warp per task.
//  - per combination D: core = sum of the core partials, the fringe-column
//    sums CS over inner rows, and CV[D][j] = core + the fringe-column sums
//    inside the box of column offset j (suffix scan over the left fringe
//    columns, prefix scan over the right ones);
//  - per (D, fringe row fr): S_in = sum of the row's partials, the row's own
//    fringe-column products (one per lane, each formed once) and the box-row
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

template <typename T>
__global__ void __launch_bounds__(128) k_reduce(const RecParams p) {
  using C2 = typename C2t<T>::type;
  __shared__ T red_s[4][4];
  __shared__ C2 part_s[128];
  __shared__ C2 cs_s[2 * kMaxPQ];
  pdl_launch_dependents();
  pdl_wait();  // the product and fringe-row kernels' partials
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int Q = p.Q, P = p.P, W = p.M - p.Q + 1;
  const int n_own = p.u_hi - p.u_lo;
  if ((int)blockIdx.x < n_own) {
    // ---- one CTA per combination: core, fringe-column sums, CV ----------
    const int D = p.u_lo + (int)blockIdx.x;
    int dr, dc;
    combo_of(P, D, dr, dc);
    Neu<T> cr, ci;
    const long long nparts = (long long)p.n_rb * p.n_cb;
    const C2 *cp = (const C2 *)p.core_part + (long long)D * nparts;
    for (long long k0 = threadIdx.x; k0 < nparts; k0 += 8 * 128) {
      C2 x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = (k0 + 128 * u < nparts) ? cp[k0 + 128 * u] : czero<C2>();
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
    if (lane == 0) {
      red_s[wib][0] = cr.s;
      red_s[wib][1] = cr.c;
      red_s[wib][2] = ci.s;
      red_s[wib][3] = ci.c;
    }
    // fringe-column sums: thread t sums fc = t % NFC over rb = t / NFC (mod G)
    const int NFC = p.NFC;
    const int G = NFC > 0 ? 128 / NFC : 0;
    const C2 *csp = (const C2 *)p.colsum_part + (long long)D * NFC * p.n_rb;
    if (NFC > 0 && (int)threadIdx.x < NFC * G) {
      const int fc = threadIdx.x % NFC, g = threadIdx.x / NFC;
      Neu<T> sr, si;
      for (int rb0 = g; rb0 < p.n_rb; rb0 += 4 * G) {
        C2 x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          x[u] = (rb0 + u * G < p.n_rb) ? csp[(long long)fc * p.n_rb + rb0 + u * G] : czero<C2>();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          sr.add(x[u].x);
          si.add(x[u].y);
        }
      }
      C2 o;
      o.x = sr.value();
      o.y = si.value();
      part_s[threadIdx.x] = o;
    }
    __syncthreads();
    if ((int)threadIdx.x < NFC) {
      Neu<T> sr, si;
      for (int g = 0; g < G; ++g) {
        sr.add(part_s[g * NFC + threadIdx.x].x);
        si.add(part_s[g * NFC + threadIdx.x].y);
      }
      C2 o;
      o.x = sr.value();
      o.y = si.value();
      cs_s[threadIdx.x] = o;
    }
    __syncthreads();
    if (wib != 0) return;
    Neu<T> vr0, vi0;
    for (int w = 0; w < 4; ++w) {
      vr0.merge(red_s[w][0], red_s[w][1]);
      vi0.merge(red_s[w][2], red_s[w][3]);
    }
    // lane k < Q-1: fringe columns m = k (left) and m = W + k (right)
    T lr = 0, li = 0, rr = 0, ri = 0;
    if (lane < Q - 1) {
      lr = cs_s[lane].x;
      li = cs_s[lane].y;
      rr = cs_s[Q - 1 + lane].x;
      ri = cs_s[Q - 1 + lane].y;
    }
    const T lsr = scan_suffix(lr, lane), lsi = scan_suffix(li, lane);
    T rpr = scan_incl(rr, lane), rpi = scan_incl(ri, lane);
    rpr = __shfl_up_sync(0xffffffffu, rpr, 1);  // exclusive
    rpi = __shfl_up_sync(0xffffffffu, rpi, 1);
    if (lane == 0) rpr = rpi = T(0);
    const int J = Q - dc;
    if (lane < J) {
      Neu<T> vr = vr0, vi = vi0;
      vr.add(lane < Q - 1 ? lsr : T(0));
      vi.add(lane < Q - 1 ? lsi : T(0));
      vr.add(rpr);
      vi.add(rpi);
      C2 o;
      o.x = vr.value();
      o.y = vi.value();
      ((C2 *)p.colval)[(long long)D * Q + lane] = o;
    }
    return;
  }
  // ---- one warp per (combination, fringe row): RV ------------------------
  const long long w2 = ((long long)blockIdx.x - n_own) * 4 + wib;
  if (w2 >= (long long)n_own * p.NFR) return;
  const int D = p.u_lo + (int)(w2 / p.NFR), fr = (int)(w2 % p.NFR);
  int dr, dc;
  combo_of(P, D, dr, dc);
  const int n = fr < P - 1 ? fr : (p.N - P + 1) + (fr - (P - 1));
  const bool rowok = n + dr >= 0 && n + dr < p.N;
  const C2 *sp = (const C2 *)p.sin_part + ((long long)D * p.NFR + fr) * p.NCH;
  const C2 *A = (const C2 *)p.A;
  C2 lft = czero<C2>(), rgt = czero<C2>();
  C2 a0 = czero<C2>(), b0 = czero<C2>(), a1 = czero<C2>(), b1 = czero<C2>();
  const bool has_r = rowok && lane < Q - 1 && W + lane + dc < p.M;
  if (rowok && lane < Q - 1) {
    const C2 *An = A + (long long)n * p.lda;
    const C2 *Ab = A + (long long)(n + dr) * p.lda + dc;
    a0 = __ldg(An + lane);
    b0 = __ldg(Ab + lane);
    if (has_r) {
      a1 = __ldg(An + W + lane);
      b1 = __ldg(Ab + W + lane);
    }
  }
  T sr = 0, si = 0;
  for (int cc = lane; cc < p.NCH; cc += 32) {
    const C2 x = sp[cc];
    sr += x.x;
    si += x.y;
  }
  cmac_conj(lft, a0, b0);
  if (has_r) cmac_conj(rgt, a1, b1);
  sr = warp_sum(sr);
  si = warp_sum(si);
  const T lsr = scan_suffix(lft.x, lane), lsi = scan_suffix(lft.y, lane);
  T rpr = scan_incl(rgt.x, lane), rpi = scan_incl(rgt.y, lane);
  rpr = __shfl_up_sync(0xffffffffu, rpr, 1);
  rpi = __shfl_up_sync(0xffffffffu, rpi, 1);
  if (lane == 0) rpr = rpi = T(0);
  const int J = Q - dc;
  if (lane < J) {
    C2 o;
    o.x = sr + (lane < Q - 1 ? lsr : T(0)) + rpr;
    o.y = si + (lane < Q - 1 ? lsi : T(0)) + rpi;
    ((C2 *)p.rowval)[((long long)D * Q + lane) * p.NFR + fr] = o;
  }
}

// ---------------------------------------------------------------------------
// Kernel 4: one CTA per P x P block (bj, bj+dc) of R, which the combinations
// (dr, dc) own entirely (Fig. 3). The block's box-row sums RV and column
// values CV are first staged in shared memory. A thread then takes one
// diagonal segment of one combination (L outputs at most): it seeds with the
// direct sum over the box, walks down the diagonal (subtract the leaving top
// fringe row, add the entering bottom fringe row; compensated), divides by K
// and stages the block; the block and its conjugate mirror are then written
// row by row (coalesced).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_walk_write(const RecParams p) {
  using C2 = typename C2t<T>::type;
  extern __shared__ __align__(16) unsigned char smem_k4[];
  const int P = p.P, D2 = 2 * P - 1, PP = P + 1, NFR = p.NFR;
  C2 *B = (C2 *)smem_k4;                 // [P][P+1]
  C2 *RVs = B + P * PP;                  // [2P-1][NFR]
  C2 *CVs = RVs + D2 * NFR;              // [2P-1]
  int b = blockIdx.x, dc = p.dc_lo;
  while (b >= p.Q - dc) {
    b -= p.Q - dc;
    ++dc;
  }
  const int bj = b;
  pdl_wait();  // RV and CV of the reduction kernel
  const C2 *rowval = (const C2 *)p.rowval;
  const C2 *colval = (const C2 *)p.colval;
#pragma unroll 4
  // stage: every thread issues all of its loads before storing any
  {
    constexpr int U = 16;  // (2P-1)(2P-2) <= 63*62 < 16*256
    C2 v[U];
    const int total = D2 * NFR;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = threadIdx.x + u * 256;
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
      const int idx = threadIdx.x + u * 256;
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
    // rows n in [is, P-2] and the bottom fringe rows N-P+1+k, k < is
    Neu<T> orr, oii;
    orr.add(cv.x);
    oii.add(cv.y);
#pragma unroll
    for (int n = 0; n < kMaxPQ - 1; ++n)
      if (n >= is && n <= P - 2) {
        orr.add(RV[n].x);
        oii.add(RV[n].y);
      }
#pragma unroll
    for (int k = 0; k < kMaxPQ - 1; ++k)
      if (k < is) {
        orr.add(RV[P - 1 + k].x);
        oii.add(RV[P - 1 + k].y);
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

template <typename T>
static cudaError_t launch_reduce_t(const RecParams &p, cudaStream_t s, bool pdl) {
  // one block per combination of the shard; then 4 (combination, fringe row)
  // pairs per block
  const long long n_own = p.u_hi - p.u_lo;
  const long long blocks = n_own + (n_own * p.NFR + 3) / 4;
  const cudaError_t e = ensure_smem_attr(k_reduce<T>, 0);
  if (e != cudaSuccess) return e;
  return launch_k(k_reduce<T>, dim3((unsigned)blocks), dim3(128), 0, s, pdl, p);
}

template <typename T>
static cudaError_t launch_walk_t(const RecParams &p, cudaStream_t s, bool pdl) {
  int nblk = 0;  // blocks (bj, bj + dc) of the shard's column lags
  for (int dc = p.dc_lo; dc < p.dc_hi; ++dc) nblk += p.Q - dc;
  const size_t smem = ((size_t)p.P * (p.P + 1) + (size_t)(2 * p.P - 1) * (p.NFR + 1)) *
                      sizeof(typename C2t<T>::type);
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
