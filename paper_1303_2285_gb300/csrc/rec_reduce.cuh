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
__device__ __forceinline__ void reduce_combo_warp(const RecParams &p, int D, int lane,
                                                  typename C2t<T>::type *cv_out = nullptr) {
  using C2 = typename C2t<T>::type;
  // CV[D][j] goes to cv_out[j] when given, else to the workspace's colval
  C2 *cvo = cv_out ? cv_out : (C2 *)p.colval + (long long)D * p.Q;
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
  if (p.NFC != 2 * (Q - 1)) {
    // window form (M < 2Q - 2): lane k holds the sums of fringe columns k and
    // k + 32 over the row blocks; lane j < J adds the HC sums of its box,
    // fetched from their lanes in order
    T c0r = 0, c0i = 0, c1r = 0, c1i = 0;
    {
      const C2 *cs = (const C2 *)p.colsum_part + (long long)D * p.n_rb * p.NFC;
      Neu<T> a, b, c, d;
      for (int rb = 0; rb < p.n_rb; ++rb) {
        const C2 x = lane < p.NFC ? cs[(long long)rb * p.NFC + lane] : czero<C2>();
        const C2 y = lane + 32 < p.NFC ? cs[(long long)rb * p.NFC + lane + 32] : czero<C2>();
        a.add(x.x);
        b.add(x.y);
        c.add(y.x);
        d.add(y.y);
      }
      c0r = a.value();
      c0i = b.value();
      c1r = c.value();
      c1i = d.value();
    }
    const int J = Q - dc;
    Neu<T> vr = cr, vi = ci;
    for (int k = 0; k < p.HC; ++k) {
      const int src = (lane + k) & 31;
      const T x0 = __shfl_sync(0xffffffffu, c0r, src), y0 = __shfl_sync(0xffffffffu, c0i, src);
      const T x1 = __shfl_sync(0xffffffffu, c1r, src), y1 = __shfl_sync(0xffffffffu, c1i, src);
      const bool hi = lane + k >= 32;
      vr.add(hi ? x1 : x0);
      vi.add(hi ? y1 : y0);
    }
    if (lane < J) {
      C2 o;
      o.x = vr.value();
      o.y = vi.value();
      cvo[lane] = o;
    }
    return;
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
    cvo[lane] = o;
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
__device__ __forceinline__ void reduce_rows_warp(const RecParams &p, int D, int lane,
                                                 typename C2t<T>::type *rv_out = nullptr) {
  using C2 = typename C2t<T>::type;
  const int P = p.P, Q = p.Q, W = p.M - p.Q + 1, NFR = p.NFR, NFC = p.NFC, NCH = p.NCH;
  int dr, dc;
  combo_of(P, D, dr, dc);
  const int J = Q - dc;
  const C2 *A = (const C2 *)p.A;
  const C2 *sin_d = (const C2 *)p.sin_part + (long long)D * NCH * NFR;
  // RV[D][j][fr] goes to rv_out[j * NFR + fr] when given, else to the
  // workspace's rowval
  C2 *rv = rv_out ? rv_out : (C2 *)p.rowval + (long long)D * Q * NFR;
  for (int fr = lane; fr < NFR; fr += 32) {
    const int n = fringe_row(P, p.n_inner, fr);
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
    if (NFC != 2 * (Q - 1)) {
      // window form (M < 2Q - 2): the row's NFC fringe-column products, each
      // formed once, then out[j] = S_in + the HC of them in the box of j
      C2 pr[2 * kMaxPQ];
      const C2 *An = A + (long long)n * p.lda;
      const C2 *Ab = A + (long long)(n + dr) * p.lda + dc;
      for (int k = 0; k < NFC; ++k) {
        const int m = fringe_col(Q, p.n_innerc, k);
        C2 v = czero<C2>();
        if (rowok && m + dc < p.M) cmac_conj(v, __ldg(An + m), __ldg(Ab + m));
        pr[k] = v;
      }
      for (int j = 0; j < J; ++j) {
        C2 w = czero<C2>();
        for (int k = j; k < j + p.HC; ++k) {
          w.x += pr[k].x;
          w.y += pr[k].y;
        }
        C2 o;
        o.x = s_r + w.x;
        o.y = s_i + w.y;
        rv[(long long)j * NFR + fr] = o;
      }
      continue;
    }
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

// ---------------------------------------------------------------------------
// The same reductions with one CTA (kRedThreads threads) per combination D,
// for the stand-alone reduction kernel. The partials of D are read by many
// threads at once (every load of a thread issued before its sums start), so a
// combination costs about one memory latency instead of one per round of a
// single warp's loop; the sums are then finished in shared memory:
//  - core: each thread a compensated sum over a strided share of the core
//    partials, the 256 states merged by one warp;
//  - CS[fc] = sum over the row blocks of the fringe-column partials: S
//    threads per fringe column, each a compensated sum over every S-th row
//    block, merged per column;
//  - S_in[fr] = sum over the column chunks of the fringe-row partials, S2
//    threads per fringe row, merged per row;
//  - the fringe-row x fringe-column products (each formed once) into a table;
//  - CV[D][j] (warp 0: suffix / prefix scans over the fringe columns as in
//    reduce_combo_warp) and RV[D][j][fr] (four threads per fringe row, each a
//    segment of the suffix over the left products and of the prefix over the
//    right ones, carried across the segments through shared memory).
// ---------------------------------------------------------------------------
constexpr int kRedThreads = 256;
constexpr int kRedSeg = 4;  // segments of the fringe-column scans per fringe row

template <typename T> struct RedSmem {
  // offsets in units of T of the regions of reduce_combo_cta's shared memory
  int prod, cs_part, sin_part, cs, sin, core, tot, core_tot;
  int total;
  __host__ __device__ RedSmem(int NFR, int NFC, int S, int S2) {
    prod = 0;                                 // [NFR][NFC | 1] complex
    cs_part = prod + 2 * NFR * (NFC | 1);     // [S][NFC] x (re s, re c, im s, im c)
    sin_part = cs_part + 4 * S * NFC;         // [S2][NFR] complex
    cs = sin_part + 2 * S2 * NFR;             // [NFC] complex
    sin = cs + 2 * NFC;                       // [NFR] complex
    core = sin + 2 * NFR;                     // [threads] x (re s, re c, im s, im c)
    tot = core + 4 * kRedThreads;             // [kRedSeg][NFR] x (left, right) complex
    core_tot = tot + 4 * kRedSeg * NFR;       // (re s, re c, im s, im c)
    total = core_tot + 4;
  }
};

// Row stride of the product table: odd in complex elements, so that the
// threads that read along a row hit different banks.
__host__ __device__ inline int red_prod_stride(int NFC) { return NFC | 1; }

__host__ __device__ inline int red_cs_slices(int NFC, int n_rb) {
  int S = NFC > 0 ? kRedThreads / NFC : 1;
  if (S > n_rb) S = n_rb;
  return S < 1 ? 1 : S;
}
__host__ __device__ inline int red_sin_slices(int NFR, int NCH) {
  int S = NFR > 0 ? kRedThreads / NFR : 1;
  if (S > NCH) S = NCH;
  return S < 1 ? 1 : S;
}
template <typename T> __host__ __device__ inline size_t reduce_cta_smem_bytes(const RecParams &p) {
  const RedSmem<T> L(p.NFR, p.NFC, red_cs_slices(p.NFC, p.n_rb), red_sin_slices(p.NFR, p.NCH));
  return (size_t)L.total * sizeof(T);
}

template <typename T>
__device__ __forceinline__ void reduce_combo_cta(const RecParams &p, int D, T *sm) {
  using C2 = typename C2t<T>::type;
  const int P = p.P, Q = p.Q, NFR = p.NFR, NFC = p.NFC, NCH = p.NCH, n_rb = p.n_rb;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int S = red_cs_slices(NFC, n_rb), S2 = red_sin_slices(NFR, NCH);
  const RedSmem<T> L(NFR, NFC, S, S2);
  // the box of a column offset holds Q - 1 fringe columns (M >= 2Q - 2):
  // suffix / prefix scans; else (M < 2Q - 2) direct window sums of HC
  const bool scan_form = NFC == 2 * (Q - 1);
  int dr, dc;
  combo_of(P, D, dr, dc);
  const int J = Q - dc;

  // ---- 1. loads and per-thread sums --------------------------------------
  // core partials [D][rb][cb]: thread tid takes tid, tid + 256, ...
  {
    Neu<T> cr, ci;
    const int nparts = n_rb * p.n_cb;
    const C2 *cp = (const C2 *)p.core_part + (long long)D * nparts;
    for (int k0 = tid; k0 < nparts; k0 += 4 * kRedThreads) {
      C2 x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (k0 + u * kRedThreads < nparts) x[u] = cp[k0 + u * kRedThreads];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (k0 + u * kRedThreads < nparts) {
          cr.add(x[u].x);
          ci.add(x[u].y);
        }
    }
    T *o = sm + L.core + 4 * tid;
    o[0] = cr.s;
    o[1] = cr.c;
    o[2] = ci.s;
    o[3] = ci.c;
  }
  // fringe-column partials [D][rb][fc]: thread (s, fc) sums rb = s, s+S, ...
  if (tid < S * NFC) {
    const int fc = tid % NFC, s0 = tid / NFC;
    const C2 *cs = (const C2 *)p.colsum_part + (long long)D * n_rb * NFC + fc;
    Neu<T> a, b;
    for (int rb0 = s0; rb0 < n_rb; rb0 += 4 * S) {
      C2 x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (rb0 + u * S < n_rb) x[u] = cs[(long long)(rb0 + u * S) * NFC];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (rb0 + u * S < n_rb) {
          a.add(x[u].x);
          b.add(x[u].y);
        }
    }
    T *o = sm + L.cs_part + 4 * (s0 * NFC + fc);
    o[0] = a.s;
    o[1] = a.c;
    o[2] = b.s;
    o[3] = b.c;
  }
  // fringe-row partials [D][chunk][fr]: thread (s, fr) sums chunks s, s+S2, ...
  if (tid < S2 * NFR) {
    const int fr = tid % NFR, s0 = tid / NFR;
    const C2 *sp = (const C2 *)p.sin_part + (long long)D * NCH * NFR + fr;
    T sr = T(0), si = T(0);
    for (int c0 = s0; c0 < NCH; c0 += 4 * S2) {
      C2 x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (c0 + u * S2 < NCH) x[u] = sp[(long long)(c0 + u * S2) * NFR];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (c0 + u * S2 < NCH) {
          sr += x[u].x;
          si += x[u].y;
        }
    }
    C2 o;
    o.x = sr;
    o.y = si;
    ((C2 *)(sm + L.sin_part))[s0 * NFR + fr] = o;
  }
  // the fringe-row x fringe-column products, each formed once (zero where
  // the partner falls outside A): warp w takes the fringe rows w, w + 8, ...;
  // lane k the fringe columns k and k + 32 (NFC <= 62); the rows' loads are
  // unrolled so that a warp's loads of all its rows are in flight together
  {
    const C2 *A = (const C2 *)p.A;
    C2 *prod = (C2 *)(sm + L.prod);
    const int PS = red_prod_stride(NFC);
    const int m0 = fringe_col(Q, p.n_innerc, lane), m1 = fringe_col(Q, p.n_innerc, lane + 32);
    const bool c0 = lane < NFC && m0 + dc < p.M, c1 = lane + 32 < NFC && m1 + dc < p.M;
#pragma unroll 8
    for (int fr = warp; fr < NFR; fr += kRedThreads / 32) {
      const int n = fringe_row(P, p.n_inner, fr);
      const bool rowok = n + dr >= 0 && n + dr < p.N;
      const C2 *An = A + (long long)n * p.lda;
      const C2 *Ab = A + (long long)(n + dr) * p.lda + dc;
      C2 a0 = czero<C2>(), b0 = czero<C2>(), a1 = czero<C2>(), b1 = czero<C2>();
      if (rowok && c0) {
        a0 = __ldg(An + m0);
        b0 = __ldg(Ab + m0);
      }
      if (rowok && c1) {
        a1 = __ldg(An + m1);
        b1 = __ldg(Ab + m1);
      }
      C2 v0 = czero<C2>(), v1 = czero<C2>();
      cmac_conj(v0, a0, b0);
      cmac_conj(v1, a1, b1);
      if (lane < NFC) prod[fr * PS + lane] = v0;
      if (lane + 32 < NFC) prod[fr * PS + lane + 32] = v1;
    }
  }
  __syncthreads();

  // ---- 2. merge the slices and the core states --------------------------
  if (tid < NFC) {
    Neu<T> a, b;
    for (int s0 = 0; s0 < S; ++s0) {
      const T *o = sm + L.cs_part + 4 * (s0 * NFC + tid);
      a.merge(o[0], o[1]);
      b.merge(o[2], o[3]);
    }
    C2 v;
    v.x = a.value();
    v.y = b.value();
    ((C2 *)(sm + L.cs))[tid] = v;
  } else if (tid >= 128 && tid - 128 < NFR) {
    const int fr = tid - 128;
    const C2 *sp = (const C2 *)(sm + L.sin_part);
    C2 v = sp[fr];
    for (int s0 = 1; s0 < S2; ++s0) {
      v.x += sp[s0 * NFR + fr].x;
      v.y += sp[s0 * NFR + fr].y;
    }
    ((C2 *)(sm + L.sin))[fr] = v;
  } else if (warp == kRedThreads / 32 - 1) {
    Neu<T> vr, vi;
    for (int t = lane; t < kRedThreads; t += 32) {
      const T *o = sm + L.core + 4 * t;
      vr.merge(o[0], o[1]);
      vi.merge(o[2], o[3]);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      const T s1 = __shfl_xor_sync(0xffffffffu, vr.s, o), c1 = __shfl_xor_sync(0xffffffffu, vr.c, o);
      const T s2 = __shfl_xor_sync(0xffffffffu, vi.s, o), c2 = __shfl_xor_sync(0xffffffffu, vi.c, o);
      vr.merge(s1, c1);
      vi.merge(s2, c2);
    }
    if (lane == 0) {
      T *o = sm + L.core_tot;
      o[0] = vr.s;
      o[1] = vr.c;
      o[2] = vi.s;
      o[3] = vi.c;
    }
  }
  __syncthreads();

  // ---- 3. RV: thread (q, fr) = segment q of fringe row fr's scans ---------
  const int NL = Q - 1;                              // fringe columns per side
  const int SEG = (NL + kRedSeg - 1) / kRedSeg;      // columns per segment
  const int q = tid / 64, fr = tid % 64;
  if (!scan_form) {
    // window form: thread (q, fr) takes the column offsets j = q, q + 4, ...
    if (fr < NFR) {
      const C2 *row = (const C2 *)(sm + L.prod) + fr * red_prod_stride(NFC);
      const C2 s_in = ((const C2 *)(sm + L.sin))[fr];
      C2 *rv = (C2 *)p.rowval + (long long)D * Q * NFR + fr;
      for (int j = q; j < J; j += kRedSeg) {
        C2 w = czero<C2>();
        for (int k = j; k < j + p.HC; ++k) {
          w.x += row[k].x;
          w.y += row[k].y;
        }
        C2 o;
        o.x = s_in.x + w.x;
        o.y = s_in.y + w.y;
        rv[(long long)j * NFR] = o;
      }
    }
  } else {
    const int k0 = q * SEG, k1 = (k0 + SEG < NL) ? k0 + SEG : NL;
    const C2 *row = (const C2 *)(sm + L.prod) + fr * red_prod_stride(NFC);
    C2 *tot = (C2 *)(sm + L.tot);
    if (fr < NFR) {
      C2 sl = czero<C2>(), sr = czero<C2>();
      for (int k = k0; k < k1; ++k) {
        sl.x += row[k].x;
        sl.y += row[k].y;
        sr.x += row[NL + k].x;
        sr.y += row[NL + k].y;
      }
      tot[2 * (q * NFR + fr)] = sl;
      tot[2 * (q * NFR + fr) + 1] = sr;
    }
    __syncthreads();
    if (fr < NFR) {
      // carries: the left sums of the later segments (suffix) and the right
      // sums of the earlier ones (prefix)
      C2 cl = czero<C2>(), cr = czero<C2>();
      for (int qq = kRedSeg - 1; qq > q; --qq) {
        cl.x += tot[2 * (qq * NFR + fr)].x;
        cl.y += tot[2 * (qq * NFR + fr)].y;
      }
      for (int qq = 0; qq < q; ++qq) {
        cr.x += tot[2 * (qq * NFR + fr) + 1].x;
        cr.y += tot[2 * (qq * NFR + fr) + 1].y;
      }
      const C2 s_in = ((const C2 *)(sm + L.sin))[fr];
      C2 *rv = (C2 *)p.rowval + (long long)D * Q * NFR + fr;
      // prefix of the right products at j = k0 is cr; the suffix of the left
      // ones at j = k is cl + the segment's left values from k on
      C2 suf[8];
      {
        C2 acc = cl;
#pragma unroll
        for (int u = 7; u >= 0; --u) {
          if (k0 + u < k1) {
            acc.x += row[k0 + u].x;
            acc.y += row[k0 + u].y;
          }
          suf[u] = acc;
        }
      }
      C2 pre = cr;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = k0 + u;
        if (j < k1) {
          if (j < J) {
            C2 o;
            o.x = s_in.x + suf[u].x + pre.x;
            o.y = s_in.y + suf[u].y + pre.y;
            rv[(long long)j * NFR] = o;
          }
          pre.x += row[NL + j].x;
          pre.y += row[NL + j].y;
        }
      }
      // the last column offset j = Q - 1 (only dc = 0 has it): no left fringe
      // column in its box, every right one
      if (q == kRedSeg - 1 && J == Q) {
        C2 o;
        o.x = s_in.x + T(0) + pre.x;
        o.y = s_in.y + T(0) + pre.y;
        rv[(long long)(Q - 1) * NFR] = o;
      }
    }
  }  // scan form

  // ---- 4. CV (warp 0) ----------------------------------------------------
  if (warp == 0 && !scan_form) {
    // window form: lane j sums the HC fringe-column sums of its box
    if (lane < J) {
      Neu<T> vr, vi;
      const T *o = sm + L.core_tot;
      vr.merge(o[0], o[1]);
      vi.merge(o[2], o[3]);
      const C2 *CS = (const C2 *)(sm + L.cs);
      for (int k = lane; k < lane + p.HC; ++k) {
        vr.add(CS[k].x);
        vi.add(CS[k].y);
      }
      C2 v;
      v.x = vr.value();
      v.y = vi.value();
      ((C2 *)p.colval)[(long long)D * Q + lane] = v;
    }
  } else if (warp == 0) {
    Neu<T> vr, vi;
    {
      const T *o = sm + L.core_tot;
      vr.merge(o[0], o[1]);
      vi.merge(o[2], o[3]);
    }
    const C2 *CS = (const C2 *)(sm + L.cs);
    const T lr = lane < Q - 1 ? CS[lane].x : T(0), li = lane < Q - 1 ? CS[lane].y : T(0);
    const T rr = lane < Q - 1 ? CS[Q - 1 + lane].x : T(0), ri = lane < Q - 1 ? CS[Q - 1 + lane].y : T(0);
    const T lsr = scan_suffix(lr, lane), lsi = scan_suffix(li, lane);
    T rpr = scan_incl(rr, lane), rpi = scan_incl(ri, lane);
    rpr = __shfl_up_sync(0xffffffffu, rpr, 1);  // exclusive
    rpi = __shfl_up_sync(0xffffffffu, rpi, 1);
    if (lane == 0) rpr = rpi = T(0);
    if (lane < J) {
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
  // stage: warp w takes the rows di = w, w + nw, ... of the (2P-1) x NFR
  // block of RV (lanes along a row's contiguous fringe rows); every thread
  // issues all of its loads before storing any
  {
    constexpr int MAXI = 8;  // 2P - 1 <= 63 rows over at least 8 warps
    const int nw = (int)blockDim.x >> 5, warp = (int)threadIdx.x >> 5, lane = threadIdx.x & 31;
    C2 v[MAXI][2];
#pragma unroll
    for (int u = 0; u < MAXI; ++u) {
      const int di = warp + u * nw, dr = di - (P - 1);
      v[u][0] = v[u][1] = czero<C2>();
      if (di < D2 && !(dc == 0 && dr < 0)) {
        const C2 *src = rowval + ((long long)combo_index(P, dr, dc) * p.Q + bj) * NFR;
        if (lane < NFR) v[u][0] = src[lane];
        if (lane + 32 < NFR) v[u][1] = src[lane + 32];
      }
    }
    C2 cvv = czero<C2>();
    if (threadIdx.x < D2) {
      const int dr = threadIdx.x - (P - 1);
      if (!(dc == 0 && dr < 0)) cvv = colval[(long long)combo_index(P, dr, dc) * p.Q + bj];
    }
#pragma unroll
    for (int u = 0; u < MAXI; ++u) {
      const int di = warp + u * nw;
      if (di < D2) {
        if (lane < NFR) RVs[di * NFR + lane] = v[u][0];
        if (lane + 32 < NFR) RVs[di * NFR + lane + 32] = v[u][1];
      }
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
    // seed: the direct sum over the box of output (is, bj): its H fringe
    // rows fr in [is, is + H) (with inner rows, the top rows n in [is, P-2]
    // and the bottom rows N-P+1+k, k < is), one contiguous range of the
    // staged entries; two interleaved compensated sums (independent
    // chains), merged
    Neu<T> orr, oii, o2r, o2i;
    orr.add(cv.x);
    oii.add(cv.y);
    {
      const int ue = is + p.H;
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
      if (i + 1 < ie) {  // walk: fringe row i leaves the box, fringe row i + H enters
        orr.add(-RV[i].x);
        oii.add(-RV[i].y);
        orr.add(RV[p.H + i].x);
        oii.add(RV[p.H + i].y);
      }
    }
  }
  __syncthreads();
  const long long DD = (long long)P * p.Q;
  C2 *R = (C2 *)p.R;
  const long long ra = (long long)P * bj, cb = (long long)P * (bj + dc);
  const int nw = (int)blockDim.x >> 5, warp = (int)threadIdx.x >> 5, lane = threadIdx.x & 31;
  // row i of the block by warps, its columns by lanes (coalesced rows of R)
  if (dc > 0) {
    for (int i = warp; i < P; i += nw)
      for (int ii = lane; ii < P; ii += 32) R[(ra + i) * DD + cb + ii] = B[i * PP + ii];
    // the conjugate mirror: row ii of block (bj + dc, bj) is column ii of B
    for (int ii = warp; ii < P; ii += nw)
      for (int i = lane; i < P; i += 32) {
        C2 v = B[i * PP + ii];
        v.y = -v.y;
        R[(cb + ii) * DD + ra + i] = v;
      }
  } else {
    for (int i = warp; i < P; i += nw)
      for (int ii = lane; ii < P; ii += 32) {
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

// ---------------------------------------------------------------------------
// Thread task: the same seed, walk and division as walk_block for one
// diagonal segment of combination (dr, dc) at column offset j, outputs
// is .. ie-1, from its box-row sums RV(u) = RV[u * rs] (any layout) and its
// CV, writing each output and its conjugate mirror to R directly (no block
// staging: for batches of small matrices, where a P x P block is too small
// to keep a CTA busy). The RV and R pointers are declared unaliased so that
// the walk's loads can be issued ahead of its stores.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void walk_segment_rv(const RecParams &p,
                                                const typename C2t<T>::type *__restrict__ RV,
                                                long long rs, typename C2t<T>::type cv,
                                                typename C2t<T>::type *__restrict__ R, int dr,
                                                int dc, int j, int is, int ie) {
  using C2 = typename C2t<T>::type;
  const int P = p.P;
  Neu<T> orr, oii, o2r, o2i;
  orr.add(cv.x);
  oii.add(cv.y);
  {
    const int ue = is + p.H;
    int u = is;
    for (; u + 2 <= ue; u += 2) {
      const C2 a = RV[u * rs], b = RV[(u + 1) * rs];
      orr.add(a.x);
      oii.add(a.y);
      o2r.add(b.x);
      o2i.add(b.y);
    }
    if (u < ue) {
      orr.add(RV[u * rs].x);
      oii.add(RV[u * rs].y);
    }
    orr.merge(o2r.s, o2r.c);
    oii.merge(o2i.s, o2i.c);
  }
  const long long DD = (long long)P * p.Q;
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
    const long long a = i + (long long)P * j, b = (i + dr) + (long long)P * (j + dc);
    C2 o;
    o.x = re;
    o.y = im;
    R[a * DD + b] = o;
    if (a != b) {
      o.y = -im;
      R[b * DD + a] = o;
    }
    if (i + 1 < ie) {
      orr.add(-RV[i * rs].x);
      oii.add(-RV[i * rs].y);
      orr.add(RV[(p.H + i) * rs].x);
      oii.add(RV[(p.H + i) * rs].y);
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
