// Device code of the product stage of the combination path (every distinct
// product over the inner rows; see cov_internal.h for the split of the work),
// shared by the stand-alone product kernel and the fused kernel.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "rec_common.cuh"

namespace cov {

// ---------------------------------------------------------------------------
// Kernel 1: products over inner rows x all columns.
//
// Work unit (warp task): one row block of TRB rows, 32 columns, one lag
// group of G lags. Tasks are ordered tile by tile (a tile = TPT row blocks x
// TC = 64 columns); each persistent CTA takes one contiguous range of tasks.
// One producer warp stages the CTA's tiles of A plus their halo in shared
// memory (TMA when A is 16-byte aligned with a 16-byte multiple row pitch,
// else cp.async), double-buffered with full/empty mbarriers; NCW consumer
// warps fetch tasks from the CTA's range through a shared-memory counter, so
// no warp waits at a tile boundary for slower warps.
//
// In a task each lane owns one column m and register-blocks R rows x G lags:
// per chunk it loads R values a = A[n][m] and R+G-1 values b = A[n+dr][m+dc]
// and forms R*G products with 4 FMA each. Lanes on inner columns are summed
// over the warp (transpose reduction) into the core partial; lanes on fringe
// columns keep their own column sums.
// ---------------------------------------------------------------------------
// Rows pw, pw + npw, ... of the tile, by producer warp pw of npw.
template <typename T, int PITCH>
__device__ void stage_tile_cpasync(const RecParams &p, long long tile,
                                   typename C2t<T>::type *S, uint64_t *full, int lane, int pw,
                                   int npw) {
  using C2 = typename C2t<T>::type;
  const int rt = (int)(tile / p.n_ct), ct = (int)(tile % p.n_ct);
  const long long r0 = (long long)p.inner_lo + (long long)rt * p.TR + p.d_lo;
  const int c0 = ct * p.TC;
  const C2 *A = (const C2 *)p.A;
  for (int sr = pw; sr < p.STR; sr += npw) {
    const long long gr = r0 + sr;
    const bool rok = gr >= 0 && gr < p.N;
    const C2 *row = A + (rok ? gr : 0) * p.lda;
    C2 *dst = S + (long long)sr * PITCH;
    for (int sc = lane; sc < PITCH; sc += 32) {
      const int gc = c0 + sc;
      const bool ok = rok && gc < p.M;
      const C2 *src = ok ? row + gc : A;
      if (sizeof(C2) == 8)
        cp_async_8(dst + sc, src, ok);
      else
        cp_async_16(dst + sc, src, ok);
    }
  }
  cp_async_mbar_arrive_noinc(full);
}

template <typename T, int G, int R, int PITCH, bool MASKED>
__device__ __forceinline__ void product_chunk(const typename C2t<T>::type *sa,
                                              const typename C2t<T>::type *sb, int valid,
                                              typename C2t<T>::type (&acc)[G]) {
  using C2 = typename C2t<T>::type;
  C2 a[R];
#pragma unroll
  for (int r = 0; r < R; ++r) a[r] = (!MASKED || r < valid) ? sa[r * PITCH] : czero<C2>();
#pragma unroll
  for (int k = 0; k < R + G - 1; ++k) {
    const C2 b = sb[k * PITCH];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int gg = k - r;
      if (gg >= 0 && gg < G) cmac_conj(acc[gg], a[r], b);
    }
  }
}

// FP32: the same products with packed FP32x2 FMA (fma.rn.f32x2). With
// a = (ar, ai) and b = (br, bi) as loaded, two accumulator pairs per lag take
//   d += (ar, ai) * (br, bi) = (ar br, ai bi)   and
//   x += (ai, ar) * (br, bi) = (ai br, ar bi),
// so that a * conj(b) summed over the rows is (d.x + d.y, x.x - x.y). b is
// used exactly as it sits in shared memory (no repacking per load); only a's
// swapped pair is formed, once per row for all G lags.

template <int G, int R, int PITCH, bool MASKED>
__device__ __forceinline__ void product_chunk_f2(const float2 *sa, const float2 *sb, int valid,
                                                 unsigned long long (&accd)[G],
                                                 unsigned long long (&accx)[G]) {
  const unsigned long long *ua = (const unsigned long long *)sa;
  const unsigned long long *ub = (const unsigned long long *)sb;
  unsigned long long a[R], as[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    a[r] = (!MASKED || r < valid) ? ua[r * PITCH] : 0ull;
    as[r] = swap2(a[r]);
  }
#pragma unroll
  for (int k = 0; k < R + G - 1; ++k) {
    const unsigned long long b = ub[k * PITCH];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int gg = k - r;
      if (gg >= 0 && gg < G) {
        ffma2(accd[gg], a[r], b);
        ffma2(accx[gg], as[r], b);
      }
    }
  }
}

template <typename T, int G, int R, int PITCH>
__device__ __forceinline__ void product_task(const RecParams &p, long long tile, long long local,
                                             const typename C2t<T>::type *S, int lane) {
  using C2 = typename C2t<T>::type;
  const int rt = (int)(tile / p.n_ct), ct = (int)(tile % p.n_ct);
  const int sub = (int)(local % p.TPT);
  const long long rest = local / p.TPT;
  const int cbl = (int)(rest % p.CBT), g = (int)(rest / p.CBT);
  const int cbg = ct * p.CBT + cbl;
  const int rb = rt * p.TPT + sub;
  if (cbg >= p.n_cb || rb >= p.n_rb) return;
  int dc, d0, cnt;
  group_of(p.P, G, p.g_lo + g, dc, d0, cnt);
  const int n0 = p.inner_lo + rb * p.TRB;
  const int rem = p.inner_lo + p.n_inner - n0;
  const int rows = rem < p.TRB ? rem : p.TRB;
  const int col_s = cbl * 32 + lane;

  C2 acc[G];
  const int srow = sub * p.TRB;  // first a-row of the task within the tile
  const C2 *Sa = S + (long long)(srow - p.d_lo) * PITCH + col_s;
  const C2 *Sb = S + (long long)(srow + d0 - p.d_lo) * PITCH + col_s + dc;
  if constexpr (sizeof(T) == 4) {
    unsigned long long accd[G], accx[G];
#pragma unroll
    for (int k = 0; k < G; ++k) accd[k] = accx[k] = 0ull;
    // Full R-row chunks, then 8-row chunks: a chunk at row r0 reads b rows up
    // to r0 + (chunk rows) + G - 2 past the task's first row, which stays in
    // the tile (and its halo) only while r0 + chunk rows <= TRB; TRB is a
    // multiple of 8, not necessarily of R.
    static_assert(R % 8 == 0, "row blocks are multiples of 8");
    int r0 = 0;
    for (; r0 + R <= rows; r0 += R)
      product_chunk_f2<G, R, PITCH, false>(Sa + r0 * PITCH, Sb + r0 * PITCH, R, accd, accx);
    for (; r0 + 8 <= rows; r0 += 8)
      product_chunk_f2<G, 8, PITCH, false>(Sa + r0 * PITCH, Sb + r0 * PITCH, 8, accd, accx);
    if (r0 < rows)
      product_chunk_f2<G, 8, PITCH, true>(Sa + r0 * PITCH, Sb + r0 * PITCH, rows - r0, accd,
                                          accx);
#pragma unroll
    for (int k = 0; k < G; ++k) {
      const float2 d = upk2(accd[k]), x = upk2(accx[k]);
      acc[k] = make_float2(d.x + d.y, x.x - x.y);
    }
  } else {
#pragma unroll
    for (int k = 0; k < G; ++k) acc[k] = czero<C2>();
    int r0 = 0;
    for (; r0 + R <= rows; r0 += R)
      product_chunk<T, G, R, PITCH, false>(Sa + r0 * PITCH, Sb + r0 * PITCH, R, acc);
    if (r0 < rows) product_chunk<T, G, R, PITCH, true>(Sa + r0 * PITCH, Sb + r0 * PITCH, rows - r0, acc);
  }

  const int m = ct * p.TC + col_s;
  const bool in_range = m < p.M;
  const bool inner = (m >= p.Q - 1) && (m <= p.M - p.Q);
  if (in_range && !inner) {
    const int fc = (m < p.Q - 1) ? m : m - p.n_innerc;
    C2 *cs = (C2 *)p.colsum_part;
#pragma unroll
    for (int k = 0; k < G; ++k)
      if (k < cnt) {
        const int D = combo_index(p.P, d0 + k, dc);
        cs[((long long)D * p.n_rb + rb) * p.NFC + fc] = acc[k];  // lanes: consecutive fc
      }
  }
  T v[2 * G];
#pragma unroll
  for (int k = 0; k < G; ++k) {
    v[2 * k] = inner ? acc[k].x : T(0);
    v[2 * k + 1] = inner ? acc[k].y : T(0);
  }
  warp_transpose_reduce<2 * G>(v, lane);
  constexpr int HS = Log2<2 * G>::v;
  const int idx = lane >> (5 - HS);
  if ((lane & ((1 << (5 - HS)) - 1)) == 0) {
    const int k = idx >> 1, comp = idx & 1;
    if (k < cnt) {
      const int D = combo_index(p.P, d0 + k, dc);
      T *cp = (T *)p.core_part;
      cp[2 * (((long long)D * p.n_rb + rb) * p.n_cb + cbg) + comp] = v[0];
    }
  }
}

template <typename T, int PITCH>
__host__ __device__ constexpr size_t tile_buf_bytes(int STR) {
  return (((size_t)STR * PITCH * sizeof(typename C2t<T>::type)) + 1023) & ~(size_t)1023;
}

// Runs the tasks [tb, te) of the product kernel in the calling CTA (NCW
// consumer warps, then NPW producer warps; `smem` holds two tile buffers and
// the barriers). With TMA the first producer warp issues each tile; with
// cp.async the NPW warps share its rows (one warp's copies queue behind the
// consumers' shared-memory loads). Every thread of the CTA calls it with the
// same range. Returns false if a bounded wait gave up (the status word is
// then set); on return the producers' copies have landed, but consumer warps
// may still be reading shared memory: synchronise the CTA before reusing it.
template <typename T, int G, int R, int PITCH, int NCW, int NPW = 1>
__device__ __forceinline__ bool products_phase(const RecParams &p, const CUtensorMap &tmap,
                                               unsigned char *smem, long long tb, long long te) {
  using C2 = typename C2t<T>::type;
  const size_t bb = tile_buf_bytes<T, PITCH>(p.STR);
  C2 *buf0 = (C2 *)smem;
  C2 *buf1 = (C2 *)(smem + bb);
  uint64_t *full = (uint64_t *)(smem + 2 * bb);
  uint64_t *empty = full + 2;
  int *ctr = (int *)(empty + 2);  // next task index within the tile held by each buffer

  if (tb >= te) return true;
  const long long tpt = p.tasks_per_tile;
  const long long tf = tb / tpt, tl = (te - 1) / tpt;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(&full[0], p.use_tma ? 1 : 32 * NPW);
    mbar_init(&full[1], p.use_tma ? 1 : 32 * NPW);
    mbar_init(&empty[0], NCW);
    mbar_init(&empty[1], NCW);
    ctr[0] = 0;
    ctr[1] = 0;
    fence_mbar_init();
  }
  __syncthreads();

  // Every warp goes through the CTA's tiles in order and waits on each tile's
  // barrier phase in turn, so a parity wait never spans more than one phase.
  if (warp >= NCW) {  // producers
    const int pw = warp - NCW;
    if (p.use_tma && pw > 0) return true;
    const unsigned bytes = (unsigned)((size_t)p.STR * PITCH * sizeof(C2));
    bool ok = true;
    long long issued = -1;  // index (from tf) of the last tile whose load was issued
    for (long long tile = tf; tile <= tl; ++tile) {
      const int b = (int)((tile - tf) & 1);
      const long long n = (tile - tf) >> 1;
      C2 *dst = b ? buf1 : buf0;
      if (n >= 1 && !mbar_wait(&empty[b], (unsigned)((n - 1) & 1), kWaitLimitNs)) {
        ok = false;
        break;
      }
      if (pw == 0 && lane == 0) ctr[b] = 0;  // all warps are done with the buffer's previous tile
      __syncwarp();
      if (p.use_tma) {
        if (lane == 0) {
          const int rt = (int)(tile / p.n_ct), ct = (int)(tile % p.n_ct);
          const int y = p.inner_lo + rt * p.TR + p.d_lo;
          const int x = ct * p.TC * (int)(sizeof(C2) / 8);
          mbar_arrive_expect_tx(&full[b], bytes);
          tma_load_2d(dst, &tmap, x, y, &full[b]);
        }
      } else {
        stage_tile_cpasync<T, PITCH>(p, tile, dst, &full[b], lane, pw, NPW);
      }
      issued = tile - tf;
    }
    if (!ok && lane == 0) *p.status = kDevTimeout;
    // Wait (bounded) for this warp's last copies before the CTA may exit or
    // reuse the buffers.
    for (long long k = (issued >= 1 ? issued - 1 : 0); k <= issued; ++k)
      if (!mbar_wait(&full[k & 1], (unsigned)((k >> 1) & 1), kWaitLimitNs)) ok = false;
    return ok;
  }

  // consumers: tasks of the current tile are handed out through ctr[b]
  for (long long tile = tf; tile <= tl; ++tile) {
    const int b = (int)((tile - tf) & 1);
    const long long n = (tile - tf) >> 1;
    if (!mbar_wait(&full[b], (unsigned)(n & 1), kWaitLimitNs)) {
      if (lane == 0) *p.status = kDevTimeout;
      return false;
    }
    const long long lo = tb > tile * tpt ? tb : tile * tpt;
    const long long hi = te < (tile + 1) * tpt ? te : (tile + 1) * tpt;
    for (;;) {
      int idx = 0;
      if (lane == 0) idx = atomicAdd(&ctr[b], 1);
      idx = __shfl_sync(0xffffffffu, idx, 0);
      if (lo + idx >= hi) break;
      product_task<T, G, R, PITCH>(p, tile, lo + idx - tile * tpt, b ? buf1 : buf0, lane);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[b]);
  }
  return true;
}

}  // namespace cov
