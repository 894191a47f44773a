// Kernel 1 of the combination path: every distinct product over the inner
// rows (see cov_internal.h for the split of the work).
#include <cuda.h>
#include <cuda_runtime.h>

#include "cov_launch.h"
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
template <typename T, int PITCH>
__device__ void stage_tile_cpasync(const RecParams &p, long long tile,
                                   typename C2t<T>::type *S, uint64_t *full, int lane) {
  using C2 = typename C2t<T>::type;
  const int rt = (int)(tile / p.n_ct), ct = (int)(tile % p.n_ct);
  const long long r0 = (long long)p.inner_lo + (long long)rt * p.TR + p.d_lo;
  const int c0 = ct * p.TC;
  const C2 *A = (const C2 *)p.A;
  for (int sr = 0; sr < p.STR; ++sr) {
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

// FP32: the same products with packed FP32x2 FMA (fma.rn.f32x2). For
// acc += a * conj(b): (re, im) += (ar, ai) * (br, br), then
// (re, im) += (ai, -ar) * (bi, bi) -- the operations of cmac_conj in the same
// order, two instructions instead of four.
__device__ __forceinline__ unsigned long long pk2(float x, float y) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
__device__ __forceinline__ void ffma2(unsigned long long &acc, unsigned long long a,
                                      unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}

template <int G, int R, int PITCH, bool MASKED>
__device__ __forceinline__ void product_chunk_f2(const float2 *sa, const float2 *sb, int valid,
                                                 unsigned long long (&acc)[G]) {
  unsigned long long a[R], as[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const float2 v = (!MASKED || r < valid) ? sa[r * PITCH] : make_float2(0.f, 0.f);
    a[r] = pk2(v.x, v.y);
    as[r] = pk2(v.y, -v.x);
  }
#pragma unroll
  for (int k = 0; k < R + G - 1; ++k) {
    const float2 b = sb[k * PITCH];
    const unsigned long long br = pk2(b.x, b.x), bi = pk2(b.y, b.y);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int gg = k - r;
      if (gg >= 0 && gg < G) {
        ffma2(acc[gg], a[r], br);
        ffma2(acc[gg], as[r], bi);
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
    unsigned long long acc2[G];
#pragma unroll
    for (int k = 0; k < G; ++k) acc2[k] = 0ull;
    int r0 = 0;
    for (; r0 + R <= rows; r0 += R)
      product_chunk_f2<G, R, PITCH, false>(Sa + r0 * PITCH, Sb + r0 * PITCH, R, acc2);
    if (r0 < rows)
      product_chunk_f2<G, R, PITCH, true>(Sa + r0 * PITCH, Sb + r0 * PITCH, rows - r0, acc2);
#pragma unroll
    for (int k = 0; k < G; ++k) acc[k] = upk2(acc2[k]);
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
    const int fc = (m < p.Q - 1) ? m : m - (p.M - 2 * p.Q + 2);
    C2 *cs = (C2 *)p.colsum_part;
#pragma unroll
    for (int k = 0; k < G; ++k)
      if (k < cnt) {
        const int D = combo_index(p.P, d0 + k, dc);
        cs[((long long)D * p.NFC + fc) * p.n_rb + rb] = acc[k];
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

template <typename T, int G, int R, int PITCH, int NCW>
__global__ void __launch_bounds__((NCW + 1) * 32, 1)
    k_products_inner(const RecParams p, const __grid_constant__ CUtensorMap tmap) {
  using C2 = typename C2t<T>::type;
  extern __shared__ __align__(1024) unsigned char smem_k1[];
  const size_t bb = tile_buf_bytes<T, PITCH>(p.STR);
  C2 *buf0 = (C2 *)smem_k1;
  C2 *buf1 = (C2 *)(smem_k1 + bb);
  uint64_t *full = (uint64_t *)(smem_k1 + 2 * bb);
  uint64_t *empty = full + 2;
  int *ctr = (int *)(empty + 2);  // next task index within the tile held by each buffer

  // the fringe-row kernel does not read this kernel's output: let it start
  // on SMs this kernel leaves free
  pdl_launch_dependents();
  const long long NT = p.n_tasks;
  const long long tb = NT * blockIdx.x / gridDim.x;
  const long long te = NT * (blockIdx.x + 1) / gridDim.x;
  if (tb >= te) return;
  const long long tpt = p.tasks_per_tile;
  const long long tf = tb / tpt, tl = (te - 1) / tpt;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(&full[0], p.use_tma ? 1 : 32);
    mbar_init(&full[1], p.use_tma ? 1 : 32);
    mbar_init(&empty[0], NCW);
    mbar_init(&empty[1], NCW);
    ctr[0] = 0;
    ctr[1] = 0;
    fence_mbar_init();
  }
  __syncthreads();

  // Every warp goes through the CTA's tiles in order and waits on each tile's
  // barrier phase in turn, so a parity wait never spans more than one phase.
  if (warp == NCW) {  // producer
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
      if (lane == 0) ctr[b] = 0;  // all warps are done with the buffer's previous tile
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
        stage_tile_cpasync<T, PITCH>(p, tile, dst, &full[b], lane);
      }
      issued = tile - tf;
    }
    if (!ok && lane == 0) *p.status = kDevTimeout;
    // Wait (bounded) for this warp's last copies before the CTA may exit.
    for (long long k = (issued >= 1 ? issued - 1 : 0); k <= issued; ++k)
      mbar_wait(&full[k & 1], (unsigned)((k >> 1) & 1), kWaitLimitNs);
    return;
  }

  // consumers: tasks of the current tile are handed out through ctr[b]
  for (long long tile = tf; tile <= tl; ++tile) {
    const int b = (int)((tile - tf) & 1);
    const long long n = (tile - tf) >> 1;
    if (!mbar_wait(&full[b], (unsigned)(n & 1), kWaitLimitNs)) {
      if (lane == 0) *p.status = kDevTimeout;
      return;
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
}

constexpr int kConsumerWarps = 16;

template <typename T, int G, int PITCH>
static cudaError_t launch_products_p(const RecParams &p, const CUtensorMap &tmap, int num_sms,
                                     cudaStream_t s) {
  auto kern = k_products_inner<T, G, 8, PITCH, kConsumerWarps>;
  const size_t smem = 2 * tile_buf_bytes<T, PITCH>(p.STR) + 64;
  cudaError_t e = ensure_smem_attr(kern, smem);
  if (e != cudaSuccess) return e;
  long long grid = num_sms;
  const long long need = (p.n_tasks + kConsumerWarps - 1) / kConsumerWarps;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  return launch_k(kern, dim3((unsigned)grid), dim3((kConsumerWarps + 1) * 32), smem, s, false, p,
                  tmap);
}

template <typename T, int G>
static cudaError_t launch_products(const RecParams &p, const CUtensorMap &tmap, int num_sms,
                                   cudaStream_t s) {
  if (p.PITCH == 80) return launch_products_p<T, G, 80>(p, tmap, num_sms, s);
  if (p.PITCH == 96) return launch_products_p<T, G, 96>(p, tmap, num_sms, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_products_any(const RecParams &p, const CUtensorMap &tmap, bool fp64, int num_sms,
                                cudaStream_t s) {
  switch (p.G) {
    case 4: return fp64 ? launch_products<double, 4>(p, tmap, num_sms, s)
                        : launch_products<float, 4>(p, tmap, num_sms, s);
    case 8: return fp64 ? launch_products<double, 8>(p, tmap, num_sms, s)
                        : launch_products<float, 8>(p, tmap, num_sms, s);
    case 16:
      if (fp64) return cudaErrorInvalidValue;  // FP64 uses at most 8 lags
      return launch_products<float, 16>(p, tmap, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace cov
