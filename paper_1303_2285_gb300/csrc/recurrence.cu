// The combination / diagonal-segment path (Sections 3.1-3.4, Algorithm 1),
// refined with the sliding-box recurrence: every distinct product of a
// unique combination is formed once, each combination's diagonal segments are
// seeded with a direct sum and walked along the diagonal, and one thread block
// writes each element of R. See cov_internal.h for the notation and the split
// of the work into the four kernels below.
#include <cuda_runtime.h>

#include "cov_device.cuh"
#include "cov_internal.h"
#include "cov_launch.h"

namespace cov {

// ---------------------------------------------------------------------------
// Kernel 1: products over inner rows x all columns, per (tile, 32 columns,
// lag group) warp task. The CTA's tile of A plus its halo is staged in shared
// memory with cp.async (zero fill outside A), double-buffered across tiles.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void stage_tile(const RecParams &p, long long tile, typename C2t<T>::type *S) {
  using C2 = typename C2t<T>::type;
  const int rt = (int)(tile / p.n_ct), ct = (int)(tile % p.n_ct);
  const long long r0 = (long long)p.inner_lo + (long long)rt * p.TR + p.d_lo;
  const int c0 = ct * p.TC;
  const C2 *A = (const C2 *)p.A;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int sr = warp; sr < p.STR; sr += nw) {
    const long long gr = r0 + sr;
    const bool rok = gr >= 0 && gr < p.N;
    const C2 *row = A + (rok ? gr : 0) * p.lda;
    C2 *dst = S + (long long)sr * p.STC;
    for (int sc = lane; sc < p.STC; sc += 32) {
      const int gc = c0 + sc;
      const bool ok = rok && gc < p.M;
      const C2 *src = ok ? row + gc : A;
      if (sizeof(C2) == 8)
        cp_async_8(dst + sc, src, ok);
      else
        cp_async_16(dst + sc, src, ok);
    }
  }
  cp_async_commit();
}

template <typename T, int G, int R>
__device__ __forceinline__ void product_task(const RecParams &p, long long tile, long long local,
                                             const typename C2t<T>::type *S, int lane) {
  using C2 = typename C2t<T>::type;
  const int rt = (int)(tile / p.n_ct), ct = (int)(tile % p.n_ct);
  const int g = (int)(local / p.CBT), cbl = (int)(local % p.CBT);
  const int cbg = ct * p.CBT + cbl;
  if (cbg >= p.n_cb) return;
  int dc, d0, cnt;
  group_of(p.P, G, g, dc, d0, cnt);
  const int n0 = p.inner_lo + rt * p.TR;
  const int rem = p.inner_lo + p.n_inner - n0;
  const int rows = rem < p.TR ? rem : p.TR;
  const int col_s = cbl * 32 + lane;
  const int STC = p.STC;

  C2 acc[G];
#pragma unroll
  for (int k = 0; k < G; ++k) acc[k] = czero<C2>();

  const C2 *Sa = S + (long long)(-p.d_lo) * STC + col_s;
  const C2 *Sb = S + (long long)(d0 - p.d_lo) * STC + col_s + dc;
  for (int r0 = 0; r0 < rows; r0 += R) {
    C2 a[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a[r] = (r0 + r < rows) ? Sa[(r0 + r) * STC] : czero<C2>();
    const C2 *sb = Sb + r0 * STC;
#pragma unroll
    for (int k = 0; k < R + G - 1; ++k) {
      const C2 b = sb[k * STC];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int gg = k - r;
        if (gg >= 0 && gg < G) cmac_conj(acc[gg], a[r], b);
      }
    }
  }

  // Epilogue: lanes on fringe columns keep their own column sums; lanes on
  // inner columns are summed over the warp into the core partial.
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
        cs[((long long)D * p.NFC + fc) * p.n_rt + rt] = acc[k];
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
      cp[2 * (((long long)D * p.n_rt + rt) * p.n_cb + cbg) + comp] = v[0];
    }
  }
}

template <typename T, int G, int R>
__global__ void __launch_bounds__(256, 1) k_products_inner(const RecParams p) {
  using C2 = typename C2t<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2 *buf0 = (C2 *)smem_raw;
  C2 *buf1 = buf0 + (size_t)p.STR * p.STC;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long long NT = p.n_tasks;
  const long long tb = NT * blockIdx.x / gridDim.x;
  const long long te = NT * (blockIdx.x + 1) / gridDim.x;
  if (tb >= te) return;
  const long long tpt = p.tasks_per_tile;
  const long long tf = tb / tpt, tl = (te - 1) / tpt;
  stage_tile<T>(p, tf, buf0);
  for (long long tile = tf; tile <= tl; ++tile) {
    const bool odd = ((tile - tf) & 1) != 0;
    C2 *cur = odd ? buf1 : buf0;
    C2 *nxt = odd ? buf0 : buf1;
    if (tile < tl) {
      stage_tile<T>(p, tile + 1, nxt);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const long long lo = tb > tile * tpt ? tb : tile * tpt;
    const long long hi = te < (tile + 1) * tpt ? te : (tile + 1) * tpt;
    for (long long t = lo + warp; t < hi; t += nw) product_task<T, G, R>(p, tile, t - tile * tpt, cur, lane);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Kernel 2: fringe rows. One warp per (side, block of RB fringe rows, lag
// group of GF lags); lanes stride over the inner columns, then the warp
// combines its per-lane sums and each lane (one row, one lag) adds its own
// fringe-column products as running prefix / suffix sums to form the box-row
// sums RV[D][j][fr] for every column offset j.
// ---------------------------------------------------------------------------
template <typename T, int GF, int RB>
__global__ void __launch_bounds__(128) k_fringe_rows(const RecParams p) {
  static_assert(GF * RB == 32, "one lane per (row, lag)");
  using C2 = typename C2t<T>::type;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long long ntask = 2LL * p.nrb * p.ngroups_f;
  if (gw >= ntask) return;
  const int g = (int)(gw % p.ngroups_f);
  const int rest = (int)(gw / p.ngroups_f);
  const int rb = rest % p.nrb, side = rest / p.nrb;
  int dc, d0, cnt;
  group_of(p.P, GF, g, dc, d0, cnt);
  const int fr0 = rb * RB;
  const int nrows = (p.P - 1 - fr0) < RB ? (p.P - 1 - fr0) : RB;
  const int nbase = side == 0 ? fr0 : (p.N - p.P + 1) + fr0;
  const C2 *A = (const C2 *)p.A;

  C2 acc[RB][GF];
#pragma unroll
  for (int r = 0; r < RB; ++r)
#pragma unroll
    for (int k = 0; k < GF; ++k) acc[r][k] = czero<C2>();

  for (int m = p.Q - 1 + lane; m <= p.M - p.Q; m += 32) {
    C2 a[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r)
      a[r] = (r < nrows) ? __ldg(A + (long long)(nbase + r) * p.lda + m) : czero<C2>();
#pragma unroll
    for (int k = 0; k < RB + GF - 1; ++k) {
      const int row = nbase + d0 + k;
      const C2 b = (row >= 0 && row < p.N) ? __ldg(A + (long long)row * p.lda + m + dc) : czero<C2>();
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int gg = k - r;
        if (gg >= 0 && gg < GF) cmac_conj(acc[r][gg], a[r], b);
      }
    }
  }
  T v[2 * RB * GF];
#pragma unroll
  for (int r = 0; r < RB; ++r)
#pragma unroll
    for (int k = 0; k < GF; ++k) {
      v[2 * (r * GF + k)] = acc[r][k].x;
      v[2 * (r * GF + k) + 1] = acc[r][k].y;
    }
  warp_transpose_reduce<2 * RB * GF>(v, lane);  // lane holds complex index `lane`

  const int r = lane / GF, k = lane % GF;
  if (r >= nrows || k >= cnt) return;
  C2 s_in;
  s_in.x = v[0];
  s_in.y = v[1];
  const int n = nbase + r, dr = d0 + k;
  const int D = combo_index(p.P, dr, dc);
  const int fr = side * (p.P - 1) + fr0 + r;
  const int J = p.Q - dc, W = p.M - p.Q + 1;
  C2 *RV = (C2 *)p.rowval + (long long)D * p.Q * p.NFR + fr;
  const long long ld = p.NFR;
  if (n + dr < 0 || n + dr >= p.N) {
    for (int j = 0; j < J; ++j) RV[j * ld] = czero<C2>();
    return;
  }
  const C2 *An = A + (long long)n * p.lda;
  const C2 *Ab = A + (long long)(n + dr) * p.lda + dc;
  // Left fringe columns m in [j, Q-2] lie in the box of column offset j.
  C2 s = czero<C2>();
  if (J == p.Q) RV[(p.Q - 1) * ld] = s_in;
  for (int mm = p.Q - 2; mm >= 0; --mm) {
    cmac_conj(s, __ldg(An + mm), __ldg(Ab + mm));
    if (mm < J) {
      C2 o;
      o.x = s_in.x + s.x;
      o.y = s_in.y + s.y;
      RV[mm * ld] = o;
    }
  }
  // Right fringe columns m in [W, W+j-1] lie in the box of column offset j.
  s = czero<C2>();
  for (int j = 0; j < J; ++j) {
    C2 o = RV[j * ld];
    o.x += s.x;
    o.y += s.y;
    RV[j * ld] = o;
    if (j + 1 < J) cmac_conj(s, __ldg(An + W + j), __ldg(Ab + W + j));
  }
}

// ---------------------------------------------------------------------------
// Kernel 3: per combination, the inner-row part of the box sum at every
// column offset j: CV[D][j] = core + fringe-column sums inside the box.
// One warp per combination; compensated sums over the partials.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) k_reduce_cols(const RecParams p) {
  using C2 = typename C2t<T>::type;
  __shared__ C2 cs_s[4][2 * kMaxPQ];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int D = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (D >= p.n_uc) return;
  int dr, dc;
  combo_of(p.P, D, dr, dc);
  Neu<T> cr, ci;
  const long long nparts = (long long)p.n_rt * p.n_cb;
  const C2 *cp = (const C2 *)p.core_part + (long long)D * nparts;
  for (long long k = lane; k < nparts; k += 32) {
    const C2 x = cp[k];
    cr.add(x.x);
    ci.add(x.y);
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const T s1 = __shfl_xor_sync(0xffffffffu, cr.s, o), c1 = __shfl_xor_sync(0xffffffffu, cr.c, o);
    const T s2 = __shfl_xor_sync(0xffffffffu, ci.s, o), c2 = __shfl_xor_sync(0xffffffffu, ci.c, o);
    cr.merge(s1, c1);
    ci.merge(s2, c2);
  }
  const C2 *csp = (const C2 *)p.colsum_part + (long long)D * p.NFC * p.n_rt;
  for (int fc = lane; fc < p.NFC; fc += 32) {
    Neu<T> sr, si;
    for (int rt = 0; rt < p.n_rt; ++rt) {
      const C2 x = csp[(long long)fc * p.n_rt + rt];
      sr.add(x.x);
      si.add(x.y);
    }
    C2 o;
    o.x = sr.value();
    o.y = si.value();
    cs_s[wib][fc] = o;
  }
  __syncwarp();
  const int J = p.Q - dc;
  C2 *cv = (C2 *)p.colval + (long long)D * p.Q;
  for (int j = lane; j < J; j += 32) {
    Neu<T> vr = cr, vi = ci;
    for (int mm = j; mm <= p.Q - 2; ++mm) {
      vr.add(cs_s[wib][mm].x);
      vi.add(cs_s[wib][mm].y);
    }
    for (int k = 0; k < j; ++k) {
      vr.add(cs_s[wib][p.Q - 1 + k].x);
      vi.add(cs_s[wib][p.Q - 1 + k].y);
    }
    C2 o;
    o.x = vr.value();
    o.y = vi.value();
    cv[j] = o;
  }
}

// ---------------------------------------------------------------------------
// Kernel 4: one CTA per P x P block (bj, bj+dc) of R, which the combinations
// (dr, dc) own entirely (Fig. 3). A thread takes one diagonal segment of one
// combination (L outputs at most): it seeds with the direct sum over the box,
// walks down the diagonal (subtract the leaving top fringe row, add the
// entering bottom fringe row), divides by K and stages the block in shared
// memory; the block and its conjugate mirror are then written row by row.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_walk_write(const RecParams p) {
  using C2 = typename C2t<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2 *B = (C2 *)smem_raw;
  int b = blockIdx.x, dc = 0;
  while (b >= p.Q - dc) {
    b -= p.Q - dc;
    ++dc;
  }
  const int bj = b;
  const int P = p.P, D2 = 2 * P - 1, PP = P + 1;
  const int nchunk = (P + p.L - 1) / p.L;
  const C2 *rowval = (const C2 *)p.rowval;
  const C2 *colval = (const C2 *)p.colval;
  for (int t = threadIdx.x; t < D2 * nchunk; t += blockDim.x) {
    const int dr = t % D2 - (P - 1), c = t / D2;
    if (dc == 0 && dr < 0) continue;
    const int adr = dr < 0 ? -dr : dr;
    const int I = P - adr, i0 = dr < 0 ? -dr : 0;
    const int is = i0 + c * p.L;
    if (is >= i0 + I) continue;
    const int ie = (i0 + I) < (is + p.L) ? (i0 + I) : (is + p.L);
    const int Dx = combo_index(P, dr, dc);
    const C2 *RV = rowval + ((long long)Dx * p.Q + bj) * p.NFR;
    const C2 cv = colval[(long long)Dx * p.Q + bj];
    // seed: the direct sum over the box of output (is, bj)
    Neu<T> orr, oii;
    orr.add(cv.x);
    oii.add(cv.y);
    for (int n = is; n <= P - 2; ++n) {
      orr.add(RV[n].x);
      oii.add(RV[n].y);
    }
    for (int k = 0; k < is; ++k) {
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

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
template <typename T, int G>
static cudaError_t launch_products(const RecParams &p, int num_sms, cudaStream_t s) {
  auto kern = k_products_inner<T, G, 8>;
  const size_t smem = 2 * (size_t)p.STR * p.STC * sizeof(typename C2t<T>::type);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)num_sms * occ;
  const long long need = (p.n_tasks + 7) / 8;  // at least one task per warp
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, 256, smem, s>>>(p);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_rec(const RecParams &p, int num_sms, cudaStream_t s,
                             const StageEvents *ev) {
  cudaError_t e = cudaSuccess;
  auto mark = [&](int k) -> cudaError_t {
    return (ev && ev->on) ? cudaEventRecord(ev->ev[k], s) : cudaSuccess;
  };
  if ((e = mark(0)) != cudaSuccess) return e;
  if (p.n_inner > 0 && p.n_tasks > 0) {
    switch (p.G) {
      case 4: e = launch_products<T, 4>(p, num_sms, s); break;
      case 8: e = launch_products<T, 8>(p, num_sms, s); break;
      case 16: e = launch_products<T, 16>(p, num_sms, s); break;
      default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  }
  if ((e = mark(1)) != cudaSuccess) return e;
  if (p.NFR > 0) {
    const long long warps = 2LL * p.nrb * p.ngroups_f;
    const long long blocks = (warps + 3) / 4;
    k_fringe_rows<T, 8, 4><<<(unsigned)blocks, 128, 0, s>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if ((e = mark(2)) != cudaSuccess) return e;
  {
    const long long blocks = ((long long)p.n_uc + 3) / 4;
    k_reduce_cols<T><<<(unsigned)blocks, 128, 0, s>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if ((e = mark(3)) != cudaSuccess) return e;
  {
    const int nblk = p.Q * (p.Q + 1) / 2;
    const int nthr_need = (2 * p.P - 1) * ((p.P + p.L - 1) / p.L);
    int nthr = ((nthr_need + 31) / 32) * 32;
    if (nthr > 256) nthr = 256;
    const size_t smem = (size_t)p.P * (p.P + 1) * sizeof(typename C2t<T>::type);
    auto kern = k_walk_write<T>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<nblk, nthr, smem, s>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return mark(4);
}

cudaError_t launch_recurrence(const RecParams &p, bool fp64, int num_sms, cudaStream_t s,
                              const StageEvents *ev) {
  return fp64 ? launch_rec<double>(p, num_sms, s, ev) : launch_rec<float>(p, num_sms, s, ev);
}

}  // namespace cov
