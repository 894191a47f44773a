// Covariance estimates of every aperture of one image (the image-processing
// use of Section 2.3: one estimate of Eq. 2.1-2.2 per overlapping aperture),
// computed strip by strip so that apertures side by side share their
// products.
//
// A CTA takes one row of apertures and G neighbours in it: the strip of the
// image under them (ap_n rows, (G-1) step_c + ap_m <= 64 columns) is staged
// in shared memory once. Column lag by column lag dc, the warps take groups
// of four row lags of one sign (dr = d0 .. d0+3, or -d0 .. -(d0+3)) of the
// combinations (dr, dc) of Eq. 3.3. For one group a warp
//  - forms the products of Eq. 3.5 over the whole strip, two columns a lane,
//    and walks their column sums down the diagonal: the sum over the box rows
//    of the first output row, then per output row one product row in and one
//    out (Eq. 3.7-3.8). The four lags share one operand row and slide along
//    the other: the seed, blocked by four rows, loads four rows of the shared
//    operand and seven of the sliding one for 16 products a column;
//  - after each output row, builds each aperture's outputs of that row as
//    sums of Wd consecutive column sums, slid along the output columns (one
//    column sum in, one out), one (aperture, lag) a lane, into a shared-
//    memory table of the lag's R blocks.
// The CTA then writes the R blocks of that column lag, (j, j + dc) and their
// conjugate mirrors (j + dc, j), in runs of P contiguous elements. A strip's
// column lags are split into contiguous ranges of about equal work, one CTA
// each (the ranges write disjoint blocks), so that the launch's last wave is
// short.
//
// Against one CTA per aperture (the batched box form), a product under k
// apertures of the strip is formed once instead of k times, every lane holds
// columns of the strip instead of the 32 - ap_m idle ones, and each output
// costs two additions instead of a doubling scan across the lanes.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/cov.h"
#include "cov_device.cuh"
#include "smem_attr.h"

namespace cov {
namespace {

constexpr int kApWarps = 4;
constexpr int kApThreads = kApWarps * 32;
constexpr int kApLag = 4;      // row lags a warp takes together
constexpr int kApBlk = 4;      // seed rows a step (register block)
constexpr int kApStrip = 64;   // strip columns staged by a CTA (two a lane)
constexpr int kApVPitch = 65;  // row pitch of a warp's column sums, in float2
constexpr int kApMaxPQ = 16;   // P, Q limit
constexpr int kApMaxRows = 64; // ap_n limit

struct ApParams {
  const float2 *img;
  long long ld;
  float2 *R;
  int nc;              // apertures in a row of apertures
  int groups;          // CTAs per row of apertures
  int an, am, sr, sc;  // aperture rows, columns; steps
  int P, Q, G;         // window; apertures a CTA takes
  int TS;              // table entries per aperture (Q P^2)
  float rK;            // 1/K (COV_MEAN, the FP32 reciprocal) or 1 (COV_SUM)
  int nsplit;          // CTAs a strip: column-lag ranges [dcb[i], dcb[i + 1])
  int dcb[kApMaxPQ + 1];
};

// The lag's output table of one aperture holds its R blocks (j, j + dc),
// j < Q - dc, entry (i, i') at j P^2 + i P + i' (dc = 0: the entries i <= i').
inline int ap_table_entries(int P, int Q) { return Q * P * P; }
// The strip with kApLag zero rows below it (read by the lags past the last
// one of a group), the warps' column sums, the lag's output table.
inline size_t ap_smem_bytes(int an, int P, int Q, int G) {
  return ((size_t)(an + kApLag) * kApStrip + (size_t)kApWarps * kApLag * kApVPitch +
          (size_t)G * ap_table_entries(P, Q)) * sizeof(float2);
}

// n / d for 0 <= n < 2^16 and 1 <= d <= 256 by a multiply-high with
// m = ceil(2^32 / d): n m / 2^32 = n / d + n (m d - 2^32) / (d 2^32), and the
// second term stays below 1 / d while n (m d - 2^32) < 2^32, i.e. n < 2^24.
struct DivSmall {
  unsigned m;
  int d;
  __device__ __forceinline__ void init(int dd) {
    d = dd;
    m = dd == 1 ? 0u : 0xffffffffu / (unsigned)dd + 1u;
  }
  __device__ __forceinline__ int q(int n) const {
    return d == 1 ? n : (int)__umulhi((unsigned)n, m);
  }
};

// acc += a conj(b) with a, b the two operands in their roles: for dr >= 0 the
// shared operand is a (row r, column x) and the sliding one b (row r + dr,
// column x + dc); for dr < 0 the shared one is b (row r) and the sliding one
// a (row r + |dr|).
template <bool NEG>
__device__ __forceinline__ void ap_mac(float2 &acc, float2 shared_op, float2 sliding_op) {
  if (NEG)
    cmac_conj(acc, sliding_op, shared_op);
  else
    cmac_conj(acc, shared_op, sliding_op);
}
// acc -= a conj(b), the operands in the roles of ap_mac.
__device__ __forceinline__ void cmsub_conj(float2 &acc, float2 a, float2 b) {
  acc.x = __fmaf_rn(-a.x, b.x, acc.x);
  acc.x = __fmaf_rn(-a.y, b.y, acc.x);
  acc.y = __fmaf_rn(-a.y, b.x, acc.y);
  acc.y = __fmaf_rn(a.x, b.y, acc.y);
}
template <bool NEG>
__device__ __forceinline__ void ap_msub(float2 &acc, float2 shared_op, float2 sliding_op) {
  if (NEG)
    cmsub_conj(acc, sliding_op, shared_op);
  else
    cmsub_conj(acc, shared_op, sliding_op);
}
// Packed FP32x2 add and subtract (each half rounded as add.rn.f32 / sub.rn.f32).
__device__ __forceinline__ unsigned long long ap_add2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long ap_sub2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// Outputs of output row s for the warp's lags: lane (aperture ap, lag k)
// sums its aperture's Wd column sums and slides along the J output columns.
template <bool NEG>
__device__ __forceinline__ void ap_row_pass(const ApParams &p, const float2 *Vw, float2 *T,
                                            int lane, int s, int d0, int Gc, int Wd, int J) {
  const int P = p.P, PP = P * P;
  for (int q = lane; q < Gc * kApLag; q += 32) {
    const int ap = q / kApLag, k = q - ap * kApLag, dd = d0 + k;  // |dr|
    if (dd >= P || s >= P - dd) continue;  // a lag past P - 1, or no output row s
    const unsigned long long *v = (const unsigned long long *)(Vw + k * kApVPitch + ap * p.sc);
    unsigned long long W = v[0], W2 = 0ull;
    int m = 1;
    for (; m + 1 < Wd; m += 2) {
      W = ap_add2(W, v[m]);
      W2 = ap_add2(W2, v[m + 1]);
    }
    if (m < Wd) W = ap_add2(W, v[m]);
    W = ap_add2(W, W2);
    // output (s, j) of lag dr is entry (i0 + s, i0 + s + dr) of block j
    const int i = NEG ? dd + s : s, ip = NEG ? s : s + dd;
    unsigned long long *t = (unsigned long long *)(T + ap * p.TS + i * P + ip);
    t[0] = W;
    for (int j = 1; j < J; ++j) {  // column j - 1 leaves the window, j - 1 + Wd enters
      W = ap_add2(W, ap_sub2(v[j - 1 + Wd], v[j - 1]));
      t[j * PP] = W;
    }
  }
}

// One group of row lags (|dr| = d0 .. d0 + kApLag - 1, sign by NEG) of
// column lag dc over the strip.
template <bool NEG>
__device__ __forceinline__ void ap_group(const ApParams &p, const float2 *As, float2 *Vw,
                                         float2 *T, int lane, int dc, int d0, int Gc, int ncol) {
  const int P = p.P, Hb = p.an - P + 1, Wd = p.am - p.Q + 1, J = p.Q - dc;
  const int Imax = P - d0;  // output rows of the group's first lag
  const int o1 = lane + 32 < ncol ? 32 : 0;  // the lane's second column (or its first again)
  const float2 *S0 = As + lane + (NEG ? dc : 0), *S1 = S0 + o1;  // shared operand, row r
  const float2 *L0 = As + d0 * kApStrip + lane + (NEG ? 0 : dc), *L1 = L0 + o1;  // row r + d0 (+ k)
  float2 V0[kApLag], V1[kApLag];
#pragma unroll
  for (int k = 0; k < kApLag; ++k) V0[k] = V1[k] = make_float2(0.f, 0.f);
  // seed: box rows 0 .. Hb-1 of output row 0, kApBlk rows a step
  int r = 0;
  for (; r + kApBlk <= Hb; r += kApBlk) {
    float2 s0[kApBlk], s1[kApBlk], l0[kApBlk + kApLag - 1], l1[kApBlk + kApLag - 1];
#pragma unroll
    for (int t = 0; t < kApBlk; ++t) {
      s0[t] = S0[(r + t) * kApStrip];
      s1[t] = S1[(r + t) * kApStrip];
    }
#pragma unroll
    for (int t = 0; t < kApBlk + kApLag - 1; ++t) {
      l0[t] = L0[(r + t) * kApStrip];
      l1[t] = L1[(r + t) * kApStrip];
    }
#pragma unroll
    for (int t = 0; t < kApBlk; ++t)
#pragma unroll
      for (int k = 0; k < kApLag; ++k) {
        ap_mac<NEG>(V0[k], s0[t], l0[t + k]);
        ap_mac<NEG>(V1[k], s1[t], l1[t + k]);
      }
  }
  for (; r < Hb; ++r) {
    const float2 s0 = S0[r * kApStrip], s1 = S1[r * kApStrip];
#pragma unroll
    for (int k = 0; k < kApLag; ++k) {
      ap_mac<NEG>(V0[k], s0, L0[(r + k) * kApStrip]);
      ap_mac<NEG>(V1[k], s1, L1[(r + k) * kApStrip]);
    }
  }
  for (int s = 0;; ++s) {
#pragma unroll
    for (int k = 0; k < kApLag; ++k) {
      Vw[k * kApVPitch + lane] = V0[k];
      Vw[k * kApVPitch + lane + 32] = V1[k];
    }
    __syncwarp();
    ap_row_pass<NEG>(p, Vw, T, lane, s, d0, Gc, Wd, J);
    __syncwarp();  // the column sums are read before the next row overwrites them
    if (s + 1 >= Imax) break;
    // walk: row s leaves the box, row s + Hb enters
    const int ri = s + Hb, ro = s;
    const float2 si0 = S0[ri * kApStrip], si1 = S1[ri * kApStrip];
    const float2 so0 = S0[ro * kApStrip], so1 = S1[ro * kApStrip];
#pragma unroll
    for (int k = 0; k < kApLag; ++k) {  // the entering product added, the leaving one subtracted
      ap_msub<NEG>(V0[k], so0, L0[(ro + k) * kApStrip]);
      ap_msub<NEG>(V1[k], so1, L1[(ro + k) * kApStrip]);
      ap_mac<NEG>(V0[k], si0, L0[(ri + k) * kApStrip]);
      ap_mac<NEG>(V1[k], si1, L1[(ri + k) * kApStrip]);
    }
  }
}

__global__ void __launch_bounds__(kApThreads, 4) k_apertures(ApParams p) {
  extern __shared__ __align__(16) unsigned char smem_ap[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int P = p.P, Q = p.Q, DD = P * Q, PP = P * P;
  const int strip = blockIdx.x / p.nsplit, part = blockIdx.x - strip * p.nsplit;
  const int ay = strip / p.groups, g = strip - ay * p.groups;
  const int ax0 = g * p.G, Gc = min(p.G, p.nc - ax0);
  const int Sw = (Gc - 1) * p.sc + p.am;  // strip columns under the CTA's apertures
  const int rows = p.an + kApLag;
  float2 *As = (float2 *)smem_ap;                                // [an + kApLag][64]
  float2 *Vw = As + rows * kApStrip + warp * kApLag * kApVPitch;  // this warp's [kApLag][65]
  float2 *T = As + rows * kApStrip + kApWarps * kApLag * kApVPitch;  // [G][TS]
  const float2 *src = p.img + (long long)ay * p.sr * p.ld + (long long)ax0 * p.sc;
  for (int e = tid; e < rows * kApStrip; e += kApThreads) {
    const int r = e >> 6, c = e & (kApStrip - 1);
    As[e] = (c < Sw && r < p.an) ? __ldg(src + (long long)r * p.ld + c) : make_float2(0.f, 0.f);
  }
  __syncthreads();

  float2 *Rg = p.R + ((long long)ay * p.nc + ax0) * DD * DD;
  DivSmall divP;
  divP.init(P);
  const int npos = (P + kApLag - 1) / kApLag, nneg = (P - 1 + kApLag - 1) / kApLag;
  for (int dc = p.dcb[part]; dc < p.dcb[part + 1]; ++dc) {
    const int J = Q - dc, ncol = Sw - dc;  // output columns; strip columns with a partner
    // groups in decreasing output rows: dr >= 0 from d0 = 0 and, for dc > 0,
    // dr < 0 from d0 = 1, alternately; dealt to the warps in a snake
    const int nu = dc ? npos + nneg : npos;
    for (int u = 0; u < nu; ++u) {
      const int rnd = u / kApWarps, pos = u - rnd * kApWarps;
      if ((rnd & 1 ? kApWarps - 1 - pos : pos) != warp) continue;
      if (dc && (u & 1))
        ap_group<true>(p, As, Vw, T, lane, dc, 1 + (u >> 1) * kApLag, Gc, ncol);
      else
        ap_group<false>(p, As, Vw, T, lane, dc, (dc ? u >> 1 : u) * kApLag, Gc, ncol);
    }
    __syncthreads();
    // ---- R blocks of this lag: (j, j + dc), and for dc > 0 the mirrors
    // (j + dc, j); a thread the entries w = tid, tid + 128, ... of every block
    const float rK = p.rK;
    for (int w = tid; w < PP; w += kApThreads) {
      const int row = divP.q(w), col = w - row * P;
      const int tw = row > col && dc == 0 ? col * P + row : w;  // dc = 0: mirror of the upper entry
      const float im_sign = dc == 0 && row > col ? -rK : rK;
      const int tlo = col * P + row;
      for (int ap = 0; ap < Gc; ++ap) {
        const float2 *Tj = T + ap * p.TS;
        float2 *Rd = Rg + (long long)ap * DD * DD + (long long)row * DD + col + P * dc;  // block (0, dc)
        float2 *Rm = Rg + (long long)ap * DD * DD + (long long)(row + P * dc) * DD + col;  // block (dc, 0)
        const long long step = (long long)P * DD + P;  // to block (j + 1, j + 1 + dc)
        for (int j = 0; j < J; ++j, Tj += PP, Rd += step, Rm += step) {
          float2 v = Tj[tw];
          v.x *= rK;
          v.y = dc == 0 && row == col ? 0.f : v.y * im_sign;
          __stcs(Rd, v);  // R is written once and not read back: evict first
          if (dc) {  // block (j + dc, j): entry (row, col) is the conjugate of (col, row)
            float2 u = Tj[tlo];
            u.x *= rK;
            u.y = -u.y * rK;
            __stcs(Rm, u);
          }
        }
      }
    }
    __syncthreads();  // the table is read before the next lag overwrites it
  }
}

// Splits the column lags 0 .. Q-1 of each strip into p.nsplit contiguous
// ranges of about equal work, one CTA each, so that the launch has some
// sixteen CTAs per resident slot and its last wave is short. Work of lag dc,
// in warp instructions: the products of the groups' seeds and walks (four
// FMA each), the output rows' window sums, the R elements written.
void ap_split_lags(ApParams &p, int an, int am, int P, int Q, int G, long long strips, size_t smem) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 152;
  }
  const long long per_sm = std::max<long long>(1, std::min<long long>(4, (228 << 10) / (smem + 1024)));
  const long long slots = sms * per_sm;
  int n = 1;
  while (n < Q && strips * n < 16 * slots) ++n;
  const int Hb = an - P + 1, Wd = am - Q + 1;
  double cost[kApMaxPQ];
  for (int dc = 0; dc < Q; ++dc) {
    const int J = Q - dc;
    double c = 0;
    for (int neg = 0; neg < (dc ? 2 : 1); ++neg)
      for (int d0 = neg; d0 < P; d0 += kApLag) {
        const int Imax = P - d0;
        c += 8.0 * kApLag * (Hb + 2.0 * (Imax - 1)) + 2.0 * Imax * (Wd + 3.0 * J);
      }
    c += (double)G * J * P * P * (dc ? 2 : 1) * 6.0 / 32.0;
    cost[dc] = c;
  }
  // contiguous ranges with the smallest largest share: best[i][k] = the
  // smallest largest range cost of lags 0 .. i-1 in k ranges
  double best[kApMaxPQ + 1][kApMaxPQ + 1];
  int cut[kApMaxPQ + 1][kApMaxPQ + 1];
  for (int i = 0; i <= Q; ++i)
    for (int k = 0; k <= n; ++k) best[i][k] = 1e300, cut[i][k] = 0;
  best[0][0] = 0;
  for (int k = 1; k <= n; ++k)
    for (int i = k; i <= Q; ++i) {
      double tail = 0;
      for (int j = i - 1; j >= k - 1; --j) {  // range [j, i)
        tail += cost[j];
        const double v = std::max(best[j][k - 1], tail);
        if (v < best[i][k]) best[i][k] = v, cut[i][k] = j;
      }
    }
  p.nsplit = n;
  for (int k = n, i = Q; k > 0; --k) {
    p.dcb[k] = i;
    i = cut[i][k];
  }
  p.dcb[0] = 0;
}

}  // namespace
}  // namespace cov

extern "C" cov_status cov_estimate_apertures(const void *image, cov_dtype dtype, int64_t H,
                                             int64_t W, int64_t ld, int ap_n, int ap_m,
                                             int step_r, int step_c, int P, int Q, void *R,
                                             cov_norm norm, cov_stream_t stream) {
  using namespace cov;
  if (!image || !R || H < 1 || W < 1 || ld < W || ap_n < 1 || ap_m < 1 || ap_n > H ||
      ap_m > W || step_r < 1 || step_c < 1 || P < 1 || Q < 1 || P > ap_n || Q > ap_m ||
      (dtype != COV_C64 && dtype != COV_C128) || (norm != COV_MEAN && norm != COV_SUM))
    return COV_EINVAL;
  const long long nr = (H - ap_n) / step_r + 1, nc = (W - ap_m) / step_c + 1;
  if (nr * nc > (1LL << 30)) return COV_EINVAL;
  if (((uintptr_t)image & 7) || ((uintptr_t)R & 7)) return COV_EINVAL;
  if (dtype != COV_C64 || P > kApMaxPQ || Q > kApMaxPQ || ap_n > kApMaxRows || ap_m > kApStrip)
    return COV_EUNSUPPORTED;
  int dev = 0, smem_max = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
          cudaSuccess) {
    cudaGetLastError();
    return COV_ECUDA;
  }
  int G = (int)std::min<long long>(nc, 1 + (kApStrip - ap_m) / step_c);
  while (G > 1 && ap_smem_bytes(ap_n, P, Q, G) > (size_t)smem_max) --G;
  const size_t smem = ap_smem_bytes(ap_n, P, Q, G);
  if (smem > (size_t)smem_max) return COV_EUNSUPPORTED;
  if (ensure_dyn_smem((const void *)k_apertures, smem, true) != cudaSuccess) {
    cudaGetLastError();
    return COV_ECUDA;
  }
  ApParams p;
  ap_split_lags(p, ap_n, ap_m, P, Q, G, nr * ((nc + G - 1) / G), smem);
  p.img = (const float2 *)image;
  p.ld = ld;
  p.R = (float2 *)R;
  p.nc = (int)nc;
  p.groups = (int)((nc + G - 1) / G);
  p.an = ap_n;
  p.am = ap_m;
  p.sr = step_r;
  p.sc = step_c;
  p.P = P;
  p.Q = Q;
  p.G = G;
  p.TS = ap_table_entries(P, Q);
  const long long K = (long long)(ap_n - P + 1) * (ap_m - Q + 1);
  p.rK = norm == COV_MEAN ? 1.0f / (float)K : 1.0f;
  const long long grid = nr * p.groups * p.nsplit;
  if (grid > 0x7fffffffLL) return COV_EUNSUPPORTED;
  k_apertures<<<(unsigned)grid, kApThreads, smem, (cudaStream_t)stream>>>(p);
  return cudaGetLastError() == cudaSuccess ? COV_OK : COV_ECUDA;
}
