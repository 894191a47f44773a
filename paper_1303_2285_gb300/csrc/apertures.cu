// Covariance estimates of every aperture of one image (the image-processing
// use of Section 2.3: one estimate of Eq. 2.1-2.2 per overlapping aperture),
// computed strip by strip so that apertures side by side share their
// products.
//
// A CTA takes one row of apertures and G neighbours in it: the strip of the
// image under them (ap_n rows, (G-1) step_c + ap_m <= 64 columns) is staged
// in shared memory once. Column lag by column lag dc, the warps take the row
// lags dr of the combinations (dr, dc) of Eq. 3.3; for one combination a warp
//  - forms the products of Eq. 3.5 over the whole strip, two columns a lane,
//    and walks their column sums down the diagonal: the sum over the box rows
//    of the first output row, then per output row one product row in and one
//    out (Eq. 3.7-3.8);
//  - builds each aperture's outputs as sums of Wd consecutive column sums,
//    slid along the output columns (one column sum in, one out), into a
//    shared-memory table of the lag's outputs.
// The CTA then writes the R blocks of that lag, (j, j + dc) and their
// conjugate mirrors (j + dc, j), in runs of P contiguous elements.
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

constexpr int kApWarps = 8;
constexpr int kApStrip = 64;   // strip columns staged by a CTA (two a lane)
constexpr int kApVPitch = 65;  // row pitch of a warp's column sums, in float2 (spreads the banks)
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
};

// The lag's output table of one aperture holds its R blocks (j, j + dc),
// j < Q - dc, entry (i, i') at j P^2 + i P + i' (dc = 0: the entries i <= i').
inline int ap_table_entries(int P, int Q) { return Q * P * P; }
// Strip, the warps' column sums and the lag's output table.
inline size_t ap_smem_bytes(int an, int P, int Q, int G) {
  return ((size_t)an * kApStrip + (size_t)kApWarps * P * kApVPitch +
          (size_t)G * ap_table_entries(P, Q)) * sizeof(float2);
}

__device__ __forceinline__ float2 ap_prod(float2 a, float2 b) {
  float2 v = make_float2(0.f, 0.f);
  cmac_conj(v, a, b);
  return v;
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

__global__ void __launch_bounds__(kApWarps * 32, 2) k_apertures(ApParams p) {
  extern __shared__ __align__(16) unsigned char smem_ap[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int P = p.P, Q = p.Q, DD = P * Q, PP = P * P;
  const int Hb = p.an - P + 1, Wd = p.am - Q + 1;  // box rows, box columns
  const int ay = blockIdx.x / p.groups, g = blockIdx.x - ay * p.groups;
  const int ax0 = g * p.G, Gc = min(p.G, p.nc - ax0);
  const int Sw = (Gc - 1) * p.sc + p.am;  // strip columns under the CTA's apertures
  float2 *As = (float2 *)smem_ap;                                 // [an][64]
  float2 *Vw = As + p.an * kApStrip + warp * P * kApVPitch;       // this warp's [P][65]
  float2 *T = As + p.an * kApStrip + kApWarps * P * kApVPitch;    // [G][TS]
  const float2 *src = p.img + (long long)ay * p.sr * p.ld + (long long)ax0 * p.sc;
  for (int e = tid; e < p.an * kApStrip; e += kApWarps * 32) {
    const int r = e >> 6, c = e & (kApStrip - 1);
    As[e] = c < Sw ? __ldg(src + (long long)r * p.ld + c) : make_float2(0.f, 0.f);
  }
  __syncthreads();

  float2 *Rg = p.R + ((long long)ay * p.nc + ax0) * DD * DD;
  for (int dc = 0; dc < Q; ++dc) {
    const int J = Q - dc, ncol = Sw - dc;  // output columns; strip columns with a partner
    const int nd = dc ? 2 * P - 1 : P;
    // row lags in decreasing output rows (0, 1, -1, 2, -2, ...), warps in turn
    for (int k = warp; k < nd; k += kApWarps) {
      const int d = dc ? ((k & 1) ? (k + 1) >> 1 : -(k >> 1)) : k;
      const int I = P - (d < 0 ? -d : d), i0 = d < 0 ? -d : 0;
      // ---- column sums of the products, walked down the diagonal --------
      // The products of rows r < I - 1 leave the box at output row r + 1:
      // they are kept in row r + 1 of the warp's column-sum buffer, which
      // that output row overwrites after reading them.
      const int o1 = lane + 32 < ncol ? 32 : 0;  // the lane's second column (or its first again)
      const float2 *pa = As + i0 * kApStrip + lane;
      const float2 *pb = As + (i0 + d) * kApStrip + lane + dc;
      float2 *vw = Vw + lane;
      float2 V0 = make_float2(0.f, 0.f), V1 = V0, U0 = V0, U1 = V0;
      const int nk = min(I - 1, Hb);  // kept rows among the seed's
      int r = 0;
      for (; r < nk; ++r) {
        const int o = r * kApStrip;
        const float2 x0 = ap_prod(pa[o], pb[o]), x1 = ap_prod(pa[o + o1], pb[o + o1]);
        vw[(r + 1) * kApVPitch] = x0;
        vw[(r + 1) * kApVPitch + 32] = x1;
        V0.x += x0.x;
        V0.y += x0.y;
        V1.x += x1.x;
        V1.y += x1.y;
      }
      for (; r + 1 < Hb; r += 2) {
        const int o = r * kApStrip;
        cmac_conj(V0, pa[o], pb[o]);
        cmac_conj(V1, pa[o + o1], pb[o + o1]);
        cmac_conj(U0, pa[o + kApStrip], pb[o + kApStrip]);
        cmac_conj(U1, pa[o + kApStrip + o1], pb[o + kApStrip + o1]);
      }
      if (r < Hb) {
        const int o = r * kApStrip;
        cmac_conj(V0, pa[o], pb[o]);
        cmac_conj(V1, pa[o + o1], pb[o + o1]);
      }
      V0.x += U0.x;
      V0.y += U0.y;
      V1.x += U1.x;
      V1.y += U1.y;
      vw[0] = V0;
      vw[32] = V1;
      for (int s = 1; s < I; ++s) {  // row s - 1 leaves the box, row s - 1 + Hb enters
        const int rin = s - 1 + Hb, oi = rin * kApStrip;
        const float2 x0 = ap_prod(pa[oi], pb[oi]), x1 = ap_prod(pa[oi + o1], pb[oi + o1]);
        if (rin < I - 1) {  // a box shorter than the walk: the entering row leaves later
          vw[(rin + 1) * kApVPitch] = x0;
          vw[(rin + 1) * kApVPitch + 32] = x1;
        }
        const float2 y0 = vw[s * kApVPitch], y1 = vw[s * kApVPitch + 32];
        V0.x += x0.x - y0.x;
        V0.y += x0.y - y0.y;
        V1.x += x1.x - y1.x;
        V1.y += x1.y - y1.y;
        vw[s * kApVPitch] = V0;
        vw[s * kApVPitch + 32] = V1;
      }
      __syncwarp();
      // ---- window sums along the columns, one (aperture, output row) a
      // lane; output (s, j) is entry (i0 + s, i0 + s + d) of block j
      for (int q = lane; q < Gc * I; q += 32) {
        const int ap = q / I, s = q - ap * I;
        const unsigned long long *v =
            (const unsigned long long *)(Vw + s * kApVPitch + ap * p.sc);
        unsigned long long W = v[0], W2 = 0ull;
        int m = 1;
        for (; m + 1 < Wd; m += 2) {
          W = ap_add2(W, v[m]);
          W2 = ap_add2(W2, v[m + 1]);
        }
        if (m < Wd) W = ap_add2(W, v[m]);
        W = ap_add2(W, W2);
        unsigned long long *t =
            (unsigned long long *)(T + ap * p.TS + (i0 + s) * P + i0 + s + d);
        t[0] = W;
        for (int j = 1; j < J; ++j) {  // column j - 1 leaves the window, j - 1 + Wd enters
          W = ap_add2(W, ap_sub2(v[j - 1 + Wd], v[j - 1]));
          t[j * PP] = W;
        }
      }
      __syncwarp();  // the column sums are read before the next row lag overwrites them
    }
    __syncthreads();
    // ---- R blocks of this lag: (j, j + dc), and for dc > 0 the mirrors
    // (j + dc, j). The two thread halves take alternate j, a thread the
    // entries w, w + 128, ... of each block.
    const int half = tid >> 7;
    for (int w = tid & 127; w < PP; w += 128) {
      const int row = w / P, col = w - row * P;
      const int up = row * P + col, lo = col * P + row;  // entry (row, col) and its transpose
      const bool below = row > col;
      const float rK = p.rK;
      for (int ap = 0; ap < Gc; ++ap) {
        const float2 *Ta = T + ap * p.TS;
        float2 *Ra = Rg + (long long)ap * DD * DD + (long long)row * DD + col;
        for (int j = half; j < J; j += 2) {
          const float2 *Tj = Ta + j * PP;
          if (dc == 0) {  // a diagonal block: entries below the diagonal mirror those above
            float2 v = Tj[below ? lo : up];
            v.x *= rK;
            v.y = row == col ? 0.f : (below ? -v.y : v.y) * rK;
            Ra[(long long)P * j * DD + P * j] = v;
          } else {
            float2 v = Tj[up];
            v.x *= rK;
            v.y *= rK;
            Ra[(long long)P * j * DD + P * (j + dc)] = v;
            v = Tj[lo];  // block (j + dc, j): entry (row, col) is the conjugate of (col, row)
            v.x *= rK;
            v.y = -v.y * rK;
            Ra[(long long)P * (j + dc) * DD + P * j] = v;
          }
        }
      }
    }
    __syncthreads();  // the table is read before the next lag overwrites it
  }
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
  const long long grid = nr * p.groups;
  k_apertures<<<(unsigned)grid, kApWarps * 32, smem, (cudaStream_t)stream>>>(p);
  return cudaGetLastError() == cudaSuccess ? COV_OK : COV_ECUDA;
}
