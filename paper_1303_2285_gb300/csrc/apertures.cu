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
  int TS;              // table entries per aperture (the largest lag's outputs)
  float rK;            // 1/K (COV_MEAN, the FP32 reciprocal) or 1 (COV_SUM)
};

// Outputs of one column lag for one aperture: dc = 0 has the row lags
// 0 .. P-1 with P - dr output rows each, Q output columns; dc > 0 the row lags
// -(P-1) .. P-1 (P^2 output rows), Q - dc output columns.
inline int ap_table_entries(int P, int Q) {
  const int z = P * (P + 1) / 2 * Q, o = Q > 1 ? P * P * (Q - 1) : 0;
  return z > o ? z : o;
}
// Strip, the warps' column sums, the lag's output table, two offset tables.
inline size_t ap_smem_bytes(int an, int P, int Q, int G) {
  return ((size_t)an * kApStrip + (size_t)kApWarps * P * kApVPitch +
          (size_t)G * ap_table_entries(P, Q)) * sizeof(float2) +
         3 * kApMaxPQ * sizeof(int);
}

// n / d for 0 <= n < 2^20 and 1 <= d <= 64 by a multiply-high with
// m = ceil(2^32 / d): n m / 2^32 = n / d + n (m d - 2^32) / (d 2^32), and the
// second term stays below 1 / d while n (m d - 2^32) < 2^32, i.e. n < 2^26.
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

__device__ __forceinline__ float2 ap_prod(float2 a, float2 b) {
  float2 v = make_float2(0.f, 0.f);
  cmac_conj(v, a, b);
  return v;
}

__global__ void __launch_bounds__(kApWarps * 32, 2) k_apertures(ApParams p) {
  extern __shared__ __align__(16) unsigned char smem_ap[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int P = p.P, Q = p.Q, DD = P * Q;
  const int Hb = p.an - P + 1, Wd = p.am - Q + 1;  // box rows, box columns
  const int ay = blockIdx.x / p.groups, g = blockIdx.x - ay * p.groups;
  const int ax0 = g * p.G, Gc = min(p.G, p.nc - ax0);
  const int Sw = (Gc - 1) * p.sc + p.am;  // strip columns under the CTA's apertures
  float2 *As = (float2 *)smem_ap;                                    // [an][64]
  float2 *Vw = As + p.an * kApStrip + warp * P * kApVPitch;          // this warp's [P][65]
  float2 *T = As + p.an * kApStrip + kApWarps * P * kApVPitch;       // [G][TS]
  int *cumN = (int *)(T + p.G * p.TS);  // dc > 0: output rows of the row lags before dr (+ P - 1)
  int *cum0 = cumN + 2 * kApMaxPQ;      // dc = 0: the same for dr >= 0
  const float2 *src = p.img + (long long)ay * p.sr * p.ld + (long long)ax0 * p.sc;
  for (int e = tid; e < p.an * kApStrip; e += kApWarps * 32) {
    const int r = e >> 6, c = e & (kApStrip - 1);
    As[e] = c < Sw ? __ldg(src + (long long)r * p.ld + c) : make_float2(0.f, 0.f);
  }
  if (tid < 2 * P - 1) {
    int s = 0;
    for (int k = 0; k < tid; ++k) s += P - abs(k - (P - 1));
    cumN[tid] = s;
  }
  if (tid < P) cum0[tid] = tid * P - tid * (tid - 1) / 2;
  __syncthreads();

  float2 *Rg = p.R + ((long long)ay * p.nc + ax0) * DD * DD;
  DivSmall divP, divG;
  divP.init(P);
  divG.init(Gc);
  for (int dc = 0; dc < Q; ++dc) {
    const int J = Q - dc, ncol = Sw - dc;  // output columns; strip columns with a partner
    const int nd = dc ? 2 * P - 1 : P;
    // row lags in decreasing output rows (0, 1, -1, 2, -2, ...), warps in turn
    for (int k = warp; k < nd; k += kApWarps) {
      const int d = dc ? ((k & 1) ? (k + 1) >> 1 : -(k >> 1)) : k;
      const int I = P - (d < 0 ? -d : d), i0 = d < 0 ? -d : 0;
      // ---- column sums of the products, walked down the diagonal --------
      const int o1 = lane + 32 < ncol ? 32 : 0;  // the lane's second column (or its first again)
      const float2 *pa = As + i0 * kApStrip + lane;
      const float2 *pb = As + (i0 + d) * kApStrip + lane + dc;
      float2 V0 = make_float2(0.f, 0.f), V1 = V0, U0 = V0, U1 = V0;
      int r = 0;
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
      Vw[lane] = V0;
      Vw[lane + 32] = V1;
      for (int s = 1; s < I; ++s) {  // row s - 1 leaves the box, row s - 1 + Hb enters
        const int oi = (s - 1 + Hb) * kApStrip, oo = (s - 1) * kApStrip;
        const float2 x0 = ap_prod(pa[oi], pb[oi]), y0 = ap_prod(pa[oo], pb[oo]);
        const float2 x1 = ap_prod(pa[oi + o1], pb[oi + o1]), y1 = ap_prod(pa[oo + o1], pb[oo + o1]);
        V0.x += x0.x - y0.x;
        V0.y += x0.y - y0.y;
        V1.x += x1.x - y1.x;
        V1.y += x1.y - y1.y;
        Vw[s * kApVPitch + lane] = V0;
        Vw[s * kApVPitch + lane + 32] = V1;
      }
      __syncwarp();
      // ---- window sums along the columns, one (aperture, output row) a lane
      const int cum = dc ? cumN[d + P - 1] : cum0[d];
      for (int q = lane; q < Gc * I; q += 32) {
        const int ap = q / I, s = q - ap * I;
        const float2 *v = Vw + s * kApVPitch + ap * p.sc;
        float2 W = v[0], W2 = make_float2(0.f, 0.f);
        int m = 1;
        for (; m + 1 < Wd; m += 2) {
          W.x += v[m].x;
          W.y += v[m].y;
          W2.x += v[m + 1].x;
          W2.y += v[m + 1].y;
        }
        if (m < Wd) {
          W.x += v[m].x;
          W.y += v[m].y;
        }
        W.x += W2.x;
        W.y += W2.y;
        float2 *t = T + ap * p.TS + J * (cum + s);
        t[0] = W;
        for (int j = 1; j < J; ++j) {  // column j - 1 leaves the window, j - 1 + Wd enters
          W.x += v[j - 1 + Wd].x - v[j - 1].x;
          W.y += v[j - 1 + Wd].y - v[j - 1].y;
          t[j] = W;
        }
      }
      __syncwarp();  // the column sums are read before the next row lag overwrites them
    }
    __syncthreads();
    // ---- R blocks of this lag: (j, j + dc), and for dc > 0 the mirrors ----
    DivSmall divJ;
    divJ.init(J);
    const int total = Gc * J * P * P * (dc ? 2 : 1);
    for (int e = tid; e < total; e += kApWarps * 32) {
      const int t1 = divP.q(e), col = e - t1 * P;
      const int t2 = divP.q(t1), row = t1 - t2 * P;
      const int t3 = divJ.q(t2), j = t2 - t3 * J;
      const int pass = divG.q(t3), ap = t3 - pass * Gc;
      // entry (i, i') of block (j, j + dc): row lag i' - i, output row min(i, i')
      const int i = pass ? col : row, ip = pass ? row : col;
      const int dd = ip - i, s = i < ip ? i : ip;
      float2 v;
      bool cj = pass != 0;
      if (dc) {
        v = T[ap * p.TS + J * (cumN[dd + P - 1] + s) + j];
      } else {  // the block on the diagonal: entries below it mirror those above
        v = T[ap * p.TS + J * (cum0[dd < 0 ? -dd : dd] + s) + j];
        cj = dd < 0;
      }
      v.x *= p.rK;
      v.y *= p.rK;
      if (cj) v.y = -v.y;
      if (dc == 0 && dd == 0) v.y = 0.f;
      const int rb = pass ? j + dc : j, cb = pass ? j : j + dc;
      Rg[(long long)ap * DD * DD + (long long)(row + P * rb) * DD + col + P * cb] = v;
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
