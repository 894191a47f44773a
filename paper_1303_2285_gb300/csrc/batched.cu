// Many input matrices of uneven N, M, P, Q in one persistent launch
// (Section 5.1: computing several covariance matrices concurrently keeps every
// core busy where one matrix has too few combinations).
//
// Each CTA owns whole matrices, taken from a schedule the host builds once by
// longest-processing-time-first assignment (cost = a model of the kernel's
// cycles per member over its work counts: products with their padding,
// passes, R elements; see batched_member_cost). A CTA never waits on another
// CTA, so the launch is one kernel and can be captured in a CUDA graph.
//
// Per matrix, the CTA goes through the column lags dc = 0..Q-1; for one dc it
// handles the combinations (dr, dc) of Eq. 3.3 together:
//   A. products over the inner rows [P-1, N-P] (every box holds them): warp
//      tasks (lag group of 8, 32 columns, row range), lanes own a column and
//      register-block 8 rows x 8 lags; inner-column lanes are summed over the
//      warp, fringe-column lanes keep their column sums;
//   B. products of the fringe rows with the inner columns: warp tasks (4 rows,
//      8 lags), lanes stride over the columns, one transpose reduction;
//   C. per combination: the inner-row part CV[j] of the box sum at column
//      offset j, and for each fringe row the box-row sums RV[j] (its own
//      fringe-column products formed once, warp scans);
//   D. per diagonal segment: seed with the direct sum over the box, walk down
//      the diagonal (subtract the leaving top row, add the entering bottom
//      row; compensated), divide by K, write R and its conjugate mirror.
// Every element of R is written by one thread; partial sums are combined in a
// fixed order in shared memory (no atomics).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <queue>
#include <vector>

#include "../../include/cov.h"
#include "batched_pipe.h"
#include "cov_device.cuh"
#include "cov_internal.h"
#include "smem_attr.h"
#include "plan.h"

namespace cov {

constexpr int kBMaxPQ = 16;      // P, Q <= 16
constexpr int kBMaxM = 512;      // M <= 512 (16 column blocks)
constexpr int kBMaxD = 2 * kBMaxPQ - 1;   // combinations per column lag
constexpr int kBMaxF = 2 * (kBMaxPQ - 1); // fringe rows / columns
constexpr int kBMaxCB = kBMaxM / 32;
constexpr int kBMaxRS = 4;       // row ranges of phase A
constexpr int kBWarps = 16;
constexpr int kBG = 8;           // lags per group
// shared memory: the per-combination arrays of one pass, for the largest
// member (P = Q = 16, M = 512: one column lag, 31 combinations)
constexpr size_t kBSmemBytes =
    (size_t)kBMaxD *
    (kBMaxCB * kBMaxRS + kBMaxF * kBMaxRS + kBMaxF + kBMaxPQ + kBMaxPQ * kBMaxF) * sizeof(float2);

struct BDesc {
  const float2 *A;
  float2 *R;
  long long lda;
  int N, M, P, Q;
};

__device__ __forceinline__ float2 ld2(const float2 *p) { return __ldg(p); }

// Combinations of a pass over the column lags [dc_a, dc_b): dc = 0 has P
// (dr = 0..P-1), every other dc 2P-1 (dr = -(P-1)..P-1), in dc order.
struct BPass {
  int P, dc_a, dc_b, n0;  // n0: combinations of dc_a (P if dc_a == 0)
  __device__ __forceinline__ int first(int dc) const {  // local index of (dr_lo(dc), dc)
    return dc == dc_a ? 0 : n0 + (dc - dc_a - 1) * (2 * P - 1);
  }
  __device__ __forceinline__ void of(int dl, int &dr, int &dc) const {
    if (dl < n0) {
      dc = dc_a;
    } else {
      dc = dc_a + 1 + (dl - n0) / (2 * P - 1);
    }
    const int lo = dc ? -(P - 1) : 0;
    dr = lo + dl - first(dc);
  }
  // group index over the pass (ng0 groups for dc_a, ng1 for each other dc)
  __device__ __forceinline__ void group(int gi, int ng0, int ng1, int &dc, int &g) const {
    if (gi < ng0) {
      dc = dc_a;
      g = gi;
    } else {
      dc = dc_a + 1 + (gi - ng0) / ng1;
      g = (gi - ng0) % ng1;
    }
  }
};

// L: re-seed interval of the walk (0: one seed per diagonal segment);
// rs_max: at most this many row ranges per column block in the products
// (1, 2 or 4) -- the tuned segment length and task shape.
__global__ void __launch_bounds__(kBWarps * 32, 1)
    k_batched(const BDesc *descs, const int *order, const int *cta_begin, int mean, int L,
              int rs_max) {
  extern __shared__ __align__(16) unsigned char smem_b[];
  float2 *pool = (float2 *)smem_b;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int mi = cta_begin[blockIdx.x]; mi < cta_begin[blockIdx.x + 1]; ++mi) {
    const BDesc d = descs[order[mi]];
    const int N = d.N, M = d.M, P = d.P, Q = d.Q;
    const long long lda = d.lda;
    const float2 *A = d.A;
    const int inner_lo = P - 1, n_inner = N - 2 * P + 2;
    const int n_cb = (M + 31) / 32, NFR = 2 * (P - 1), NFC = 2 * (Q - 1), W = M - Q + 1;
    const long long K = (long long)(N - P + 1) * (M - Q + 1);
    const long long DD = (long long)P * Q;
    // K exact in FP32 up to 2^24: the mean multiplies by its reciprocal
    const bool smallK = K <= (1LL << 24);
    const float rK = smallK ? 1.0f / (float)K : 1.0f;
    // row ranges of phase A: as many as keep 4 row chunks each (at most 4)
    int RS = 1;
    while (RS < rs_max && n_inner >= 32 * RS * 2) RS *= 2;
    // per-pass shared arrays (float2), the pass's combination index dl
    // fastest (threads of phases C and D take consecutive dl): core
    // [n_cb*RS][dl], cs [NFC*RS][dl], sin [NFR][dl], cv [Q][dl], rv [Q][NFR][dl]
    const int per = n_cb * RS + NFC * RS + NFR + Q + Q * NFR;
    const int cap = (int)(kBSmemBytes / sizeof(float2)) / per;  // combinations per pass
    for (int dc_a = 0; dc_a < Q;) {
      // as many whole column lags as fit
      int dc_b = dc_a, nDp = 0;
      while (dc_b < Q && nDp + (dc_b ? 2 * P - 1 : P) <= cap) nDp += dc_b++ ? 2 * P - 1 : P;
      const BPass ps = {P, dc_a, dc_b, dc_a ? 2 * P - 1 : P};
      float2 *core = pool;
      float2 *cs = core + nDp * n_cb * RS;
      float2 *sinp = cs + nDp * NFC * RS;
      float2 *cv = sinp + nDp * NFR;
      float2 *rv = cv + nDp * Q;
      const int ng0 = (ps.n0 + kBG - 1) / kBG, ng1 = (2 * P - 1 + kBG - 1) / kBG;
      const int ngp = ng0 + (dc_b - dc_a - 1) * ng1;  // groups of the pass
      // ---- A: products over inner rows -------------------------------------
      // Packed FP32x2 FMA with direct and cross accumulator pairs (as the
      // single-matrix product kernel). Loads use clamped addresses instead of
      // predicates: a lane past the last column reads column M-1 and its sums
      // are dropped; a lane whose partner column m+dc is past M zeroes its a
      // values (no valid product); partner rows past N-1 occur only for the
      // unused lag slots of the last group, whose sums are dropped.
      // consecutive warps take the lag groups of one (column block, row range),
      // so the A block they share stays in L1
      const int nA = ngp * n_cb * RS;
      for (int t = warp; t < nA; t += kBWarps) {
        const int gi = t % ngp, rs = (t / ngp) % RS, cb = t / (ngp * RS);
        int dc, g;
        ps.group(gi, ng0, ng1, dc, g);
        const int dr_lo = dc ? -(P - 1) : 0;
        const int d0 = dr_lo + g * kBG;
        const int cnt = min(kBG, P - d0);
        const int dl0 = ps.first(dc) + g * kBG;
        const int r_beg = inner_lo + (int)((long long)n_inner * rs / RS);
        const int r_end = inner_lo + (int)((long long)n_inner * (rs + 1) / RS);
        const int m = cb * 32 + lane;
        const bool mok = m < M, bok = m + dc < M;
        const int ma = mok ? m : M - 1, mb = bok ? m + dc : M - 1;
        const unsigned long long amask = bok ? ~0ull : 0ull;
        const unsigned long long *ua = (const unsigned long long *)A;
        unsigned long long accd[kBG], accx[kBG];
#pragma unroll
        for (int k = 0; k < kBG; ++k) accd[k] = accx[k] = 0ull;
        const int ld = (int)lda;  // N * lda < 2^31 (checked when the plan is made)
        for (int n = r_beg; n < r_end; n += 8) {
          const int nv = r_end - n;  // valid a rows of this chunk (>= 8 except the last)
          const int b0 = n + d0;     // >= 0: n >= P - 1 and d0 >= -(P - 1)
          unsigned long long a[8], as[8];
          if (nv >= 8 && b0 + 8 + kBG - 1 <= N) {
            // whole chunk, every partner row inside A: plain 32-bit offsets
            const unsigned long long *pa = ua + (n * ld + ma), *pb = ua + (b0 * ld + mb);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
              a[r] = __ldg(pa + r * ld) & amask;
              as[r] = swap2(a[r]);
            }
#pragma unroll
            for (int k = 0; k < 8 + kBG - 1; ++k) {
              const unsigned long long b = __ldg(pb + k * ld);
#pragma unroll
              for (int r = 0; r < 8; ++r) {
                const int gg = k - r;
                if (gg >= 0 && gg < kBG) {
                  ffma2(accd[gg], a[r], b);
                  ffma2(accx[gg], as[r], b);
                }
              }
            }
            continue;
          }
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int row = n + r < r_end ? n + r : r_end - 1;
            a[r] = (r < nv ? __ldg(ua + (long long)row * lda + ma) : 0ull) & amask;
            as[r] = swap2(a[r]);
          }
          const bool clamp = b0 + 8 + kBG - 1 > N;
#pragma unroll
          for (int k = 0; k < 8 + kBG - 1; ++k) {
            const int row = clamp ? min(b0 + k, N - 1) : b0 + k;
            const unsigned long long b = __ldg(ua + (long long)row * lda + mb);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
              const int gg = k - r;
              if (gg >= 0 && gg < kBG) {
                ffma2(accd[gg], a[r], b);
                ffma2(accx[gg], as[r], b);
              }
            }
          }
        }
        float2 acc[kBG];
#pragma unroll
        for (int k = 0; k < kBG; ++k) {
          const float2 dd = upk2(accd[k]), xx = upk2(accx[k]);
          acc[k] = make_float2(dd.x + dd.y, xx.x - xx.y);
        }
        const bool inner = m >= Q - 1 && m <= M - Q;
        if (mok && !inner) {
          const int fc = m < Q - 1 ? m : m - (M - 2 * Q + 2);
#pragma unroll
          for (int k = 0; k < kBG; ++k)
            if (k < cnt) cs[(fc * RS + rs) * nDp + dl0 + k] = acc[k];
        }
        float v[2 * kBG];
#pragma unroll
        for (int k = 0; k < kBG; ++k) {
          v[2 * k] = inner ? acc[k].x : 0.f;
          v[2 * k + 1] = inner ? acc[k].y : 0.f;
        }
        warp_transpose_reduce<2 * kBG>(v, lane);  // lane holds value index lane >> 1
        if ((lane & 1) == 0) {
          const int k = lane >> 2, comp = (lane >> 1) & 1;
          if (k < cnt) ((float *)&core[(cb * RS + rs) * nDp + dl0 + k])[comp] = v[0];
        }
      }
      // ---- B: fringe rows x inner columns ---------------------------------
      // narrow members (few inner columns): one thread per (combination,
      // fringe row), serial over the inner columns with two accumulators;
      // otherwise warp tasks (4 rows x 8 lags, lanes over the columns)
      const int n_ic = M - 2 * Q + 2;
      const bool narrow = n_ic <= 64;
      if (narrow) {
        for (int t = threadIdx.x; t < nDp * NFR; t += blockDim.x) {
          const int dl = t % nDp, fr = t / nDp;
          int dr, dc;
          ps.of(dl, dr, dc);
          const int n = fr < P - 1 ? fr : (N - P + 1) + (fr - (P - 1));
          float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
          if (n + dr >= 0 && n + dr < N) {
            const float2 *An = A + (long long)n * lda + (Q - 1);
            const float2 *Ab = A + (long long)(n + dr) * lda + (Q - 1) + dc;
            int m = 0;
            for (; m + 1 < n_ic; m += 2) {
              cmac_conj(s0, ld2(An + m), ld2(Ab + m));
              cmac_conj(s1, ld2(An + m + 1), ld2(Ab + m + 1));
            }
            if (m < n_ic) cmac_conj(s0, ld2(An + m), ld2(Ab + m));
          }
          sinp[fr * nDp + dl] = make_float2(s0.x + s1.x, s0.y + s1.y);
        }
      }
      const int nrb = (P - 1 + 3) / 4;
      const int nB = narrow ? 0 : 2 * nrb * ngp;
      for (int t = warp; t < nB; t += kBWarps) {
        const int gi = t % ngp, rb = (t / ngp) % nrb, side = t / (ngp * nrb);
        int dc, g;
        ps.group(gi, ng0, ng1, dc, g);
        const int dr_lo = dc ? -(P - 1) : 0;
        const int d0 = dr_lo + g * kBG, cnt = min(kBG, P - d0);
        const int dl0 = ps.first(dc) + g * kBG;
        const int fr0 = rb * 4, nrows = min(4, P - 1 - fr0);
        const int nbase = side == 0 ? fr0 : (N - P + 1) + fr0;
        // acc += a * conj(b) as packed (re, im) pairs: (ar, ai) * (br, br) then
        // (ai, -ar) * (bi, bi), the roundings and order of cmac_conj;
        // 32-bit row offsets (N * lda < 2^31)
        unsigned long long acc[4][kBG];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int k = 0; k < kBG; ++k) acc[r][k] = 0ull;
        const int ld = (int)lda;
        const int rb0 = nbase + d0;
        for (int m = Q - 1 + lane; m <= M - Q; m += 32) {
          unsigned long long a1[4], a2[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const float2 x = r < nrows ? ld2(A + ((nbase + r) * ld + m)) : make_float2(0.f, 0.f);
            a1[r] = pk2(x.x, x.y);
            a2[r] = pk2(x.y, -x.x);
          }
#pragma unroll
          for (int k = 0; k < 4 + kBG - 1; ++k) {
            const int row = rb0 + k;
            const float2 b = (row >= 0 && row < N) ? ld2(A + (row * ld + m + dc)) : make_float2(0.f, 0.f);
            const unsigned long long bx = pk2(b.x, b.x), by = pk2(b.y, b.y);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              const int gg = k - r;
              if (gg >= 0 && gg < kBG) {
                ffma2(acc[r][gg], a1[r], bx);
                ffma2(acc[r][gg], a2[r], by);
              }
            }
          }
        }
        float v[2 * 4 * kBG];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int k = 0; k < kBG; ++k) {
            const float2 x = upk2(acc[r][k]);
            v[2 * (r * kBG + k)] = x.x;
            v[2 * (r * kBG + k) + 1] = x.y;
          }
        warp_transpose_reduce<2 * 4 * kBG>(v, lane);  // lane holds complex index lane
        const int r = lane / kBG, k = lane % kBG;
        if (r < nrows && k < cnt)
          sinp[(side * (P - 1) + fr0 + r) * nDp + dl0 + k] = make_float2(v[0], v[1]);
      }
      __syncthreads();
      // ---- C: CV per combination, RV per (combination, fringe row) ---------
      // one thread per value set: suffix sums over the left fringe columns,
      // prefix sums over the right ones, as running sums
      const int nC = nDp * (1 + NFR);
      for (int t = threadIdx.x; t < nC; t += blockDim.x) {
        const int dl = t % nDp, kind = t / nDp;  // kind 0: CV, kind 1+fr: RV of fringe row fr
        int dr, dc;
        ps.of(dl, dr, dc);
        const int J = Q - dc;
        float2 *cvd = cv + dl;  // cv[j][dl] at cvd[j * nDp]
        if (kind == 0) {
          Neu<float> cr, ci;
          for (int k = 0; k < n_cb * RS; ++k) {
            const float2 x = core[k * nDp + dl];
            cr.add(x.x);
            ci.add(x.y);
          }
          const float2 *csd = cs + dl;  // cs[fc*RS + rs][dl] at csd[(fc*RS + rs) * nDp]
          // left fringe columns k = Q-2 .. j (suffix), then right ones k < j
          float2 suf = make_float2(0.f, 0.f);
          for (int k = Q - 2; k >= 0; --k) {
            float2 l = make_float2(0.f, 0.f);
            for (int rs = 0; rs < RS; ++rs) {
              l.x += csd[(k * RS + rs) * nDp].x;
              l.y += csd[(k * RS + rs) * nDp].y;
            }
            suf.x += l.x;
            suf.y += l.y;
            if (k < J) cvd[k * nDp] = suf;
          }
          if (Q - 1 < J) cvd[(Q - 1) * nDp] = make_float2(0.f, 0.f);
          float2 pre = make_float2(0.f, 0.f);
          for (int j = 0; j < J; ++j) {
            Neu<float> vr = cr, vi = ci;
            vr.add(cvd[j * nDp].x);
            vi.add(cvd[j * nDp].y);
            vr.add(pre.x);
            vi.add(pre.y);
            cvd[j * nDp] = make_float2(vr.value(), vi.value());
            if (j < Q - 1) {
              for (int rs = 0; rs < RS; ++rs) {
                pre.x += csd[((Q - 1 + j) * RS + rs) * nDp].x;
                pre.y += csd[((Q - 1 + j) * RS + rs) * nDp].y;
              }
            }
          }
        } else {
          const int fr = kind - 1;
          const int n = fr < P - 1 ? fr : (N - P + 1) + (fr - (P - 1));
          const bool rowok = n + dr >= 0 && n + dr < N;
          const float2 si = rowok ? sinp[fr * nDp + dl] : make_float2(0.f, 0.f);
          const float2 *An = A + (long long)n * lda;
          const float2 *Ab = A + (long long)(rowok ? n + dr : 0) * lda + dc;
          float2 *rvd = rv + fr * nDp + dl;  // rv[j][fr][dl] at rvd[j * NFR * nDp]
          const int RJ = NFR * nDp;
          // own left fringe-column products, suffix sums
          float2 suf = make_float2(0.f, 0.f);
#pragma unroll 4
          for (int k = Q - 2; k >= 0; --k) {
            if (rowok) cmac_conj(suf, ld2(An + k), ld2(Ab + k));
            if (k < J) rvd[k * RJ] = make_float2(si.x + suf.x, si.y + suf.y);
          }
          if (Q - 1 < J) rvd[(Q - 1) * RJ] = si;
          // own right fringe-column products, prefix sums
          float2 pre = make_float2(0.f, 0.f);
#pragma unroll 4
          for (int j = 1; j < J; ++j) {
            const int k = j - 1;
            if (rowok && W + k + dc < M) cmac_conj(pre, ld2(An + W + k), ld2(Ab + W + k));
            rvd[j * RJ].x += pre.x;
            rvd[j * RJ].y += pre.y;
          }
        }
      }
      __syncthreads();
      // ---- D: seed, walk, write -------------------------------------------
      // one thread per (combination, column offset j, segment of L outputs;
      // one segment when L = 0): the diagonal of block (j, j + dc) from
      // output is on. The seed's terms, the top fringe rows still in the
      // box and the bottom ones already in, are the contiguous range
      // rv[is .. is+P-2] of the staged row sums, summed as two interleaved
      // compensated chains. The mean's 1/K is a multiplication by the
      // reciprocal (within 1.5 ulp of the quotient; R has (PQ)^2 elements,
      // so this is per-element work).
      const int nseg = L > 0 ? (P + L - 1) / L : 1;
      for (int t = threadIdx.x; t < nDp * Q * nseg; t += blockDim.x) {
        const int dl = t % nDp, rest = t / nDp, j = rest % Q, c = rest / Q;
        int dr, dc;
        ps.of(dl, dr, dc);
        if (j >= Q - dc) continue;
        const int adr = dr < 0 ? -dr : dr;
        const int i0 = dr < 0 ? -dr : 0, I = P - adr;
        const int is = i0 + (L > 0 ? c * L : 0);
        if (is >= i0 + I) continue;
        const int ie = L > 0 && is + L < i0 + I ? is + L : i0 + I;
        const float2 *rvj = rv + j * NFR * nDp + dl;  // rv[j][n][dl] at rvj[n * nDp]
        Neu<float> orr, oii, o2r, o2i;
        orr.add(cv[j * nDp + dl].x);
        oii.add(cv[j * nDp + dl].y);
        {
          const int ue = is + P - 1;
          int u = is;
          for (; u + 2 <= ue; u += 2) {
            const float2 x = rvj[u * nDp], y = rvj[(u + 1) * nDp];
            orr.add(x.x);
            oii.add(x.y);
            o2r.add(y.x);
            o2i.add(y.y);
          }
          if (u < ue) {
            orr.add(rvj[u * nDp].x);
            oii.add(rvj[u * nDp].y);
          }
          orr.merge(o2r.s, o2r.c);
          oii.merge(o2i.s, o2i.c);
        }
        // element (i, i + dr) of the block and its mirror; R has < 2^31 elements
        int e1 = (is + P * j) * (int)DD + (is + dr) + P * (j + dc);
        int e2 = ((is + dr) + P * (j + dc)) * (int)DD + is + P * j;
        for (int i = is; i < ie; ++i) {
          float re = orr.value(), im = oii.value();
          if (mean) {
            if (smallK) {
              re *= rK;
              im *= rK;
            } else {
              re = (float)((double)re / (double)K);
              im = (float)((double)im / (double)K);
            }
          }
          if (dr == 0 && dc == 0) im = 0.f;
          d.R[e1] = make_float2(re, im);
          if (e1 != e2) d.R[e2] = make_float2(re, -im);
          e1 += (int)DD + 1;
          e2 += (int)DD + 1;
          if (i + 1 < ie) {  // walk: row i leaves the box, row i+N-P+1 enters
            orr.add(-rvj[i * nDp].x);
            oii.add(-rvj[i * nDp].y);
            orr.add(rvj[(P - 1 + i) * nDp].x);
            oii.add(rvj[(P - 1 + i) * nDp].y);
          }
        }
      }
      __syncthreads();
      dc_a = dc_b;
    }
  }
}

// ---------------------------------------------------------------------------
// Batches whose members are all small (M <= 32, N M <= 1024): one warp per
// member, whose A it stages in shared memory, 16 members in flight per SM,
// no CTA barriers. Lanes own columns m. Per
// combination (dr, dc) of Eq. 3.3, in the notation of Section 4.2:
//  - the column sums C(i, m) of the products over the box rows n = i ..
//    i+H-1 of the first output i (H = N-P+1) seed the walk; the products
//    of the first I-1 box rows are kept (per lane, in shared memory);
//  - the walk down the diagonal adds the entering row's products and
//    subtracts the kept products of the leaving row (compensated), so each
//    distinct product (Eq. 3.5) is formed once;
//  - for every output i, the box sums over the columns j .. j+Wd-1
//    (Wd = M-Q+1) of all column offsets j come from one warp scan of C:
//    S(i, j) = pre(j+Wd-1) - pre(j-1), the column walk in closed form;
//    lane j writes element (i + P j, i + dr + P (j + dc)) of R and its
//    conjugate mirror.
// ---------------------------------------------------------------------------
constexpr int kWWarps = 8;    // members in flight per CTA (two CTAs an SM)
constexpr int kWMaxM = 32;    // one column per lane
constexpr int kWMaxPQ = 16;
constexpr int kWMaxElems = 1024;  // N * M: the member's A is staged whole
constexpr size_t kWWarpBytes = ((size_t)(kWMaxPQ - 1) * 32 + kWMaxElems) * sizeof(float2);

__device__ __forceinline__ float warp_scan_incl(float x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

__global__ void __launch_bounds__(kWWarps * 32, 2)
    k_batched_warp(const BDesc *descs, const int *order, const int *slot_begin, int mean) {
  // per warp: the kept products of the leaving rows [P-1][32], then the
  // member's A (row pitch M)
  extern __shared__ __align__(16) unsigned char smem_w[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = blockIdx.x * kWWarps + warp;
  float2(*keep)[32] = (float2(*)[32])(smem_w + (size_t)warp * kWWarpBytes);
  float2 *As = (float2 *)(smem_w + (size_t)warp * kWWarpBytes) + (kWMaxPQ - 1) * 32;
  for (int mi = slot_begin[slot]; mi < slot_begin[slot + 1]; ++mi) {
    const BDesc d = descs[order[mi]];
    const int N = d.N, M = d.M, P = d.P, Q = d.Q;
    const int H = N - P + 1, Wd = M - Q + 1, DD = P * Q;
    const long long K = (long long)H * Wd;
    const bool smallK = K <= (1LL << 24);
    const float rK = smallK ? 1.0f / (float)K : 1.0f;
    // stage A (row pitch M) into the warp's buffer
    __syncwarp();  // the previous member's reads of As are done
#pragma unroll 4
    for (int r = 0; r < N; ++r)
      if (lane < M) As[r * M + lane] = __ldg(d.A + (long long)r * d.lda + lane);
    __syncwarp();
    const int ld = M;
    const float2 *A = As;
    const bool mok = lane < M;
    for (int dc = 0; dc < Q; ++dc) {
      const bool bok = mok && lane + dc < M;  // a product exists in this column
      for (int dr = dc == 0 ? 0 : -(P - 1); dr < P; ++dr) {
        const int i_lo = dr < 0 ? -dr : 0, I = P - (dr < 0 ? -dr : dr);
        // seed: rows i_lo .. i_lo+H-1 (two plain accumulators), keeping the
        // first I-1 rows' products
        float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
        if (bok) {
          const float2 *pa = A + (i_lo * ld + lane), *pb = A + ((i_lo + dr) * ld + lane + dc);
          int r = 0;
#pragma unroll 4
          for (; r < I - 1; ++r) {
            float2 v = make_float2(0.f, 0.f);
            cmac_conj(v, pa[r * ld], pb[r * ld]);
            keep[r][lane] = v;
            s0.x += v.x;
            s0.y += v.y;
          }
#pragma unroll 4
          for (; r + 1 < H; r += 2) {
            cmac_conj(s0, pa[r * ld], pb[r * ld]);
            cmac_conj(s1, pa[(r + 1) * ld], pb[(r + 1) * ld]);
          }
          if (r < H) cmac_conj(s0, pa[r * ld], pb[r * ld]);
        }
        Neu<float> cr, ci;
        cr.add(s0.x + s1.x);
        ci.add(s0.y + s1.y);
        const int J = Q - dc;
        for (int i = i_lo; i < i_lo + I; ++i) {
          const float pr = warp_scan_incl(cr.value(), lane), pi = warp_scan_incl(ci.value(), lane);
          const int hi = lane + Wd - 1 < 31 ? lane + Wd - 1 : 31;
          const float hr = __shfl_sync(0xffffffffu, pr, hi), hm = __shfl_sync(0xffffffffu, pi, hi);
          const float lr = __shfl_sync(0xffffffffu, pr, lane > 0 ? lane - 1 : 0);
          const float lm = __shfl_sync(0xffffffffu, pi, lane > 0 ? lane - 1 : 0);
          if (lane < J) {
            float re = lane > 0 ? hr - lr : hr, im = lane > 0 ? hm - lm : hm;
            if (mean) {
              if (smallK) {
                re *= rK;
                im *= rK;
              } else {
                re = (float)((double)re / (double)K);
                im = (float)((double)im / (double)K);
              }
            }
            if (dr == 0 && dc == 0) im = 0.f;
            const int a = i + P * lane, b = i + dr + P * (lane + dc);
            d.R[a * DD + b] = make_float2(re, im);
            if (a != b) d.R[b * DD + a] = make_float2(re, -im);
          }
          if (i + 1 < i_lo + I && bok) {  // walk: row i leaves the box, row i+H enters
            float2 vin = make_float2(0.f, 0.f);
            cmac_conj(vin, A[(i + H) * ld + lane], A[(i + H + dr) * ld + lane + dc]);
            const float2 vout = keep[i - i_lo][lane];
            cr.add(-vout.x);
            ci.add(-vout.y);
            cr.add(vin.x);
            ci.add(vin.y);
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Batches of small members (M <= 32, N M <= 1024, P, Q <= 16, PQ <= 100;
// the apertures of an image, Section 2.3): one CTA (8 warps) per member in
// flight, several CTAs an SM. The member's A is staged in shared memory;
// warp w takes the combinations w, w + 8, ... of Eq. 3.3 and, per
// combination (dr, dc), computes every owned output (i, j) (Eq. 3.7-3.8) as
// a separable box sum of its product image:
//  - lanes own columns m; the column sums V(m) over the box rows of the first
//    output i0 are seeded directly, the products of the rows that later leave
//    the box are kept (per warp, in shared memory), and the walk down the
//    diagonal adds the entering row's products and subtracts the kept ones
//    (every distinct product of Eq. 3.5 formed once);
//  - per output i, the sums over the box columns j .. j + Wd - 1 are window
//    sums across the lanes, built by doubling (windows of 1, 2, 4, ... lanes,
//    one shuffle each) and composed from the binary digits of Wd, so no
//    difference of prefix sums is formed.
// The outputs go to a shared-memory table of the upper triangle (combination
// by combination, i then j); the CTA then writes R row by row, both
// triangles, coalesced, scaling by the FP32 reciprocal of K.
// ---------------------------------------------------------------------------
constexpr int kXWarps = 8;
constexpr int kXMaxM = 32;
constexpr int kXMaxPQ = 16;
constexpr int kXMaxD = 100;        // PQ: the output table holds PQ (PQ + 1) / 2 entries
constexpr int kXMaxElems = 1024;   // N * M

__host__ __device__ inline int box_table_entries(int P, int Q) { return P * Q * (P * Q + 1) / 2; }
// Shared memory of one member: the kept products [warps][P-1][32], A, the
// output table and the combinations' table offsets.
__host__ __device__ inline size_t box_smem_bytes(int NM, int P, int Q) {
  const int uc = P * Q + (P - 1) * (Q - 1);
  return ((size_t)kXWarps * (P - 1) * 32 + (size_t)NM + (size_t)box_table_entries(P, Q)) *
             sizeof(float2) +
         (size_t)uc * sizeof(int);
}

// Offset in the output table of combination (dr, dc)'s outputs: the
// combinations in the order of combo_index, each with (P - |dr|) x (Q - dc)
// entries.
__device__ __forceinline__ int box_table_offset(int P, int Q, int dr, int dc) {
  if (dc == 0) return Q * (dr * P - dr * (dr - 1) / 2);
  const int first = Q * P * (P + 1) / 2 + P * P * ((dc - 1) * Q - dc * (dc - 1) / 2);
  const int before = dr <= 0 ? (P + dr - 1) * (P + dr) / 2 : P * (P - 1) / 2 + dr * P - dr * (dr - 1) / 2;
  return first + (Q - dc) * before;
}

// Sum of v over lanes lane .. lane + Wd - 1, for the lanes whose window ends
// at lane 31 or before (the other lanes receive unspecified values): windows
// of 1, 2, 4, ... lanes by doubling (one 64-bit shuffle and one packed FP32x2
// add each), composed from the binary digits of Wd.
__device__ __forceinline__ unsigned long long add_f32x2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ float2 lane_window_sum(float2 v, int Wd) {
  unsigned long long w = pk2(v.x, v.y);
  if ((Wd & (Wd - 1)) == 0) {  // a power of two: doubling alone
#pragma unroll
    for (int k = 0; k < 5; ++k)
      if ((1 << k) < Wd) w = add_f32x2(w, __shfl_down_sync(0xffffffffu, w, 1 << k));
    return upk2(w);
  }
  unsigned long long r = 0ull;
  int off = 0;
  bool first = true;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int b = 1 << k;
    if (b > Wd) break;
    if (Wd & b) {
      const unsigned long long t = off == 0 ? w : __shfl_down_sync(0xffffffffu, w, off);
      r = first ? t : add_f32x2(r, t);
      first = false;
      off += b;
    }
    if (2 * b <= Wd) w = add_f32x2(w, __shfl_down_sync(0xffffffffu, w, b));
  }
  return upk2(r);
}

__device__ __forceinline__ float2 prod_conj(float2 a, float2 b) {
  float2 v = make_float2(0.f, 0.f);
  cmac_conj(v, a, b);
  return v;
}

__global__ void __launch_bounds__(kXWarps * 32, 3)
    k_batched_box(const BDesc *descs, const int *order, const int *slot_begin, int mean) {
  extern __shared__ __align__(16) unsigned char smem_x[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int mi = slot_begin[blockIdx.x]; mi < slot_begin[blockIdx.x + 1]; ++mi) {
    const BDesc d = descs[order[mi]];
    const int N = d.N, M = d.M, P = d.P, Q = d.Q;
    const int H = N - P + 1, Wd = M - Q + 1, DD = P * Q, nUC = DD + (P - 1) * (Q - 1);
    float2 *keep = (float2 *)smem_x + warp * (P - 1) * 32 + lane;  // [warp][P-1][32]
    float2 *As = (float2 *)smem_x + kXWarps * (P - 1) * 32;     // [N][M]
    float2 *OT = As + N * M;                       // upper-triangle outputs
    int *offs = (int *)(OT + box_table_entries(P, Q));
    __syncthreads();  // the previous member's reads of shared memory are done
    for (int r = warp; r < N; r += kXWarps)
      if (lane < M) As[r * M + lane] = __ldg(d.A + (long long)r * d.lda + lane);
    for (int c = tid; c < nUC; c += kXWarps * 32) {
      int dr, dc;
      combo_of(P, c, dr, dc);
      offs[c] = box_table_offset(P, Q, dr, dc);
    }
    __syncthreads();
    // ---- box sums of every combination ------------------------------------
    for (int c = warp; c < nUC; c += kXWarps) {
      int dr, dc;
      combo_of(P, c, dr, dc);
      const int i0 = dr < 0 ? -dr : 0, I = P - (dr < 0 ? -dr : dr), J = Q - dc;
      const bool mok = lane < M - dc;  // the column's partner m + dc lies in A
      const float2 *pa = As + i0 * M + (mok ? lane : 0);
      const float2 *pb = As + (i0 + dr) * M + (mok ? lane + dc : 0);
      // seed: the box rows r = 0 .. H-1 of output i0; rows r < I-1 leave the
      // box later and are kept
      float2 V = make_float2(0.f, 0.f), V2 = make_float2(0.f, 0.f);
      if (mok) {
        for (int r = 0; r < I - 1; ++r) {
          const float2 x = prod_conj(pa[r * M], pb[r * M]);
          keep[r * 32] = x;
          V.x += x.x;
          V.y += x.y;
        }
        int r = I - 1 > 0 ? I - 1 : 0;
        for (; r + 1 < H; r += 2) {
          cmac_conj(V, pa[r * M], pb[r * M]);
          cmac_conj(V2, pa[(r + 1) * M], pb[(r + 1) * M]);
        }
        if (r < H) cmac_conj(V, pa[r * M], pb[r * M]);
      }
      V.x += V2.x;
      V.y += V2.y;
      float2 *op = OT + offs[c] + lane;
      const float2 *pain = pa + H * M, *pbin = pb + H * M, *kp = keep;
      for (int s = 0; s < I; ++s) {
        const float2 o = lane_window_sum(V, Wd);
        if (lane < J) *op = o;
        op += J;
        if (s < I - 1 && mok) {  // row s leaves the box, row s + H enters
          const float2 xin = prod_conj(*pain, *pbin);
          const float2 xout = *kp;
          V.x += xin.x - xout.x;
          V.y += xin.y - xout.y;
        }
        pain += M;
        pbin += M;
        kp += 32;
      }
    }
    __syncthreads();
    // ---- R, row by row (both triangles) ------------------------------------
    const long long K = (long long)H * Wd;
    const float rK = mean ? 1.0f / (float)K : 1.0f;
    int ib[4], jb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int b = lane + 32 * q;
      ib[q] = b % P;
      jb[q] = b / P;
    }
    for (int a = warp; a < DD; a += kXWarps) {
      const int ia = a % P, ja = a / P;
      float2 *Ra = d.R + (long long)a * DD;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int b = lane + 32 * q;
        if (b < DD) {
          const bool mir = b < a;
          const int dr = mir ? ia - ib[q] : ib[q] - ia, dc = mir ? ja - jb[q] : jb[q] - ja;
          const int s = (mir ? ib[q] : ia) - (dr < 0 ? -dr : 0), j = mir ? jb[q] : ja;
          float2 v = OT[offs[combo_index(P, dr, dc)] + s * (Q - dc) + j];
          v.x *= rK;
          v.y *= rK;
          if (mir) v.y = -v.y;
          if (a == b) v.y = 0.f;
          Ra[b] = v;
        }
      }
    }
  }
}

}  // namespace cov

// ---------------------------------------------------------------------------
// Host side: plan (validation + LPT schedule), upload, launch.
// ---------------------------------------------------------------------------
struct cov_batched_plan {
  std::vector<cov::BDesc> descs;
  std::vector<int> order;      // matrix indices, slot by slot
  std::vector<int> cta_begin;  // slots + 1 offsets into order
  int grid;
  int sms;
  int cta_ok;                  // every member fits k_batched
  int narrow_ok;               // every member fits k_batched_warp
  int box_ok;                  // every member fits k_batched_box
  int pipe_ok;                 // every member fits the stage form (batched_pipe.cu)
  size_t box_smem;             // k_batched_box's shared memory for the largest member
  cov::PipePlan pipe;          // the stage form's member plans and tables
  int form;                    // tuned: 0 = CTA form, 1 = one warp per member, 2 = box form,
                               // 3 = stage form
  int L;                       // tuned: re-seed interval of the CTA form's walk (0: none)
  int rs_max;                  // tuned: row ranges per column block (1, 2, 4)
  int mean;
  size_t off_desc, off_order, off_begin, total;
};

namespace {

// A member the CTA, warp and box forms can take (they also need the
// per-form limits checked in cov_batched_plan_create).
bool batched_shape_ok(const cov_desc &d) {
  return d.A && d.R && d.N >= 1 && d.M >= 1 && d.P >= 1 && d.Q >= 1 && d.P <= cov::kBMaxPQ &&
         d.Q <= cov::kBMaxPQ && d.N >= 2 * d.P - 1 && d.M >= 2 * d.Q - 1 && d.M <= cov::kBMaxM &&
         d.lda >= d.M && (long long)d.N * d.lda < (1LL << 31) && (((uintptr_t)d.A) & 7) == 0 &&
         (((uintptr_t)d.R) & 7) == 0;
}

// The stage form keeps every member's partial sums in the workspace: it is
// offered only while they stay within this many bytes (always where no other
// form takes the members).
constexpr size_t kPipeMaxWorkspace = (size_t)4 << 30;

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Cost of one member in k_batched, in SM cycles: a linear model over the
// kernel's own work counts (padded inner-row products of phase A, its warp
// tasks, the fringe-row tasks, passes over the column lags, R elements, ...),
// with non-negative weights fitted to per-member cycle counts measured on
// GB300 for the 4096-member uneven workload (median error 2 %). It replaces
// the distinct-product count in the LPT schedule, whose error on small and
// narrow members (padding, per-pass and per-element work) left the slowest
// CTA 12 % above the mean.
double batched_member_cost(long long N, long long M, int P, int Q) {
  const long long n_inner = N - 2LL * P + 2;
  int RS = 1;
  while (RS < cov::kBMaxRS && n_inner >= 32LL * RS * 2) RS *= 2;
  const long long n_cb = (M + 31) / 32;
  const int NFR = 2 * (P - 1), NFC = 2 * (Q - 1);
  const long long n_ic = M - 2LL * Q + 2;
  const long long uc = (long long)P * Q + (long long)(P - 1) * (Q - 1);
  double issuedA = 0;  // phase A: lag slots x column lanes x chunk rows
  long long ngt = 0;   // lag groups over all column lags
  for (int dc = 0; dc < Q; ++dc) {
    const long long ng = ((dc ? 2 * P - 1 : P) + cov::kBG - 1) / cov::kBG;
    ngt += ng;
    for (int rs = 0; rs < RS; ++rs) {
      const long long nr = n_inner * (rs + 1) / RS - n_inner * rs / RS;
      issuedA += (double)(ng * cov::kBG) * (n_cb * 32) * (((nr + 7) / 8) * 8);
    }
  }
  // passes over the column lags, as the kernel forms them
  const long long per = n_cb * RS + (long long)NFC * RS + NFR + Q + (long long)Q * NFR;
  const long long cap = (long long)(cov::kBSmemBytes / sizeof(float2)) / per;
  long long passes = 0;
  for (int dc_a = 0; dc_a < Q;) {
    long long n = 0;
    int dc_b = dc_a;
    while (dc_b < Q && n + (dc_b ? 2 * P - 1 : P) <= cap) n += dc_b++ ? 2 * P - 1 : P;
    if (dc_b == dc_a) dc_b = dc_a + 1;  // (cannot happen for accepted shapes)
    ++passes;
    dc_a = dc_b;
  }
  const double tasksA = (double)ngt * n_cb * RS;
  const double tasksB = n_ic > 64 ? 2.0 * ((P - 1 + 3) / 4) * ngt * ((n_ic + 31) / 32) : 0.0;
  const double narrowB = n_ic <= 64 ? (double)uc * NFR * (n_ic > 0 ? n_ic : 0) : 0.0;
  const double DD = (double)P * Q;
  return 0.05762 * issuedA + 2.111 * DD * DD + 11380.0 * passes + 120.1 + 136.0 * tasksA +
         99.76 * tasksB + 0.2717 * narrowB + 9.607 * (double)uc * Q + 0.2529 * (double)N * M;
}

}  // namespace

extern "C" {

cov_status cov_partition_matrices(const cov_desc *descs, int count, int n_ranks, int32_t *rank_of,
                                  int64_t *rank_cost) {
  if (!descs || count < 1 || n_ranks < 1 || n_ranks > 65536 || !rank_of) return COV_EINVAL;
  std::vector<long long> cost(count);
  for (int i = 0; i < count; ++i) {
    const cov_desc &d = descs[i];
    if (d.N < 1 || d.M < 1 || d.P < 1 || d.Q < 1 || d.P > d.N || d.Q > d.M) return COV_EINVAL;
    cost[i] = cov::matrix_cost(d.N, d.M, d.P, d.Q);
  }
  std::vector<int> bin(count);
  std::vector<long long> load(n_ranks);
  cov::lpt_assign(cost.data(), count, n_ranks, bin.data(), load.data());
  for (int i = 0; i < count; ++i) rank_of[i] = bin[i];
  if (rank_cost)
    for (int r = 0; r < n_ranks; ++r) rank_cost[r] = load[r];
  return COV_OK;
}

cov_status cov_aperture_descs(const void *image, cov_dtype dtype, int64_t H, int64_t W, int64_t ld,
                              int ap_n, int ap_m, int step_r, int step_c, int P, int Q, void *R,
                              cov_desc *descs, int max_count, int *count) {
  if (!count || H < 1 || W < 1 || ld < W || ap_n < 1 || ap_m < 1 || ap_n > H || ap_m > W ||
      step_r < 1 || step_c < 1 || P < 1 || Q < 1 || P > ap_n || Q > ap_m || max_count < 0 ||
      (dtype != COV_C64 && dtype != COV_C128))
    return COV_EINVAL;
  const long long nr = (H - ap_n) / step_r + 1, nc = (W - ap_m) / step_c + 1;
  if (nr * nc > (1LL << 30)) return COV_EINVAL;
  *count = (int)(nr * nc);
  if (!descs) return COV_OK;  // size query
  if (!image || !R || max_count < *count) return COV_EINVAL;
  const size_t elem = dtype == COV_C128 ? 16 : 8;
  const size_t rbytes = (size_t)P * Q * P * Q * elem;
  for (long long a = 0; a < nr; ++a)
    for (long long b = 0; b < nc; ++b) {
      const long long k = a * nc + b;
      cov_desc &d = descs[k];
      d.A = (const char *)image + ((size_t)(a * step_r) * ld + (size_t)(b * step_c)) * elem;
      d.R = (char *)R + (size_t)k * rbytes;
      d.lda = ld;
      d.N = ap_n;
      d.M = ap_m;
      d.P = P;
      d.Q = Q;
    }
  return COV_OK;
}

namespace {

// The schedule of the plan's current form: member costs, grid, slots (CTAs,
// or warps of the warp form), LPT assignment, each slot's members in
// decreasing cost order.
void build_schedule(cov_batched_plan *pl) {
  const int count = (int)pl->descs.size();
  std::vector<long long> cost(count);
  for (int i = 0; i < count; ++i) {
    const cov::BDesc &d = pl->descs[i];
    if (pl->form == 1 || pl->form == 2) {
      // the warp and box forms: distinct products plus the per-output-row
      // window sums and, for the box form, the R elements written
      long long steps = 0;  // outputs i of every combination
      for (int dc = 0; dc < d.Q; ++dc)
        for (int dr = dc ? -(d.P - 1) : 0; dr < d.P; ++dr) steps += d.P - (dr < 0 ? -dr : dr);
      const long long DD = (long long)d.P * d.Q;
      cost[i] = pl->form == 1 ? cov::distinct_products(d.N, d.M, d.P, d.Q) / 8 + 40 * steps + 200
                              : cov::distinct_products(d.N, d.M, d.P, d.Q) / 8 + 24 * steps +
                                    DD * DD / 8 + 200;
    } else {
      cost[i] = (long long)batched_member_cost(d.N, d.M, d.P, d.Q);
    }
  }
  // (the warp kernel fits two CTAs an SM: twice the warps to hide latency;
  // the box kernel three CTAs an SM, one member each)
  const int grid = pl->form == 1 ? std::min(2 * pl->sms, (count + cov::kWWarps - 1) / cov::kWWarps)
                   : pl->form == 2 ? std::min(3 * pl->sms, count)
                                   : std::min(pl->sms, count);
  const int slots = pl->form == 1 ? grid * cov::kWWarps : grid;
  std::vector<int> bin(count);
  cov::lpt_assign(cost.data(), count, slots, bin.data(), nullptr);
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    return cost[a] > cost[b] || (cost[a] == cost[b] && a < b);
  });
  std::vector<std::vector<int>> per(slots);
  for (int i : order) per[bin[i]].push_back(i);
  pl->grid = grid;
  pl->order.clear();
  pl->cta_begin.assign(slots + 1, 0);
  for (int c = 0; c < slots; ++c) {
    pl->cta_begin[c + 1] = pl->cta_begin[c] + (int)per[c].size();
    for (int i : per[c]) pl->order.push_back(i);
  }
}

}  // namespace

cov_status cov_batched_plan_create(const cov_desc *descs, int count, cov_dtype dtype, cov_algo algo,
                                   cov_norm norm, cov_batched_plan **plan) {
  if (!descs || count < 1 || !plan || (norm != COV_MEAN && norm != COV_SUM)) return COV_EINVAL;
  if ((dtype != COV_C64 && dtype != COV_C128) || (algo != COV_AUTO && algo != COV_RECURRENCE))
    return COV_EUNSUPPORTED;
  bool cta = dtype == COV_C64;  // every member fits the CTA form (and the warp / box forms' base rule)
  for (int i = 0; i < count; ++i) cta = cta && batched_shape_ok(descs[i]);
  const bool pipe_members = cov::pipe_members_ok(descs, count);
  if (!cta && !pipe_members) return COV_EINVAL;
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    sms = 152;  // no device visible (host-only use): plan for a GB300 (152 SMs)
  }
  cov_batched_plan *pl = new cov_batched_plan();
  pl->mean = norm == COV_MEAN ? 1 : 0;
  pl->sms = sms;
  pl->descs.resize(count);
  bool narrow = true;  // every member small enough for one warp
  bool box = true;     // every member small enough for the box form
  size_t box_smem = 0;
  narrow = narrow && cta;
  box = box && cta;
  for (int i = 0; i < count; ++i) {
    const cov_desc &d = descs[i];
    pl->descs[i] = {(const float2 *)d.A, (float2 *)d.R, d.lda, d.N, d.M, d.P, d.Q};
    narrow = narrow && d.M <= cov::kWMaxM && d.P <= cov::kWMaxPQ && d.Q <= cov::kWMaxPQ &&
             d.N * d.M <= cov::kWMaxElems;
    box = box && d.M <= cov::kXMaxM && d.P <= cov::kXMaxPQ && d.Q <= cov::kXMaxPQ &&
          d.P * d.Q <= cov::kXMaxD && d.N * d.M <= cov::kXMaxElems;
    if (box) box_smem = std::max(box_smem, cov::box_smem_bytes(d.N * d.M, d.P, d.Q));
  }
  pl->cta_ok = cta ? 1 : 0;
  pl->narrow_ok = narrow ? 1 : 0;
  pl->box_ok = box ? 1 : 0;
  pl->box_smem = box ? box_smem : 0;
  pl->L = 0;
  pl->rs_max = cov::kBMaxRS;
  // the tables are laid out for the larger of the two forms' slot counts
  const int max_slots = std::max({std::min(sms, count),
                                  narrow ? std::min(2 * sms, (count + cov::kWWarps - 1) / cov::kWWarps) *
                                               cov::kWWarps
                                         : 0,
                                  box ? std::min(3 * sms, count) : 0});
  size_t off = cov::kWsHeader;
  pl->off_desc = off;
  off = al256(off + sizeof(cov::BDesc) * count);
  pl->off_order = off;
  off = al256(off + sizeof(int) * count);
  pl->off_begin = off;
  off = al256(off + sizeof(int) * (max_slots + 1));
  pl->total = off;
  // the stage form's tables and member regions follow, where offered
  pl->pipe_ok = 0;
  if (pipe_members) {
    cov::pipe_plan_build(pl->pipe, descs, count, dtype == COV_C128 ? 16 : 8, pl->mean, off, sms);
    if (pl->pipe.total <= kPipeMaxWorkspace || !cta) {
      pl->pipe_ok = 1;
      pl->total = pl->pipe.total;
    } else {
      pl->pipe = cov::PipePlan();
    }
  }
  if (!cta && !pl->pipe_ok) {
    delete pl;
    return COV_EINVAL;
  }
  // defaults (cov_batched_autotune times the alternatives): the box and warp
  // forms for small members, else the stage form (faster than the CTA form
  // on the 4096-member uneven batch: 4.56 ms against 5.22 ms)
  pl->form = pl->box_ok ? 2 : pl->narrow_ok ? 1 : pl->pipe_ok ? 3 : 0;
  build_schedule(pl);
  *plan = pl;
  return COV_OK;
}

cov_status cov_batched_workspace_size(const cov_batched_plan *plan, size_t *bytes) {
  if (!plan || !bytes) return COV_EINVAL;
  *bytes = plan->total;
  return COV_OK;
}

// COV_OK when the current device has the SM count the plan's schedule was
// balanced for; COV_EUNSUPPORTED on another device (re-create the plan there).
static cov_status plan_matches_device(const cov_batched_plan *pl) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return COV_ECUDA;
  }
  return sms == pl->sms ? COV_OK : COV_EUNSUPPORTED;
}

cov_status cov_batched_upload(const cov_batched_plan *plan, void *workspace, size_t ws_bytes,
                              cov_stream_t stream) {
  if (!plan || !workspace) return COV_EINVAL;
  if (ws_bytes < plan->total || ((uintptr_t)workspace & 255) != 0) return COV_EWORKSPACE;
  const cov_status dst = plan_matches_device(plan);
  if (dst != COV_OK) return dst;
  cudaStream_t s = (cudaStream_t)stream;
  char *w = (char *)workspace;
  if (cudaMemcpyAsync(w + plan->off_desc, plan->descs.data(), sizeof(cov::BDesc) * plan->descs.size(),
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(w + plan->off_order, plan->order.data(), sizeof(int) * plan->order.size(),
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(w + plan->off_begin, plan->cta_begin.data(), sizeof(int) * plan->cta_begin.size(),
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return COV_ECUDA;
  if (plan->pipe_ok && cov::pipe_upload(plan->pipe, w, s) != cudaSuccess) return COV_ECUDA;
  // pageable host memory: make sure the copies have read it before returning
  if (cudaStreamSynchronize(s) != cudaSuccess) return COV_ECUDA;
  return COV_OK;
}

cov_status cov_estimate_batched(const cov_batched_plan *plan, void *workspace, size_t ws_bytes,
                                cov_stream_t stream) {
  if (!plan || !workspace) return COV_EINVAL;
  if (ws_bytes < plan->total || ((uintptr_t)workspace & 255) != 0) return COV_EWORKSPACE;
  const cov_status dst = plan_matches_device(plan);
  if (dst != COV_OK) return dst;
  cudaStream_t s = (cudaStream_t)stream;
  char *w = (char *)workspace;
  // the status word, and the stage form's chunk counters (header words 1..4)
  if (cudaMemsetAsync(w, 0, plan->form == 3 ? 32 : 4, s) != cudaSuccess) return COV_ECUDA;
  if (plan->form == 3)
    return cov::pipe_launch(plan->pipe, w, plan->sms, s) == cudaSuccess ? COV_OK : COV_ECUDA;
  const size_t smem = cov::kBSmemBytes;
  if (cov::ensure_dyn_smem((const void *)cov::k_batched, smem, false) != cudaSuccess)
    return COV_ECUDA;
  if (plan->form == 2) {
    if (cov::ensure_dyn_smem((const void *)cov::k_batched_box, plan->box_smem, false) != cudaSuccess)
      return COV_ECUDA;
    cov::k_batched_box<<<plan->grid, cov::kXWarps * 32, plan->box_smem, s>>>(
        (const cov::BDesc *)(w + plan->off_desc), (const int *)(w + plan->off_order),
        (const int *)(w + plan->off_begin), plan->mean);
    return cudaGetLastError() == cudaSuccess ? COV_OK : COV_ECUDA;
  }
  if (plan->form == 1) {
    const size_t wsmem = cov::kWWarps * cov::kWWarpBytes;
    if (cov::ensure_dyn_smem((const void *)cov::k_batched_warp, wsmem, false) != cudaSuccess)
      return COV_ECUDA;
    cov::k_batched_warp<<<plan->grid, cov::kWWarps * 32, wsmem, s>>>(
        (const cov::BDesc *)(w + plan->off_desc), (const int *)(w + plan->off_order),
        (const int *)(w + plan->off_begin), plan->mean);
    return cudaGetLastError() == cudaSuccess ? COV_OK : COV_ECUDA;
  }
  cov::k_batched<<<plan->grid, cov::kBWarps * 32, smem, s>>>(
      (const cov::BDesc *)(w + plan->off_desc), (const int *)(w + plan->off_order),
      (const int *)(w + plan->off_begin), plan->mean, plan->L, plan->rs_max);
  return cudaGetLastError() == cudaSuccess ? COV_OK : COV_ECUDA;
}

void cov_batched_plan_destroy(cov_batched_plan *plan) { delete plan; }

cov_status cov_batched_get_tuning(const cov_batched_plan *plan, cov_batched_tuning_t *t) {
  if (!plan || !t) return COV_EINVAL;
  t->form = plan->form;
  t->reseed_interval = plan->L;
  t->row_ranges = plan->rs_max;
  return COV_OK;
}

cov_status cov_batched_set_tuning(cov_batched_plan *plan, const cov_batched_tuning_t *t) {
  if (!plan || !t) return COV_EINVAL;
  if (t->form < 0 || t->form > 3 || (t->form == 0 && !plan->cta_ok) ||
      (t->form == 1 && !plan->narrow_ok) || (t->form == 2 && !plan->box_ok) ||
      (t->form == 3 && !plan->pipe_ok))
    return COV_EINVAL;
  if (t->reseed_interval < 0 || t->reseed_interval > cov::kBMaxPQ) return COV_EINVAL;
  if (t->row_ranges != 1 && t->row_ranges != 2 && t->row_ranges != 4) return COV_EINVAL;
  const bool rebuild = t->form != plan->form;
  plan->form = t->form;
  plan->L = t->reseed_interval;
  plan->rs_max = t->row_ranges;
  if (rebuild) build_schedule(plan);
  return COV_OK;
}

cov_status cov_batched_autotune(cov_batched_plan *plan, void *workspace, size_t ws_bytes, int reps,
                                cov_stream_t stream) {
  if (!plan || !workspace || reps < 1) return COV_EINVAL;
  if (ws_bytes < plan->total || ((uintptr_t)workspace & 255) != 0) return COV_EWORKSPACE;
  const cov_status dst = plan_matches_device(plan);
  if (dst != COV_OK) return dst;
  cudaStream_t s = (cudaStream_t)stream;
  // candidates: the box and warp forms where every member fits them; the CTA
  // form with segments of the whole diagonal or of 2 or 4 outputs, and 2 or
  // 4 row ranges
  std::vector<cov_batched_tuning_t> cand;
  if (plan->box_ok) cand.push_back({2, 0, cov::kBMaxRS});
  if (plan->narrow_ok) cand.push_back({1, 0, cov::kBMaxRS});
  if (plan->pipe_ok) cand.push_back({3, 0, cov::kBMaxRS});
  if (plan->cta_ok)
    for (int L : {0, 2, 4})
      for (int rs : {2, 4}) cand.push_back({0, L, rs});
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return COV_ECUDA;
  }
  cov_status st = COV_OK;
  float best_ms = 0.f;
  cov_batched_tuning_t best = cand[0];
  for (size_t k = 0; k < cand.size() && st == COV_OK; ++k) {
    if ((st = cov_batched_set_tuning(plan, &cand[k])) != COV_OK) break;
    if ((st = cov_batched_upload(plan, workspace, ws_bytes, stream)) != COV_OK) break;
    if ((st = cov_estimate_batched(plan, workspace, ws_bytes, stream)) != COV_OK) break;  // warm-up
    if (cudaEventRecord(e0, s) != cudaSuccess) { st = COV_ECUDA; break; }
    for (int r = 0; r < reps && st == COV_OK; ++r) st = cov_estimate_batched(plan, workspace, ws_bytes, stream);
    if (st != COV_OK) break;
    float ms = 0.f;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = COV_ECUDA;
      break;
    }
    if (k == 0 || ms < best_ms) {
      best_ms = ms;
      best = cand[k];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != COV_OK) return st;
  if ((st = cov_batched_set_tuning(plan, &best)) != COV_OK) return st;
  return cov_batched_upload(plan, workspace, ws_bytes, stream);
}

}  // extern "C"
