// Internal definitions shared by the host plan layer and the CUDA kernels.
//
// Notation (0-based restatement of Sections 2.2 and 3):
//   A is N x M; window (p, q) holds A[p+i][q+j] at x[i + P*j]   (Eq. 2.1).
//   A combination is Delta = (dr, dc) = (r2 - r1, c2 - c1)      (Eq. 3.1).
//   Unique combinations UC (Eq. 3.3): dc = 0 with dr in [0, P-1], and
//   dc in [1, Q-1] with dr in [-(P-1), P-1].
//   Product image: Pi_D[n][m] = A[n][m] * conj(A[n+dr][m+dc]).
//   Combination D owns the outputs (i, j), i in [max(0,-dr), P-1-max(0,dr)],
//   j in [0, Q-1-dc]  (Eq. 3.7-3.8, Fig. 2): K*R[i+Pj, (i+dr)+P(j+dc)] is the
//   box sum of Pi_D over rows [i, i+N-P] and columns [j, j+M-Q].
//
// Work split used by the kernels (rows; columns are analogous):
//   inner rows  [P-1, N-P]: inside the box of every output of every Delta
//     (n_inner = max(0, N-2P+2) of them);
//   fringe rows: every other row, NFR = N - n_inner of them, in row order
//     (index fr; row n = fr for fr < P-1, else fr + n_inner). A box holds
//     the inner rows and H = N-P+1 - n_inner consecutive fringe rows: the
//     fringe rows fr in [i, i+H) for the box starting at row i. With
//     N >= 2P-1 these are the top rows [i, P-2] and the bottom rows
//     [N-P+1, N-P+i] (H = P-1); with N < 2P-1 there are no inner rows and
//     every row is a fringe row (H = N-P+1).
//   inner cols  [Q-1, M-Q] (n_innerc = max(0, M-2Q+2)); fringe cols fc in
//     [0, NFC), NFC = M - n_innerc, column m = fc for fc < Q-1 else
//     fc + n_innerc; the box of column offset j holds the fringe columns
//     fc in [j, j+HC), HC = M-Q+1 - n_innerc.
//   Kernel 1 (products_inner): inner rows x all columns. For each Delta the
//     sum over (inner rows x inner cols) -> core partials; per fringe column
//     the sum over inner rows -> colsum partials.
//   Kernel 2 (fringe_rows): each fringe row's sums over chunks of the inner
//     columns (partials of S_in[Delta][fr]).
//   Kernel 3 (reduce): CV[Delta][j] = sum over inner rows of the box-row sums
//     at column offset j (core + fringe-column sums), and the box-row sums
//     RV[Delta][j][fr] = sum_{m in [j, j+M-Q]} Pi_D[n][m] of each fringe row
//     (S_in plus the row's own fringe-column products).
//   Kernel 4 (walk_write): per output block, seed each diagonal segment with
//     the direct sum CV + sum of RV over the H fringe rows inside the box,
//     walk down the diagonal by subtracting the leaving row fr = i and adding
//     the entering row fr = i + H (re-seeding every L steps), divide by K and
//     write the block and its conjugate mirror with coalesced stores.
//   Without inner rows the product kernel has no work (CV = 0); without
//   inner columns the fringe-row kernel has none (S_in = 0) and the box sums
//   over the fringe columns are direct window sums instead of the suffix /
//   prefix scans used when the box holds Q-1 of them.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define COV_HD __host__ __device__ __forceinline__
#else
#define COV_HD inline
#endif

namespace cov {

constexpr int kMaxPQ = 32;       // recurrence path: P, Q <= 32 (smem tile fits)

constexpr int kWsHeader = 256;   // status word + padding at the workspace head

// Status codes written by kernels into the workspace status word.
constexpr unsigned kDevOk = 0;
constexpr unsigned kDevTimeout = 4;
constexpr unsigned kDevCheck = 6;

// Index of combination (dr, dc) in [0, |UC|): dc = 0 first (dr = 0..P-1),
// then each dc >= 1 with dr = -(P-1)..P-1.
COV_HD int combo_index(int P, int dr, int dc) {
  return dc == 0 ? dr : P + (dc - 1) * (2 * P - 1) + (dr + P - 1);
}

COV_HD void combo_of(int P, int idx, int &dr, int &dc) {
  if (idx < P) {
    dr = idx;
    dc = 0;
  } else {
    const int k = idx - P;
    dc = 1 + k / (2 * P - 1);
    dr = k % (2 * P - 1) - (P - 1);
  }
}

// Fringe row fr -> row of A, fringe column fc -> column of A.
COV_HD int fringe_row(int P, int n_inner, int fr) { return fr < P - 1 ? fr : fr + n_inner; }
COV_HD int fringe_col(int Q, int n_innerc, int fc) { return fc < Q - 1 ? fc : fc + n_innerc; }

// Lag groups: consecutive dr values of one dc, G per group. Group g gives
// (dc, d0, cnt): lags dr = d0 .. d0+cnt-1 (cnt <= G). The G - cnt unused
// slots of the last group of each dc form products that are never used
// (their accumulators are dropped); the smem halo covers their rows.
COV_HD int groups_dc0(int P, int G) { return (P + G - 1) / G; }
COV_HD int groups_per_dc(int P, int G) { return (2 * P - 1 + G - 1) / G; }
COV_HD int n_groups(int P, int Q, int G) {
  return groups_dc0(P, G) + (Q - 1) * groups_per_dc(P, G);
}
COV_HD void group_of(int P, int G, int g, int &dc, int &d0, int &cnt) {
  const int g0 = groups_dc0(P, G);
  if (g < g0) {
    dc = 0;
    d0 = g * G;
  } else {
    const int gp = g - g0, gpc = groups_per_dc(P, G);
    dc = 1 + gp / gpc;
    d0 = -(P - 1) + (gp % gpc) * G;
  }
  const int c = P - d0;  // lags up to dr = P-1
  cnt = c < G ? c : G;
}
// First lag group and first combination of column lag dc (dc <= Q gives the
// end of the range).
COV_HD int first_group(int P, int G, int dc) {
  return dc == 0 ? 0 : groups_dc0(P, G) + (dc - 1) * groups_per_dc(P, G);
}
COV_HD int first_combo(int P, int dc) { return dc == 0 ? 0 : P + (dc - 1) * (2 * P - 1); }
// Largest lag (including unused slots) over all groups.
COV_HD int group_lag_hi(int P, int Q, int G) {
  int hi = groups_dc0(P, G) * G - 1;
  if (Q > 1) {
    const int h2 = -(P - 1) + groups_per_dc(P, G) * G - 1;
    hi = h2 > hi ? h2 : hi;
  }
  return hi;
}
COV_HD int group_lag_lo(int P, int Q) { return Q > 1 ? -(P - 1) : 0; }

// Everything a kernel of the recurrence path needs about one problem.
// Sizes are int32 (N, M < 2^31); element offsets are int64.
struct RecParams {
  const void *A;
  void *R;
  long long lda;  // complex elements
  int N, M, P, Q;
  long long K;
  int mean;
  int div_double;  // divide by K in double (FP32 path, K > 2^24)
  int n_uc;
  // product kernel (inner rows)
  int G;                // lags per group
  int ngroups;
  int inner_lo;         // P-1
  int n_inner;          // max(0, N-2P+2) inner rows
  int n_innerc;         // max(0, M-2Q+2) inner columns
  int H, HC;            // fringe rows / fringe columns inside one box
  int TRB;              // rows per warp task (one partial row block)
  int TPT;              // row blocks per smem tile
  int TR, TC, CBT;      // tile rows (TRB*TPT), tile cols (64), 32-col blocks per tile
  int n_rb;             // row blocks over the inner rows
  int n_rt, n_ct, n_cb; // row tiles, col tiles, 32-col blocks over [0, M)
  int d_lo, d_hi;       // lag range covered by the smem tile
  int STR, PITCH;       // smem tile rows and pitch (complex elements; 80 or 96)
  int use_tma;          // stage tiles with TMA (set at launch)
  long long tasks_per_tile, n_tasks;
  // fringe-row kernel
  int NFR, NFC;         // N - n_inner, M - n_innerc (2(P-1), 2(Q-1) when both >= 0)
  int GF, ngroups_f, RB, nrb;
  int CWF, NCH;         // inner-column chunk width and count of the fringe-row kernel
  int FPB;              // its (fringe row, row lag) pairs per CTA (= threads)
  int QMAXF, FPITCH;    // its column-lag register count (>= Q) and smem pitch
  // walk
  int L;                // re-seed interval along the diagonal
  int fused;            // FP32: run the four stages as one cooperative kernel
  // shard: the column lags dc in [dc_lo, dc_hi) (the R blocks (a, b) with
  // |b - a| in that range); lag groups [g_lo, g_lo + ngroups) and
  // combinations [u_lo, u_hi) are theirs. The full problem is [0, Q).
  int dc_lo, dc_hi, g_lo, u_lo, u_hi;
  // workspace
  unsigned *status;
  void *core_part;      // [n_uc][n_rb][n_cb]
  void *colsum_part;    // [n_uc][n_rb][NFC]
  void *sin_part;       // [n_uc][NCH][NFR]
  void *rowval;         // [n_uc][Q][NFR]
  void *colval;         // [n_uc][Q]
};

}  // namespace cov
