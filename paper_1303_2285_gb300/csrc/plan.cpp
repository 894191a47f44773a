// Host plan layer of the combination path (integer arithmetic only).
#include "plan.h"

#include <string.h>

namespace cov {

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

long long n_positions(long long N, long long M, int P, int Q) {
  return (N - P + 1) * (M - Q + 1);
}

long long n_unique_combinations(int P, int Q) {
  return (long long)P * Q + (long long)(P - 1) * (Q - 1);
}

long long distinct_products(long long N, long long M, int P, int Q) {
  long long um = 0;
  for (int dc = 0; dc < Q; ++dc) {
    const int lo = dc == 0 ? 0 : -(P - 1);
    for (int dr = lo; dr <= P - 1; ++dr) um += (N - (dr < 0 ? -dr : dr)) * (M - dc);
  }
  return um;
}

bool recurrence_ok(long long N, long long M, int P, int Q) {
  return P >= 1 && Q >= 1 && P <= kMaxPQ && Q <= kMaxPQ && N >= 2LL * P - 1 &&
         M >= 2LL * Q - 1 && N < (1LL << 30) && M < (1LL << 30);
}

int choose_group(int P, int Q) {
  const int cand[3] = {16, 8, 4};
  const double uc = (double)n_unique_combinations(P, Q);
  double waste[3], best = 1e30;
  for (int k = 0; k < 3; ++k) {
    waste[k] = (double)n_groups(P, Q, cand[k]) * cand[k] / uc - 1.0;
    if (waste[k] < best) best = waste[k];
  }
  for (int k = 0; k < 3; ++k)
    if (waste[k] <= best + 0.02) return cand[k];
  return 4;
}

void plan_recurrence(long long N, long long M, long long lda, int P, int Q, int elem,
                     RecParams &p, WsLayout &ws) {
  memset(&p, 0, sizeof(p));
  p.N = (int)N;
  p.M = (int)M;
  p.P = P;
  p.Q = Q;
  p.lda = lda;
  p.K = n_positions(N, M, P, Q);
  p.n_uc = (int)n_unique_combinations(P, Q);
  p.G = choose_group(P, Q);
  p.ngroups = n_groups(P, Q, p.G);
  p.inner_lo = P - 1;
  p.n_inner = (int)(N - 2LL * P + 2);
  p.d_lo = group_lag_lo(P, Q);
  p.d_hi = group_lag_hi(P, Q, p.G);
  const int span = p.d_hi - p.d_lo;
  p.TC = M >= 64 ? 64 : 32;
  p.CBT = p.TC / 32;
  p.STC = p.TC + Q - 1;
  p.STC += p.STC & 1;
  p.n_cb = (int)((M + 31) / 32);
  p.n_ct = (int)((M + p.TC - 1) / p.TC);
  // Tile rows: two buffers of at most `budget` bytes each; prefer a budget
  // that leaves room for two CTAs per SM when the tile is not too short.
  const int R = 8;
  const long long row_bytes = (long long)p.STC * elem;
  long long budget = 56 * 1024;
  long long tr_max = budget / row_bytes - span;
  if (tr_max < 48) {
    budget = 110 * 1024;
    tr_max = budget / row_bytes - span;
  }
  if (tr_max < R) tr_max = R;  // shapes this large in Q are rejected earlier
  if (tr_max > 128) tr_max = 128;
  int n_rt = (int)((p.n_inner + tr_max - 1) / tr_max);
  if (n_rt < 1) n_rt = 1;
  int TR = 0;
  for (;; ++n_rt) {
    const int per = (p.n_inner + n_rt - 1) / n_rt;
    TR = ((per + R - 1) / R) * R;
    if (TR <= tr_max || TR <= R) break;
  }
  p.TR = TR;
  p.n_rt = (p.n_inner + TR - 1) / TR;
  p.STR = TR + span;
  p.tasks_per_tile = (long long)p.ngroups * p.CBT;
  p.n_tasks = (long long)p.n_rt * p.n_ct * p.tasks_per_tile;
  // fringe rows
  p.NFR = 2 * (P - 1);
  p.NFC = 2 * (Q - 1);
  p.GF = 8;
  p.RB = 4;
  p.ngroups_f = n_groups(P, Q, p.GF);
  p.nrb = (P - 1 + p.RB - 1) / p.RB;
  p.L = 8;
  p.div_double = (elem == 8 && p.K > (1LL << 24)) ? 1 : 0;
  // workspace
  size_t off = kWsHeader;
  ws.core_off = off;
  off = align256(off + (size_t)p.n_uc * p.n_rt * p.n_cb * elem);
  ws.colsum_off = off;
  off = align256(off + (size_t)p.n_uc * p.NFC * p.n_rt * elem);
  ws.rowval_off = off;
  off = align256(off + (size_t)p.n_uc * Q * p.NFR * elem);
  ws.colval_off = off;
  off = align256(off + (size_t)p.n_uc * Q * elem);
  ws.total = off;
}

}  // namespace cov
