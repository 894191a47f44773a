// Host plan layer of the combination path (integer arithmetic only).
#include "plan.h"

#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <mutex>
#include <queue>
#include <utility>
#include <vector>

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
  return P >= 1 && Q >= 1 && P <= kMaxPQ && Q <= kMaxPQ && N >= P && M >= Q &&
         N < (1LL << 30) && M < (1LL << 30);
}

int choose_group(int P, int Q, int elem) {
  const int cand[3] = {16, 8, 4};
  const int first = elem > 8 ? 1 : 0;  // FP64: at most 8 lags (registers)
  const double uc = (double)n_unique_combinations(P, Q);
  double waste[3], best = 1e30;
  for (int k = first; k < 3; ++k) {
    waste[k] = (double)n_groups(P, Q, cand[k]) * cand[k] / uc - 1.0;
    if (waste[k] < best) best = waste[k];
  }
  for (int k = first; k < 3; ++k)
    if (waste[k] <= best + 0.02) return cand[k];
  return 4;
}

void plan_recurrence(long long N, long long M, long long lda, int P, int Q, int elem, int sms,
                     RecParams &p, WsLayout &ws, const Tuning *tune) {
  Tuning t = {0, 0, 0, 0, 0, 0};
  if (tune) t = *tune;
  else lookup_tuning(elem, N, M, P, Q, sms, t);
  memset(&p, 0, sizeof(p));
  p.N = (int)N;
  p.M = (int)M;
  p.P = P;
  p.Q = Q;
  p.lda = lda;
  p.K = n_positions(N, M, P, Q);
  p.n_uc = (int)n_unique_combinations(P, Q);
  p.G = choose_group(P, Q, elem);
  if (t.G == 4 || t.G == 8 || (t.G == 16 && elem == 8)) p.G = t.G;
  p.ngroups = n_groups(P, Q, p.G);
  p.inner_lo = P - 1;
  // inner rows / columns (none where N < 2P-1 / M < 2Q-1), the fringe rows
  // and columns, and how many of them one box holds
  p.n_inner = N >= 2LL * P - 1 ? (int)(N - 2LL * P + 2) : 0;
  p.n_innerc = M >= 2LL * Q - 1 ? (int)(M - 2LL * Q + 2) : 0;
  p.NFR = (int)(N - p.n_inner);
  p.NFC = (int)(M - p.n_innerc);
  p.H = (int)(N - P + 1 - p.n_inner);
  p.HC = (int)(M - Q + 1 - p.n_innerc);
  p.d_lo = group_lag_lo(P, Q);
  p.d_hi = group_lag_hi(P, Q, p.G);
  const int span = p.d_hi - p.d_lo;
  // Tiles: TC = 64 or 32 columns (each a 32-column block a warp task
  // covers), smem pitch TC + 16 (Q <= 17) or TC + 32 (Q <= 33) complex
  // elements (the partner columns of every column lag); two buffers of STR
  // rows each within the 227 KB of a CTA. A narrower tile holds more rows,
  // so a task's row block (and each partial sum) covers more rows: the
  // default is 32 columns where a 64-column tile would hold fewer than 96
  // rows besides its halo.
  const long long buf_bytes = (232448LL - 1024) / 2;
  auto rows_for = [&](int tc) {
    const int pitch = tc + (Q <= 17 ? 16 : 32);
    long long rm = buf_bytes / ((long long)pitch * elem);
    if (rm > 256) rm = 256;  // TMA box height
    return rm - span;
  };
  p.TC = (t.TC == 32 || t.TC == 64) ? t.TC : (rows_for(64) < 96 ? 32 : 64);
  p.CBT = p.TC / 32;
  p.PITCH = p.TC + (Q <= 17 ? 16 : 32);
  p.n_cb = (int)((M + 31) / 32);
  p.n_ct = (int)((M + p.TC - 1) / p.TC);
  long long tr_max = rows_for(p.TC);
  if (tr_max < 8) tr_max = 8;
  // FP32: the longest row block up to 128 rows (fewer partial sums and task
  // epilogues), shortened while the tasks (about row blocks x column blocks x
  // lag groups) number fewer than 8 per SM; FP64: 48 rows, shortened until
  // the tasks cover twice the SMs (one SM's FP64 pipe is slow, so every SM
  // needs a task)
  const long long trb_cap = elem == 8 ? 128 : 48;
  int TRB = (int)((tr_max < trb_cap ? tr_max : trb_cap) / 8) * 8;
  if (sms > 0) {
    const long long per_rb = (long long)((M + 31) / 32) * p.ngroups;
    const long long want = elem == 8 ? 8LL * sms : 2LL * sms;
    const int floor_rows = elem == 8 ? 16 : 8;
    while (TRB > floor_rows && (long long)((p.n_inner + TRB - 1) / TRB) * per_rb < want) TRB -= 8;
  }
  // no longer than the inner rows (rounded up to 8): a longer block only
  // stages rows no task reads
  const int inner8 = ((p.n_inner + 7) / 8) * 8;
  if (inner8 >= 8 && TRB > inner8) TRB = inner8;
  if (t.TRB >= 8 && t.TRB % 8 == 0 && t.TRB <= tr_max) TRB = t.TRB;
  if (TRB < 8) TRB = 8;
  int TPT = (int)(tr_max / TRB);
  if (TPT > 4) TPT = 4;
  p.TRB = TRB;
  p.n_rb = (p.n_inner + TRB - 1) / TRB;  // 0 without inner rows: no product tasks
  if (TPT > p.n_rb) TPT = p.n_rb;
  if (TPT < 1) TPT = 1;
  p.TPT = TPT;
  p.TR = TRB * TPT;
  p.n_rt = (p.n_rb + TPT - 1) / TPT;
  p.STR = p.TR + span;
  p.tasks_per_tile = (long long)p.ngroups * p.CBT * p.TPT;
  p.n_tasks = (long long)p.n_rt * p.n_ct * p.tasks_per_tile;
  // fringe rows (NFR, NFC set above)
  p.GF = 8;
  p.RB = 4;
  p.ngroups_f = n_groups(P, Q, p.GF);
  p.nrb = (P - 1 + p.RB - 1) / p.RB;
  p.CWF = elem == 16 ? 8 : 32;
  if (t.CWF >= 8 && t.CWF <= 256 && t.CWF % 8 == 0) p.CWF = t.CWF;
  p.FPB = elem == 16 ? 32 : 256;
  p.NCH = (p.n_innerc + p.CWF - 1) / p.CWF;  // 0 without inner columns
  p.QMAXF = Q <= 4 ? 4 : Q <= 8 ? 8 : Q <= 16 ? 16 : 32;
  p.FPITCH = ((p.CWF + p.QMAXF - 1 + 14) / 16) * 16 + 1;  // >= CWF+QMAXF-1, = 1 mod 16
  p.L = (t.L >= 1 && t.L <= kMaxPQ) ? t.L : 8;
  // FP32: one fused kernel by default where the reductions are small (they
  // run with one CTA per SM there); four kernels otherwise
  p.fused = elem == 8 && (t.K == 1 || (t.K == 0 && (long long)p.n_uc * p.NFR <= 32768)) ? 1 : 0;
  p.dc_lo = 0;
  p.dc_hi = Q;
  p.g_lo = 0;
  p.u_lo = 0;
  p.u_hi = p.n_uc;
  p.div_double = (elem == 8 && p.K > (1LL << 24)) ? 1 : 0;
  // workspace
  size_t off = kWsHeader;
  ws.core_off = off;
  off = align256(off + (size_t)p.n_uc * p.n_rb * p.n_cb * elem);
  ws.colsum_off = off;
  off = align256(off + (size_t)p.n_uc * p.NFC * p.n_rb * elem);
  ws.sin_off = off;
  off = align256(off + (size_t)p.n_uc * p.NFR * p.NCH * elem);
  ws.rowval_off = off;
  off = align256(off + (size_t)p.n_uc * Q * p.NFR * elem);
  ws.colval_off = off;
  off = align256(off + (size_t)p.n_uc * Q * elem);
  ws.total = off;
}

void restrict_to_lags(RecParams &p, int dc_lo, int dc_hi) {
  p.dc_lo = dc_lo;
  p.dc_hi = dc_hi;
  p.g_lo = first_group(p.P, p.G, dc_lo);
  p.ngroups = first_group(p.P, p.G, dc_hi) - p.g_lo;
  p.u_lo = first_combo(p.P, dc_lo);
  p.u_hi = first_combo(p.P, dc_hi);
  p.tasks_per_tile = (long long)p.ngroups * p.CBT * p.TPT;
  p.n_tasks = (long long)p.n_rt * p.n_ct * p.tasks_per_tile;
}

// cost of the combinations of column lag dc: their distinct products plus a
// per-combination share of the reduction and walk
static long long lag_cost(long long N, long long M, int P, int dc) {
  long long c = 0;
  const int lo = dc == 0 ? 0 : -(P - 1);
  for (int dr = lo; dr <= P - 1; ++dr) c += (N - (dr < 0 ? -dr : dr)) * (M - dc) + 2000;
  return c;
}

void partition_lags(long long N, long long M, int P, int Q, int n_ranks, int *dc_begin,
                    long long *rank_cost) {
  // contiguous ranges of dc minimising the largest rank cost (exact DP over
  // the Q lags; ties go to the earlier split)
  std::vector<long long> pre(Q + 1, 0);
  for (int dc = 0; dc < Q; ++dc) pre[dc + 1] = pre[dc] + lag_cost(N, M, P, dc);
  const int R = n_ranks;
  const long long INF = (long long)1 << 62;
  // best[r][k]: smallest max cost placing lags [0, k) on ranks [0, r)
  std::vector<long long> best((size_t)(R + 1) * (Q + 1), INF);
  std::vector<int> cut((size_t)(R + 1) * (Q + 1), 0);
  best[0] = 0;
  for (int r = 1; r <= R; ++r)
    for (int k = 0; k <= Q; ++k)
      for (int j = 0; j <= k; ++j) {
        const long long prev = best[(size_t)(r - 1) * (Q + 1) + j];
        if (prev >= INF) continue;
        const long long seg = pre[k] - pre[j];
        const long long v = prev > seg ? prev : seg;
        if (v < best[(size_t)r * (Q + 1) + k]) {
          best[(size_t)r * (Q + 1) + k] = v;
          cut[(size_t)r * (Q + 1) + k] = j;
        }
      }
  dc_begin[R] = Q;
  int k = Q;
  for (int r = R; r >= 1; --r) {
    const int j = cut[(size_t)r * (Q + 1) + k];
    dc_begin[r - 1] = j;
    k = j;
  }
  dc_begin[0] = 0;
  if (rank_cost)
    for (int r = 0; r < R; ++r) rank_cost[r] = pre[dc_begin[r + 1]] - pre[dc_begin[r]];
}

long long matrix_cost(long long N, long long M, int P, int Q) {
  return distinct_products(N, M, P, Q) + 2000LL * n_unique_combinations(P, Q) + 20000;
}

void lpt_assign(const long long *cost, int count, int n_bins, int *bin, long long *load) {
  // longest processing time first: the costliest item to the least-loaded
  // bin (ties: lower item index first, lower bin index first)
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    return cost[a] > cost[b] || (cost[a] == cost[b] && a < b);
  });
  std::priority_queue<std::pair<long long, int>, std::vector<std::pair<long long, int>>,
                      std::greater<std::pair<long long, int>>> q;
  for (int c = 0; c < n_bins; ++c) q.push({0, c});
  std::vector<long long> l(n_bins, 0);
  for (int i : order) {
    const auto top = q.top();
    q.pop();
    bin[i] = top.second;
    l[top.second] = top.first + cost[i];
    q.push({l[top.second], top.second});
  }
  if (load)
    for (int c = 0; c < n_bins; ++c) load[c] = l[c];
}

// ---- tuned knobs: process-wide cache ---------------------------------------
namespace {
struct TuneEntry {
  int elem;
  long long N, M;
  int P, Q, sms;
  Tuning t;
};
std::mutex g_tune_mutex;
std::vector<TuneEntry> g_tune;
}  // namespace

bool lookup_tuning(int elem, long long N, long long M, int P, int Q, int sms, Tuning &out) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  for (const TuneEntry &e : g_tune)
    if (e.elem == elem && e.N == N && e.M == M && e.P == P && e.Q == Q && e.sms == sms) {
      out = e.t;
      return true;
    }
  return false;
}

void store_tuning(int elem, long long N, long long M, int P, int Q, int sms, const Tuning *t) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  for (size_t k = 0; k < g_tune.size(); ++k) {
    TuneEntry &e = g_tune[k];
    if (e.elem == elem && e.N == N && e.M == M && e.P == P && e.Q == Q && e.sms == sms) {
      if (t) e.t = *t;
      else g_tune.erase(g_tune.begin() + (long)k);
      return;
    }
  }
  if (t) g_tune.push_back({elem, N, M, P, Q, sms, *t});
}

void clear_tuning() {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune.clear();
}

int save_tuning(const char *path) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  FILE *f = fopen(path, "w");
  if (!f) return -1;
  fprintf(f, "# elem N M P Q sms G TRB L K TC\n");
  for (const TuneEntry &e : g_tune)
    fprintf(f, "%d %lld %lld %d %d %d %d %d %d %d %d\n", e.elem, e.N, e.M, e.P, e.Q, e.sms, e.t.G,
            e.t.TRB, e.t.L, e.t.K, e.t.TC);
  return fclose(f) == 0 ? 0 : -1;
}

int load_tuning(const char *path) {
  FILE *f = fopen(path, "r");
  if (!f) return -1;
  char line[256];
  int n = 0;
  while (fgets(line, sizeof(line), f)) {
    if (line[0] == '#') continue;
    int elem, P, Q, sms, G, TRB, L, K, TC = 0;
    long long N, M;
    const int got = sscanf(line, "%d %lld %lld %d %d %d %d %d %d %d %d", &elem, &N, &M, &P, &Q,
                           &sms, &G, &TRB, &L, &K, &TC);
    if (got == 10 || got == 11) {  // files written before the TC knob have 10 fields
      const Tuning t = {G, TRB, L, K, got == 11 ? TC : 0};
      store_tuning(elem, N, M, P, Q, sms, &t);
      ++n;
    } else {
      n = -1;
      break;
    }
  }
  fclose(f);
  return n;
}

}  // namespace cov
