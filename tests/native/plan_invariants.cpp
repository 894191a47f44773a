// Host-only invariants of the combination path's plan (plan.cpp), over a
// sweep of shapes (with and without inner rows and columns), element sizes
// and tuned knobs: tiles cover the inner rows
// and all columns; the staged tile holds every partner row and column of its
// tasks and its two buffers fit the shared memory the kernels request; the
// workspace regions are 256-byte aligned, disjoint and large enough for the
// arrays the kernels index; shards by column lag split the lag groups and the
// combinations exactly. Prints one line per violation; exit status = count.
#include <stdio.h>

#include <initializer_list>

#include "plan.h"

using namespace cov;

static int fails = 0;
#define CHECK(cond, ...)                                           \
  do {                                                             \
    if (!(cond)) {                                                 \
      if (fails < 40) {                                            \
        printf("FAIL %s: N=%lld M=%lld P=%d Q=%d elem=%d: ", #cond, N, M, P, Q, elem); \
        printf(__VA_ARGS__);                                       \
        printf("\n");                                              \
      }                                                            \
      ++fails;                                                     \
    }                                                              \
  } while (0)

static void check_plan(long long N, long long M, int P, int Q, int elem, const Tuning *t) {
  RecParams p;
  WsLayout ws;
  plan_recurrence(N, M, M, P, Q, elem, 152, p, ws, t);
  const long long span = p.d_hi - p.d_lo;
  // lag range of the groups: every (dr, dc) of UC and the unused slots
  CHECK(p.d_lo == (Q > 1 ? -(P - 1) : 0), "d_lo %d", p.d_lo);
  CHECK(p.d_hi >= P - 1, "d_hi %d", p.d_hi);
  // row tiling of the inner rows [P-1, N-P]
  CHECK(p.n_inner == (N >= 2 * P - 1 ? N - 2 * P + 2 : 0), "n_inner %d", p.n_inner);
  CHECK(p.n_innerc == (M >= 2 * Q - 1 ? M - 2 * Q + 2 : 0), "n_innerc %d", p.n_innerc);
  // fringe rows / columns and the share of them inside one box
  CHECK(p.NFR == N - p.n_inner && p.NFC == M - p.n_innerc, "NFR/NFC");
  CHECK(p.NFR <= 2 * (P - 1) && p.NFC <= 2 * (Q - 1), "NFR %d NFC %d above the fringe", p.NFR, p.NFC);
  CHECK(p.H == N - P + 1 - p.n_inner && p.HC == M - Q + 1 - p.n_innerc, "H/HC");
  CHECK(p.H >= 0 && p.H <= P - 1 && p.HC >= 0 && p.HC <= Q - 1, "H %d HC %d", p.H, p.HC);
  // the last walk step of the longest segment reads fringe row (P - 2) + H
  CHECK(P == 1 || P - 2 + p.H < p.NFR || p.NFR == 0, "walk reads past the fringe rows");
  CHECK(p.TRB >= 8 && p.TRB % 8 == 0, "TRB %d", p.TRB);
  CHECK((long long)p.n_rb * p.TRB >= p.n_inner && (long long)(p.n_rb - 1) * p.TRB < p.n_inner,
        "n_rb %d", p.n_rb);
  CHECK(p.TPT >= 1 && p.TPT <= 4 && p.TR == p.TRB * p.TPT, "TPT %d", p.TPT);
  CHECK((long long)p.n_rt * p.TPT >= p.n_rb, "n_rt %d", p.n_rt);
  // column tiling: 64- or 32-column tiles of 32-column blocks
  CHECK((p.TC == 64 || p.TC == 32) && p.CBT * 32 == p.TC, "TC %d", p.TC);
  if (t && (t->TC == 32 || t->TC == 64)) CHECK(p.TC == t->TC, "TC %d not the knob's", p.TC);
  CHECK(p.PITCH == p.TC + (Q <= 17 ? 16 : 32), "PITCH %d", p.PITCH);
  CHECK((long long)p.n_ct * p.TC >= M && (long long)p.n_cb * 32 >= M, "n_ct %d", p.n_ct);
  // the staged tile: rows r0 + d_lo .. r0 + TR - 1 + d_hi, columns c0 .. c0 + 63 + (Q - 1)
  CHECK(p.STR == p.TR + span, "STR %d", p.STR);
  CHECK(p.STR <= 256, "STR %d above the TMA box height", p.STR);
  CHECK(p.PITCH >= p.TC + Q - 1, "PITCH %d", p.PITCH);
  // two buffers rounded up to 1 KB each, plus the barriers: within 227 KB
  const long long bb = ((long long)p.STR * p.PITCH * elem + 1023) & ~1023LL;
  CHECK(2 * bb + 64 <= 232448, "tile buffers %lld B", 2 * bb + 64);
  CHECK(p.tasks_per_tile == (long long)p.ngroups * p.CBT * p.TPT, "tasks_per_tile");
  CHECK(p.n_tasks == (long long)p.n_rt * p.n_ct * p.tasks_per_tile, "n_tasks");
  CHECK(p.ngroups == n_groups(P, Q, p.G), "ngroups");
  // fringe-row stage
  CHECK(p.QMAXF >= Q, "QMAXF %d", p.QMAXF);
  CHECK((long long)p.NCH * p.CWF >= p.n_innerc && (p.NCH == 0) == (p.n_innerc == 0), "NCH %d", p.NCH);
  CHECK(p.FPITCH >= p.CWF + p.QMAXF - 1 && p.FPITCH % 16 == 1, "FPITCH %d", p.FPITCH);
  CHECK(p.L >= 1 && p.L <= kMaxPQ, "L %d", p.L);
  CHECK(p.div_double == (elem == 8 && p.K > (1LL << 24) ? 1 : 0), "div_double");
  CHECK(p.fused == 0 || elem == 8, "fused FP64");
  // workspace: aligned, in order, each region as large as its array
  const size_t e = (size_t)elem, uc = (size_t)p.n_uc;
  const size_t offs[5] = {ws.core_off, ws.colsum_off, ws.sin_off, ws.rowval_off, ws.colval_off};
  const size_t need[5] = {uc * p.n_rb * p.n_cb * e, uc * p.n_rb * p.NFC * e, uc * p.NCH * p.NFR * e,
                          uc * Q * p.NFR * e, uc * Q * e};
  CHECK(ws.core_off >= (size_t)kWsHeader, "header");
  for (int k = 0; k < 5; ++k) {
    CHECK(offs[k] % 256 == 0, "region %d misaligned", k);
    const size_t end = offs[k] + need[k];
    CHECK(end <= (k < 4 ? offs[k + 1] : ws.total), "region %d overlaps the next", k);
  }
  // shards by column lag: contiguous ranges split groups and combinations exactly
  for (int nr = 2; nr <= 3 && nr <= Q; ++nr) {
    int g_next = 0, u_next = 0;
    for (int r = 0; r < nr; ++r) {
      const int lo = Q * r / nr, hi = Q * (r + 1) / nr;
      RecParams s = p;
      restrict_to_lags(s, lo, hi);
      CHECK(s.g_lo == g_next && s.u_lo == u_next, "shard %d of %d starts", r, nr);
      g_next = s.g_lo + s.ngroups;
      u_next = s.u_hi;
    }
    CHECK(g_next == n_groups(P, Q, p.G) && u_next == p.n_uc, "shards of %d end", nr);
  }
}

int main() {
  const Tuning knobs[6] = {{4, 16, 2, 4, 0},    {8, 64, 8, 1, 64},   {16, 128, 32, 0, 32},
                           {16, 256, 1, 4, 64}, {16, 160, 4, 4, 32}, {8, 192, 16, 1, 32}};
  long long N = 0, M = 0;
  int P = 0, Q = 0, elem = 0;
  for (P = 1; P <= 32; P += (P < 8 ? 1 : 3))
    for (Q = 1; Q <= 32; Q += (Q < 8 ? 1 : 5))
      for (elem = 8; elem <= 16; elem += 8) {
        // shapes with and without inner rows / columns (N < 2P - 1, M < 2Q - 1)
        const long long sizes[6] = {P, 2LL * P - 2, 2LL * P - 1, 2LL * P + 37, 300, 1024};
        for (long long n : sizes)
          for (long long m : {(long long)Q, 2LL * Q - 2, 2LL * Q - 1, 2LL * Q + 70, 1000LL}) {
            N = n < P ? P : n;
            M = m < Q ? Q : m;
            check_plan(N, M, P, Q, elem, nullptr);
            for (const Tuning &t : knobs) check_plan(N, M, P, Q, elem, &t);
          }
      }
  printf("%d violations\n", fails);
  return fails > 255 ? 255 : fails;
}
