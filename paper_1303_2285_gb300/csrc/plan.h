// Host plan layer (integer only, no CUDA calls): combination counts, lag
// groups, tiles and the workspace layout of the combination path.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "cov_internal.h"

namespace cov {

struct WsLayout {
  size_t core_off, colsum_off, sin_off, rowval_off, colval_off, total;
};

// Number of window positions, |UC| and UM for an N x M input, P x Q window
// (Eq. 3.4-3.6 with mu = (N-|dr|)(M-|dc|)).
long long n_positions(long long N, long long M, int P, int Q);
long long n_unique_combinations(int P, int Q);
long long distinct_products(long long N, long long M, int P, int Q);

// True if the combination path takes the shape (N >= 2P-1, M >= 2Q-1,
// 1 <= P, Q <= kMaxPQ).
bool recurrence_ok(long long N, long long M, int P, int Q);

// Lags per group: the largest of 16, 8, 4 (8, 4 for FP64) whose unused
// slots stay within 2% of the fewest.
int choose_group(int P, int Q, int elem);

// Tuned knobs of the combination path (0 = the plan's default): lags per
// group G, rows per product task TRB, walk re-seed interval L, kernels per
// call K (1 = the fused cooperative kernel, FP32 only; 4 = four kernels),
// columns per shared-memory tile TC (32 or 64), inner columns per fringe-row
// chunk CWF (a multiple of 8 up to 256; not a public knob: the batched stage
// form widens it for small members).
struct Tuning {
  int G, TRB, L, K, TC, CWF;
};

// Fills every field of p that depends on the shape only (not the pointers);
// returns the workspace layout. elem = bytes of one complex number. `tune`
// overrides the knobs; when null, the cached tuning for (elem, shape, sms),
// if any, is used, else the defaults.
void plan_recurrence(long long N, long long M, long long lda, int P, int Q, int elem, int sms,
                     RecParams &p, WsLayout &ws, const Tuning *tune = nullptr);

// Restricts a plan to the column lags [dc_lo, dc_hi) (one shard).
void restrict_to_lags(RecParams &p, int dc_lo, int dc_hi);

// Splits the column lags [0, Q) into n_ranks contiguous ranges (dc_begin has
// n_ranks + 1 entries) minimising the largest per-rank cost; rank_cost
// (optional) receives each rank's cost.
void partition_lags(long long N, long long M, int P, int Q, int n_ranks, int *dc_begin,
                    long long *rank_cost);

// Scheduling cost of one matrix (distinct products plus per-combination and
// per-matrix overheads) and the longest-processing-time-first assignment of
// `count` items to `n_bins` bins (bin[i] per item; load per bin, optional).
long long matrix_cost(long long N, long long M, int P, int Q);
void lpt_assign(const long long *cost, int count, int n_bins, int *bin, long long *load);

// Process-wide cache of tuned knobs, keyed by (elem, N, M, P, Q, SM count).
bool lookup_tuning(int elem, long long N, long long M, int P, int Q, int sms, Tuning &out);
void store_tuning(int elem, long long N, long long M, int P, int Q, int sms,
                  const Tuning *t);  // t == null removes the entry
void clear_tuning();
int save_tuning(const char *path);  // 0 on success, -1 on error
int load_tuning(const char *path);  // entries read, -1 on a malformed file

}  // namespace cov
