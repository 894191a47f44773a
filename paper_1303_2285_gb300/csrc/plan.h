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

// Fills every field of p that depends on the shape only (not the pointers);
// returns the workspace layout. elem = bytes of one complex number.
void plan_recurrence(long long N, long long M, long long lda, int P, int Q, int elem,
                     RecParams &p, WsLayout &ws);

}  // namespace cov
