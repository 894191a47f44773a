// Host-side launch entry points of the kernel files (internal).
#pragma once

#include <cuda_runtime.h>

#include "cov_internal.h"

namespace cov {

// Parameters of the plain per-element path (one thread per element of R).
struct DirectParams {
  const void *A;
  void *R;
  long long lda;
  int N, M, P, Q;
  long long K;
  int mean;
};

// Optional events recorded around the four kernels (see cov_set_stage_events).
struct StageEvents {
  cudaEvent_t ev[5];
  bool on;
};

cudaError_t launch_recurrence(const RecParams &p, bool fp64, int num_sms, cudaStream_t s,
                              const StageEvents *events);
cudaError_t launch_direct(const DirectParams &p, bool c128, cudaStream_t s);

}  // namespace cov
