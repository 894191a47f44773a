// Host-side launch entry points of the kernel files (internal).
#pragma once

#include <cuda.h>
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

// Optional events recorded around the four kernels (see cov_set_stage_events):
// call number c uses ev[5*(c % rounds) .. 5*(c % rounds)+4].
struct StageEvents {
  cudaEvent_t *ev;
  int rounds;
  long long calls;
  bool on;
};

cudaError_t launch_recurrence(const RecParams &p, bool fp64, int num_sms, cudaStream_t s,
                              StageEvents *events);

// The four kernels of the combination path (rec_products.cu, rec_fringe.cu,
// rec_reduce.cu). `pdl`: launch with programmatic stream serialization.
cudaError_t launch_products_any(const RecParams &p, const CUtensorMap &tmap, bool fp64, int num_sms,
                                cudaStream_t s);
cudaError_t launch_fringe(const RecParams &p, bool fp64, cudaStream_t s, bool pdl);
cudaError_t launch_reduce(const RecParams &p, bool fp64, cudaStream_t s, bool pdl);
cudaError_t launch_walk(const RecParams &p, bool fp64, cudaStream_t s, bool pdl);
cudaError_t launch_direct(const DirectParams &p, bool c128, cudaStream_t s);

// The same four stages as one cooperative kernel (rec_fused.cu, FP32).
// cudaErrorNotSupported when it cannot run here (then use the four kernels).
bool fused_supported(const RecParams &p, bool fp64);
cudaError_t launch_fused(const RecParams &p, const CUtensorMap &tmap, int num_sms, cudaStream_t s);

// 2-D tiled tensor map (FLOAT64 or FLOAT32 elements; out-of-bounds reads are
// zero): dim0 innermost. False if the driver entry point is missing or the
// encode fails (alignment, box limits).
bool encode_tiled_2d(CUtensorMap &map, bool f64, const void *base, unsigned long long dim0,
                     unsigned long long dim1, unsigned long long row_bytes, unsigned box0,
                     unsigned box1);

// Dense form on tcgen05 (gemm_tc.cu); complex64 input and output.
bool gemm_shape_ok(long long N, long long M, int P, int Q);
size_t gemm_workspace_size(long long N, long long M, int P, int Q);
cudaError_t launch_gemm_tf32x3(const void *A, long long N, long long M, long long lda, int P, int Q,
                               void *R, int mean, void *workspace, size_t ws_bytes, int sms,
                               cudaStream_t s, bool *ws_ok);
cudaError_t launch_gemm_bf16x3(const void *A, long long N, long long M, long long lda, int P, int Q,
                               void *R, int mean, void *workspace, size_t ws_bytes, int sms,
                               cudaStream_t s, bool *ws_ok);

}  // namespace cov
