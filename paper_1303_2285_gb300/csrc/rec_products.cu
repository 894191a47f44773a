// Kernel 1 of the combination path: every distinct product over the inner
// rows (see cov_internal.h for the split of the work).
#include <cuda.h>
#include <cuda_runtime.h>

#include "cov_launch.h"
#include "rec_products.cuh"

namespace cov {

template <typename T, int G, int R, int PITCH, int NCW>
__global__ void __launch_bounds__((NCW + 1) * 32, 1)
    k_products_inner(const RecParams p, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(1024) unsigned char smem_k1[];
  // the fringe-row kernel does not read this kernel's output: let it start
  // on SMs this kernel leaves free
  pdl_launch_dependents();
  const long long NT = p.n_tasks;
  const long long tb = NT * blockIdx.x / gridDim.x;
  const long long te = NT * (blockIdx.x + 1) / gridDim.x;
  products_phase<T, G, R, PITCH, NCW>(p, tmap, smem_k1, tb, te);
}

constexpr int kConsumerWarps = 16;

template <typename T, int G, int PITCH>
static cudaError_t launch_products_p(const RecParams &p, const CUtensorMap &tmap, int num_sms,
                                     cudaStream_t s) {
  // FP32: 16 rows per register block (each shared-memory load then feeds
  // more FMAs; the loads are within a factor two of the FMA time), 12
  // consumer warps for the registers of two accumulator pairs per lag
  constexpr bool f32 = sizeof(T) == 4;
  constexpr int NCW = f32 ? 12 : kConsumerWarps;
  auto kern = k_products_inner<T, G, f32 ? 16 : 8, PITCH, NCW>;
  const size_t smem = 2 * tile_buf_bytes<T, PITCH>(p.STR) + 64;
  cudaError_t e = ensure_smem_attr(kern, smem);
  if (e != cudaSuccess) return e;
  long long grid = num_sms;
  // FP32: a CTA's warps share its tasks. FP64 runs at a small fraction of the
  // FP32 rate per SM, so its tasks go one per SM first, up to the SM count.
  const long long per = sizeof(T) == 8 ? 1 : NCW;
  const long long need = (p.n_tasks + per - 1) / per;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  return launch_k(kern, dim3((unsigned)grid), dim3((NCW + 1) * 32), smem, s, false, p, tmap);
}

template <typename T, int G>
static cudaError_t launch_products(const RecParams &p, const CUtensorMap &tmap, int num_sms,
                                   cudaStream_t s) {
  switch (p.PITCH) {
    case 48: return launch_products_p<T, G, 48>(p, tmap, num_sms, s);
    case 64: return launch_products_p<T, G, 64>(p, tmap, num_sms, s);
    case 80: return launch_products_p<T, G, 80>(p, tmap, num_sms, s);
    case 96: return launch_products_p<T, G, 96>(p, tmap, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_products_any(const RecParams &p, const CUtensorMap &tmap, bool fp64, int num_sms,
                                cudaStream_t s) {
  switch (p.G) {
    case 4: return fp64 ? launch_products<double, 4>(p, tmap, num_sms, s)
                        : launch_products<float, 4>(p, tmap, num_sms, s);
    case 8: return fp64 ? launch_products<double, 8>(p, tmap, num_sms, s)
                        : launch_products<float, 8>(p, tmap, num_sms, s);
    case 16:
      if (fp64) return cudaErrorInvalidValue;  // FP64 uses at most 8 lags
      return launch_products<float, 16>(p, tmap, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace cov
