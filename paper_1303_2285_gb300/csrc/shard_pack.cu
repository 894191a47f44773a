// Packing of the R blocks a column-lag shard owns, for the exchange between
// ranks (Section 4.2: the combinations of the column lags [dc_lo, dc_hi) own
// exactly the P x P blocks (a, b) of R with dc_lo <= |b - a| < dc_hi, so a
// sharded estimate is assembled by gathering those blocks, with no
// reduction). The packed layout lists the blocks lag by lag, and within lag
// dc for a = 0 .. Q - dc - 1 the block (a, a + dc) followed, for dc > 0, by
// its mirror (a + dc, a); each block is P x P, row-major.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cov.h"

namespace cov {

__host__ __device__ inline long long shard_block_count(int Q, int dc_lo, int dc_hi) {
  long long n = 0;
  for (int dc = dc_lo; dc < dc_hi; ++dc) n += dc == 0 ? Q : 2LL * (Q - dc);
  return n;
}

// Block k of the shard's list.
__device__ __forceinline__ void shard_block_of(int Q, int dc_lo, long long k, int &a, int &b) {
  int dc = dc_lo;
  for (;;) {
    const long long nb = dc == 0 ? Q : 2LL * (Q - dc);
    if (k < nb) break;
    k -= nb;
    ++dc;
  }
  if (dc == 0) {
    a = b = (int)k;
  } else {
    const int aa = (int)(k >> 1);
    if ((k & 1) == 0) {
      a = aa;
      b = aa + dc;
    } else {
      a = aa + dc;
      b = aa;
    }
  }
}

// One CTA per block; E = the complex element (float2 or double2), copied as is.
template <typename E, bool PACK>
__global__ void __launch_bounds__(256) k_shard_copy(const E *src, E *dst, int P, int Q, int dc_lo) {
  int a, b;
  shard_block_of(Q, dc_lo, blockIdx.x, a, b);
  const long long D = (long long)P * Q;
  const long long base = (long long)blockIdx.x * P * P;
  for (int i = threadIdx.y; i < P; i += blockDim.y)
    for (int ii = threadIdx.x; ii < P; ii += blockDim.x) {
      const long long r = ((long long)a * P + i) * D + (long long)b * P + ii;
      const long long k = base + (long long)i * P + ii;
      if (PACK)
        dst[k] = src[r];
      else
        dst[r] = src[k];
    }
}

template <bool PACK>
static cov_status shard_copy(const void *src, cov_dtype dtype, int P, int Q, int dc_lo, int dc_hi,
                             void *dst, cudaStream_t s) {
  const long long nb = shard_block_count(Q, dc_lo, dc_hi);
  if (nb == 0) return COV_OK;
  if (nb > 0x7fffffffLL) return COV_EINVAL;
  const dim3 block(32, 8);
  if (dtype == COV_C128)
    k_shard_copy<double2, PACK><<<(unsigned)nb, block, 0, s>>>((const double2 *)src, (double2 *)dst, P,
                                                               Q, dc_lo);
  else
    k_shard_copy<float2, PACK><<<(unsigned)nb, block, 0, s>>>((const float2 *)src, (float2 *)dst, P, Q,
                                                              dc_lo);
  return cudaGetLastError() == cudaSuccess ? COV_OK : COV_ECUDA;
}

static bool shard_args_ok(cov_dtype dtype, int P, int Q, int dc_lo, int dc_hi) {
  return (dtype == COV_C64 || dtype == COV_C128) && P >= 1 && Q >= 1 &&
         (long long)P * Q <= (1LL << 15) && dc_lo >= 0 && dc_hi >= dc_lo && dc_hi <= Q;
}

}  // namespace cov

extern "C" cov_status cov_shard_packed_size(cov_dtype dtype, int P, int Q, int dc_lo, int dc_hi,
                                            size_t *bytes) {
  if (!bytes || !cov::shard_args_ok(dtype, P, Q, dc_lo, dc_hi)) return COV_EINVAL;
  *bytes = (size_t)cov::shard_block_count(Q, dc_lo, dc_hi) * P * P * (dtype == COV_C128 ? 16 : 8);
  return COV_OK;
}

extern "C" cov_status cov_shard_pack(const void *R, cov_dtype dtype, int P, int Q, int dc_lo,
                                     int dc_hi, void *packed, cov_stream_t stream) {
  if (!cov::shard_args_ok(dtype, P, Q, dc_lo, dc_hi)) return COV_EINVAL;
  if (dc_hi > dc_lo && (!R || !packed)) return COV_EINVAL;
  return cov::shard_copy<true>(R, dtype, P, Q, dc_lo, dc_hi, packed, (cudaStream_t)stream);
}

extern "C" cov_status cov_shard_unpack(const void *packed, cov_dtype dtype, int P, int Q, int dc_lo,
                                       int dc_hi, void *R, cov_stream_t stream) {
  if (!cov::shard_args_ok(dtype, P, Q, dc_lo, dc_hi)) return COV_EINVAL;
  if (dc_hi > dc_lo && (!R || !packed)) return COV_EINVAL;
  return cov::shard_copy<false>(packed, dtype, P, Q, dc_lo, dc_hi, R, (cudaStream_t)stream);
}
