// Measured FMA rates of the FP32 and FP64 pipes (instrumentation; not in the
// paper). The combination path is bound by plain FMA arithmetic (4 FMA per
// distinct product), so its roofline needs the rate of the pipe it runs on:
// FP32 (paired fma.rn.f32x2, as the product kernels issue it) or FP64
// (fma.rn.f64, the COV_C128 path). GB300's FP64 rate per SM is a small
// fraction of its FP32 rate and is not printed next to the clock, so it is
// measured here.
//
// Kernel: SMs x 4 CTAs of 256 threads, every thread running CH independent
// dependent-FMA chains (enough in flight to cover the pipe latency). The
// chains' results feed one conditional store that never happens, so nothing
// is optimised away and no memory traffic is timed.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cov.h"
#include "cov_device.cuh"

namespace cov {

__device__ float g_fma_sink_f32;
__device__ double g_fma_sink_f64;

template <int CH>
__global__ void __launch_bounds__(256) k_fma_rate_f32x2(int iters) {
  unsigned long long acc[CH];
  const float b = 1e-3f * (float)(threadIdx.x & 31);
#pragma unroll
  for (int k = 0; k < CH; ++k) acc[k] = pk2(b + (float)k, b - (float)k);
  const unsigned long long m = pk2(0.99990f, 1.00010f), c = pk2(1e-7f, -1e-7f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CH; ++k)
      asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(acc[k]) : "l"(m), "l"(c));
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < CH; ++k) {
    const float2 v = upk2(acc[k]);
    s += v.x + v.y;
  }
  if (s == 1234.5f) g_fma_sink_f32 = s;
}

template <int CH>
__global__ void __launch_bounds__(256) k_fma_rate_f64(int iters) {
  double acc[CH];
  const double b = 1e-3 * (double)(threadIdx.x & 31);
#pragma unroll
  for (int k = 0; k < CH; ++k) acc[k] = b + (double)k;
  const double m = 0.9999, c = 1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CH; ++k) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(acc[k]) : "d"(m), "d"(c));
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CH; ++k) s += acc[k];
  if (s == 1234.5) g_fma_sink_f64 = s;
}

}  // namespace cov

extern "C" cov_status cov_measure_fma_rate(cov_dtype dtype, int reps, double *fma_per_s,
                                           cov_stream_t stream) {
  if (!fma_per_s || reps < 1 || reps > 100 || (dtype != COV_C64 && dtype != COV_C128))
    return COV_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    return COV_ECUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  constexpr int CH = 8, THREADS = 256;
  const int blocks = sms * 4;
  // about 4e10 FP32 or 1.3e9 FP64 lane FMAs per launch (about 1 and 2 ms)
  const int iters = dtype == COV_C64 ? 16384 : 512;
  const double fmas = (double)blocks * THREADS * iters * CH * (dtype == COV_C64 ? 2.0 : 1.0);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return COV_ECUDA;
  }
  cov_status st = COV_OK;
  float best = -1.f;
  for (int r = 0; r <= reps && st == COV_OK; ++r) {  // the first launch warms up
    if (cudaEventRecord(e0, s) != cudaSuccess) st = COV_ECUDA;
    if (st == COV_OK) {
      if (dtype == COV_C64)
        cov::k_fma_rate_f32x2<CH><<<blocks, THREADS, 0, s>>>(iters);
      else
        cov::k_fma_rate_f64<CH><<<blocks, THREADS, 0, s>>>(iters);
      if (cudaGetLastError() != cudaSuccess) st = COV_ECUDA;
    }
    if (st == COV_OK && cudaEventRecord(e1, s) != cudaSuccess) st = COV_ECUDA;
    if (st == COV_OK && cudaEventSynchronize(e1) != cudaSuccess) st = COV_ECUDA;
    float ms = 0.f;
    if (st == COV_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = COV_ECUDA;
    if (st == COV_OK && r > 0 && ms > 0.f && (best < 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != COV_OK) {
    cudaGetLastError();
    return st;
  }
  if (best <= 0.f) return COV_ECUDA;
  *fma_per_s = fmas / ((double)best * 1e-3);
  return COV_OK;
}
