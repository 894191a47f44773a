// Device helpers shared by the kernels of this library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cov {

template <typename T> struct C2t;
template <> struct C2t<float> { using type = float2; };
template <> struct C2t<double> { using type = double2; };

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename C2> __device__ __forceinline__ C2 czero() {
  C2 z;
  z.x = 0;
  z.y = 0;
  return z;
}

// acc += a * conj(b): re += ar*br + ai*bi, im += ai*br - ar*bi (4 FMA).
template <typename C2>
__device__ __forceinline__ void cmac_conj(C2 &acc, const C2 &a, const C2 &b) {
  acc.x = fma_rn(a.x, b.x, acc.x);
  acc.x = fma_rn(a.y, b.y, acc.x);
  acc.y = fma_rn(a.y, b.x, acc.y);
  acc.y = fma_rn(-a.x, b.y, acc.y);
}

// Packed FP32x2: two floats in one 64-bit register pair, and the paired FMA
// (fma.rn.f32x2: both halves rounded as two fma.rn.f32).
__device__ __forceinline__ unsigned long long pk2(float x, float y) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
__device__ __forceinline__ void ffma2(unsigned long long &acc, unsigned long long a,
                                      unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}
// (ar, ai) -> (ai, ar)
__device__ __forceinline__ unsigned long long swap2(unsigned long long a) {
  const float2 v = upk2(a);
  return pk2(v.y, v.x);
}

// |x| in x's own precision (an FP32 compare must not round-trip via FP64,
// whose pipe is narrow).
__device__ __forceinline__ float abs_of(float x) { return fabsf(x); }
__device__ __forceinline__ double abs_of(double x) { return fabs(x); }

// Compensated (Neumaier) running sum: the error of each addition is kept in c.
template <typename T> struct Neu {
  T s, c;
  __device__ __forceinline__ Neu() : s(0), c(0) {}
  __device__ __forceinline__ void add(T x) {
    const T t = s + x;
    c += (abs_of(s) >= abs_of(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
  }
  __device__ __forceinline__ void merge(T s2, T c2) {
    add(s2);
    c += c2;
  }
  __device__ __forceinline__ T value() const { return s + c; }
};

// Reduce V values per lane over the 32 lanes of a warp with V/2 + V/4 + ...
// shuffles instead of 5V: at each step a lane keeps one half of its values and
// sends the other half to its partner.
// V <= 32: afterwards v[0] holds the warp total of value index lane >> (5 - log2 V).
// V = 64:  afterwards v[0], v[1] hold the totals of indices 2*lane, 2*lane+1.
template <int V> struct Log2 { static constexpr int v = 1 + Log2<V / 2>::v; };
template <> struct Log2<1> { static constexpr int v = 0; };

template <int V, typename T>
__device__ __forceinline__ void warp_transpose_reduce(T (&v)[V], int lane) {
  static_assert((V & (V - 1)) == 0 && V <= 64, "V must be a power of two <= 64");
  constexpr int HS = Log2<V>::v < 5 ? Log2<V>::v : 5;  // halving steps
  int h = V / 2;
  int o = 16;
#pragma unroll
  for (int s = 0; s < HS; ++s) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < V / 2; ++i) {
      if (i < h) {
        const T send = up ? v[i] : v[i + h];
        const T keep = up ? v[i + h] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
    h >>= 1;
    o >>= 1;
  }
  if (HS < 5) {
#pragma unroll
    for (int oo = 16 >> HS; oo >= 1; oo >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], oo);
  }
}

// cp.async copies with zero fill: src_size 0 writes zeros without reading.
// No memory clobber: the copy lands asynchronously, and its completion is
// ordered by the wait that follows it (cp.async.wait_group or an mbarrier
// wait), which carries one; a clobber here would make the compiler reload
// every value it keeps in memory (kernel parameters read through a pointer)
// after each copy of a staging loop.
__device__ __forceinline__ void cp_async_8(void *smem, const void *gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async_16(void *smem, const void *gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---- mbarrier (shared::cta) -------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}
// Every prior cp.async of this thread arrives on `bar` when it completes.
__device__ __forceinline__ void cp_async_mbar_arrive_noinc(uint64_t *bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Waits for the phase of `bar` with the given parity to complete. Gives up
// after `limit_ns` nanoseconds and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity,
                                          unsigned long long limit_ns) {
  const unsigned a = smem_u32(bar);
  unsigned long long t0 = 0;
  for (unsigned it = 0;; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (it == 0) t0 = global_ns();
    else if ((it & 63) == 0 && global_ns() - t0 > limit_ns) return false;
  }
}

// ---- TMA: 2-D tiled bulk tensor load into shared memory ---------------------
__device__ __forceinline__ void tma_load_2d(void *smem_dst, const void *tmap, int x, int y,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_u32(smem_dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace cov
