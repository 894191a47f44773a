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

// Compensated (Neumaier) running sum: the error of each addition is kept in c.
template <typename T> struct Neu {
  T s, c;
  __device__ __forceinline__ Neu() : s(0), c(0) {}
  __device__ __forceinline__ void add(T x) {
    const T t = s + x;
    c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
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
__device__ __forceinline__ void cp_async_8(void *smem, const void *gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(sz)
               : "memory");
}
__device__ __forceinline__ void cp_async_16(void *smem, const void *gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(sz)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace cov
