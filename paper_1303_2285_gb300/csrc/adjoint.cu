// Adjoint of the estimate (not in the paper; the derivative of Eq. 2.2).
//
// With G = dL/dR and dA in the convention dL/dRe + i dL/dIm:
//   dL/dx_w = H x_w,  H = (G + G^H) / K   (G + G^H for the plain sum),
//   dA[n][m] = sum over windows w = (p, q) that hold (n, m) of (H x_w)[a],
//   a = (n - p) + P (m - q).
// Kernel 1 forms Y = H X for tiles of windows: X (PQ x K, column w = the
// window's column stack) is never stored; each CTA gathers its windows' values
// from a staged patch of A. Kernel 2 is the col2im in gather form: one thread
// per element of dA sums the entries of Y that belong to it, so every element
// of dA has one writer and no atomics are needed. Both are templated on the
// real type: FP32 for complex64, FP64 for complex128 (this dense form is the
// adjoint of complex128 estimates).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cov.h"
#include "cov_device.cuh"
#include "cov_internal.h"
#include "smem_attr.h"
#include "plan.h"

namespace cov {

// stencil form (adjoint_stencil.cu)
bool stencil_adjoint_ok(long long N, long long M, int P, int Q);
size_t stencil_adjoint_workspace(int P, int Q, int batch);
cudaError_t launch_stencil_adjoint(const void *A, const void *G, long long N, long long M, int P,
                                   int Q, int mean, void *dA, void *workspace, cudaStream_t s,
                                   int batch, long long sA, long long sG, long long sdA);

constexpr int kAdjTA = 48;   // rows a of Y per CTA
constexpr int kAdjTW = 128;  // windows per CTA (one window row p, consecutive q)
constexpr int kAdjPQMax = 1024;

template <typename T> struct AdjParams {
  using C2 = typename C2t<T>::type;
  const C2 *A;
  const C2 *G;
  C2 *Y;   // [PQ][KW], window index w = p * W + q
  C2 *dA;  // N x M, leading dimension M
  long long lda;
  int N, M, P, Q, W, Hn;  // W = M-Q+1 window columns, Hn = N-P+1 window rows
  long long KW;           // number of windows
  int mean;
};

// Y[a][w] for a in [a0, a0+48), w = p*W + q, q in [q0, q0+128).
// Thread (ta, tw) of a 16 x 16 grid: a = a0 + ta + 16k (k < 3),
// q = q0 + tw + 16l (l < 8): 24 complex accumulators.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_hx(const AdjParams<T> p) {
  using C2 = typename C2t<T>::type;
  extern __shared__ __align__(16) unsigned char smem_adj[];
  const int D = p.P * p.Q;
  C2 *Hs = (C2 *)smem_adj;                        // [48][D]
  C2 *As = Hs + kAdjTA * D;                       // [P][128 + Q - 1]
  const int AP = kAdjTW + p.Q - 1;
  const int nqc = (p.W + kAdjTW - 1) / kAdjTW;
  int bid = blockIdx.x;
  const int qc = bid % nqc;
  bid /= nqc;
  const int pw = bid % p.Hn;
  const int a0 = (bid / p.Hn) * kAdjTA;
  const int q0 = qc * kAdjTW;
  // H rows a0..a0+47: H[a][b] = (G[a][b] + conj(G[b][a])) / K
  for (int e = threadIdx.x; e < kAdjTA * D; e += blockDim.x) {
    const int ar = e / D, b = e - ar * D, a = a0 + ar;
    C2 h = czero<C2>();
    if (a < D) {
      const C2 g1 = p.G[(long long)a * D + b], g2 = p.G[(long long)b * D + a];
      h.x = g1.x + g2.x;
      h.y = g1.y - g2.y;
      if (p.mean) {
        h.x = h.x / (T)p.KW;
        h.y = h.y / (T)p.KW;
      }
    }
    Hs[e] = h;
  }
  // patch of A: rows pw..pw+P-1, columns q0..q0+127+Q-1 (zero outside A)
  for (int e = threadIdx.x; e < p.P * AP; e += blockDim.x) {
    const int r = e / AP, c = e - r * AP;
    const int gc = q0 + c;
    As[e] = gc < p.M ? p.A[(long long)(pw + r) * p.lda + gc] : czero<C2>();
  }
  __syncthreads();
  const int ta = threadIdx.x >> 4, tw = threadIdx.x & 15;
  C2 acc[3][8];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int l = 0; l < 8; ++l) acc[k][l] = czero<C2>();
  for (int jb = 0, b = 0; jb < p.Q; ++jb)
  for (int ib = 0; ib < p.P; ++ib, ++b) {
    C2 h[3], x[8];
#pragma unroll
    for (int k = 0; k < 3; ++k) h[k] = Hs[(ta + 16 * k) * D + b];
#pragma unroll
    for (int l = 0; l < 8; ++l) x[l] = As[ib * AP + tw + 16 * l + jb];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = 0; l < 8; ++l) {  // acc += h * x
        acc[k][l].x = fma_rn(h[k].x, x[l].x, acc[k][l].x);
        acc[k][l].x = fma_rn(-h[k].y, x[l].y, acc[k][l].x);
        acc[k][l].y = fma_rn(h[k].x, x[l].y, acc[k][l].y);
        acc[k][l].y = fma_rn(h[k].y, x[l].x, acc[k][l].y);
      }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int a = a0 + ta + 16 * k;
    if (a >= D) continue;
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      const int q = q0 + tw + 16 * l;
      if (q < p.W) p.Y[(long long)a * p.KW + (long long)pw * p.W + q] = acc[k][l];
    }
  }
}

// dA[n][m] = sum over (i, j) with window (n-i, m-j) valid of Y[i + P j][(n-i) W + (m-j)].
template <typename T>
__global__ void __launch_bounds__(256) k_adj_col2im(const AdjParams<T> p) {
  using C2 = typename C2t<T>::type;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)p.N * p.M) return;
  const int n = (int)(idx / p.M), m = (int)(idx - (long long)n * p.M);
  const int i_lo = n - (p.Hn - 1) > 0 ? n - (p.Hn - 1) : 0, i_hi = n < p.P - 1 ? n : p.P - 1;
  const int j_lo = m - (p.W - 1) > 0 ? m - (p.W - 1) : 0, j_hi = m < p.Q - 1 ? m : p.Q - 1;
  T sr = T(0), si = T(0);
  for (int j = j_lo; j <= j_hi; ++j)
    for (int i = i_lo; i <= i_hi; ++i) {
      const C2 y = p.Y[(long long)(i + p.P * j) * p.KW + (long long)(n - i) * p.W + (m - j)];
      sr += y.x;
      si += y.y;
    }
  C2 o;
  o.x = sr;
  o.y = si;
  p.dA[idx] = o;
}

}  // namespace cov

namespace {
template <typename T>
cov_status dense_adjoint(const void *A, const void *G, int64_t N, int64_t M, int P, int Q,
                         cov_norm norm, void *dA, void *workspace, cudaStream_t s) {
  using C2 = typename cov::C2t<T>::type;
  cov::AdjParams<T> p;
  p.A = (const C2 *)A;
  p.G = (const C2 *)G;
  p.Y = (C2 *)((char *)workspace + cov::kWsHeader);
  p.dA = (C2 *)dA;
  p.lda = M;
  p.N = (int)N;
  p.M = (int)M;
  p.P = P;
  p.Q = Q;
  p.W = (int)(M - Q + 1);
  p.Hn = (int)(N - P + 1);
  p.KW = (long long)p.W * p.Hn;
  p.mean = norm == COV_MEAN ? 1 : 0;
  const int D = P * Q;
  const size_t smem = ((size_t)cov::kAdjTA * D + (size_t)P * (cov::kAdjTW + Q - 1)) * sizeof(C2);
  if (smem > 227 * 1024) return COV_EUNSUPPORTED;
  if (cov::ensure_dyn_smem((const void *)cov::k_adj_hx<T>, smem, false) != cudaSuccess)
    return COV_ECUDA;
  const long long nqc = (p.W + cov::kAdjTW - 1) / cov::kAdjTW;
  const long long grid1 = nqc * p.Hn * ((D + cov::kAdjTA - 1) / cov::kAdjTA);
  cov::k_adj_hx<T><<<(unsigned)grid1, 256, smem, s>>>(p);
  if (cudaGetLastError() != cudaSuccess) return COV_ECUDA;
  const long long grid2 = (N * M + 255) / 256;
  cov::k_adj_col2im<T><<<(unsigned)grid2, 256, 0, s>>>(p);
  return cudaGetLastError() == cudaSuccess ? COV_OK : COV_ECUDA;
}
}  // namespace

extern "C" {

cov_status cov_partition_rows(int64_t N, int P, int n_ranks, int64_t *row_begin, int64_t *halo_lo,
                              int64_t *halo_hi) {
  if (!row_begin || N < 1 || P < 1 || P > N || n_ranks < 1 || n_ranks > 65536) return COV_EINVAL;
  for (int r = 0; r <= n_ranks; ++r) row_begin[r] = (int64_t)((__int128)N * r / n_ranks);
  for (int r = 0; r < n_ranks; ++r) {
    // rows of every window that covers a row of the band
    const int64_t lo = row_begin[r] - (P - 1), hi = row_begin[r + 1] + (P - 1);
    if (halo_lo) halo_lo[r] = lo < 0 ? 0 : lo;
    if (halo_hi) halo_hi[r] = hi > N ? N : hi;
  }
  return COV_OK;
}

static bool bwd_args_ok(int64_t N, int64_t M, int P, int Q) {
  return N >= 1 && M >= 1 && P >= 1 && Q >= 1 && P <= N && Q <= M && N < (1LL << 30) &&
         M < (1LL << 30);
}

// the form AUTO resolves to: the stencil wherever it applies
static cov_bwd_form resolve_bwd(cov_bwd_form f, int64_t N, int64_t M, int P, int Q) {
  if (f != COV_BWD_AUTO) return f;
  return cov::stencil_adjoint_ok(N, M, P, Q) ? COV_BWD_STENCIL : COV_BWD_DENSE;
}

cov_status cov_backward_workspace_size_ex(cov_dtype dtype, int64_t N, int64_t M, int P, int Q,
                                          cov_bwd_form form, size_t *bytes) {
  if (!bytes || !bwd_args_ok(N, M, P, Q)) return COV_EINVAL;
  if (dtype != COV_C64 && dtype != COV_C128) return COV_EINVAL;
  // complex128: the dense form (FP64) only
  form = dtype == COV_C128 && form == COV_BWD_AUTO ? COV_BWD_DENSE : resolve_bwd(form, N, M, P, Q);
  if (dtype == COV_C128 && form == COV_BWD_STENCIL) return COV_EUNSUPPORTED;
  if (form == COV_BWD_STENCIL) {
    if (!cov::stencil_adjoint_ok(N, M, P, Q)) return COV_EUNSUPPORTED;
    *bytes = cov::stencil_adjoint_workspace(P, Q, 1);
    return COV_OK;
  }
  if (form != COV_BWD_DENSE) return COV_EINVAL;
  if ((long long)P * Q > cov::kAdjPQMax) return COV_EUNSUPPORTED;
  const long long KW = (N - P + 1) * (M - Q + 1);
  const size_t elem = dtype == COV_C128 ? 16 : 8;
  *bytes = cov::kWsHeader + (((size_t)P * Q * KW * elem + 255) & ~(size_t)255);
  return COV_OK;
}

cov_status cov_backward_workspace_size(cov_dtype dtype, int64_t N, int64_t M, int P, int Q,
                                       size_t *bytes) {
  return cov_backward_workspace_size_ex(dtype, N, M, P, Q, COV_BWD_AUTO, bytes);
}

cov_status cov_estimate_backward_ex(const void *A, const void *G, cov_dtype dtype, int64_t N,
                                    int64_t M, int P, int Q, cov_norm norm, cov_bwd_form form,
                                    void *dA, void *workspace, size_t ws_bytes, cov_stream_t stream) {
  if (!A || !G || !dA || !bwd_args_ok(N, M, P, Q) || (norm != COV_MEAN && norm != COV_SUM))
    return COV_EINVAL;
  if (dtype != COV_C64 && dtype != COV_C128) return COV_EINVAL;
  const uintptr_t al = dtype == COV_C128 ? 15 : 7;
  if ((((uintptr_t)A) & al) || (((uintptr_t)G) & al) || (((uintptr_t)dA) & al)) return COV_EINVAL;
  form = dtype == COV_C128 && form == COV_BWD_AUTO ? COV_BWD_DENSE : resolve_bwd(form, N, M, P, Q);
  size_t need = 0;
  const cov_status st = cov_backward_workspace_size_ex(dtype, N, M, P, Q, form, &need);
  if (st != COV_OK) return st;
  if (!workspace || ws_bytes < need || ((uintptr_t)workspace & 255) != 0) return COV_EWORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(workspace, 0, 4, s) != cudaSuccess) return COV_ECUDA;
  if (form == COV_BWD_STENCIL)
    return cov::launch_stencil_adjoint(A, G, N, M, P, Q, norm == COV_MEAN ? 1 : 0, dA, workspace,
                                       s, 1, 0, 0, 0) == cudaSuccess
               ? COV_OK
               : COV_ECUDA;
  return dtype == COV_C128 ? dense_adjoint<double>(A, G, N, M, P, Q, norm, dA, workspace, s)
                           : dense_adjoint<float>(A, G, N, M, P, Q, norm, dA, workspace, s);
}

cov_status cov_backward_strided_workspace_size(int batch, int64_t N, int64_t M, int P, int Q,
                                               size_t *bytes) {
  if (!bytes || batch < 1 || batch > 65535 || !bwd_args_ok(N, M, P, Q)) return COV_EINVAL;
  if (!cov::stencil_adjoint_ok(N, M, P, Q)) return COV_EUNSUPPORTED;
  *bytes = cov::stencil_adjoint_workspace(P, Q, batch);
  return COV_OK;
}

cov_status cov_estimate_backward_strided(const void *A, int64_t stride_A, const void *G,
                                         int64_t stride_G, void *dA, int64_t stride_dA, int batch,
                                         int64_t N, int64_t M, int P, int Q, cov_norm norm,
                                         void *workspace, size_t ws_bytes, cov_stream_t stream) {
  if (!A || !G || !dA || batch < 1 || batch > 65535 || !bwd_args_ok(N, M, P, Q) ||
      (norm != COV_MEAN && norm != COV_SUM))
    return COV_EINVAL;
  const long long D = (long long)P * Q;
  if (stride_A < N * M || stride_dA < N * M || stride_G < D * D) return COV_EINVAL;
  if ((((uintptr_t)A) & 7) || (((uintptr_t)G) & 7) || (((uintptr_t)dA) & 7)) return COV_EINVAL;
  if (!cov::stencil_adjoint_ok(N, M, P, Q)) return COV_EUNSUPPORTED;
  const size_t need = cov::stencil_adjoint_workspace(P, Q, batch);
  if (!workspace || ws_bytes < need || ((uintptr_t)workspace & 255) != 0) return COV_EWORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(workspace, 0, 4, s) != cudaSuccess) return COV_ECUDA;
  return cov::launch_stencil_adjoint(A, G, N, M, P, Q, norm == COV_MEAN ? 1 : 0, dA, workspace, s,
                                     batch, stride_A, stride_G, stride_dA) == cudaSuccess
             ? COV_OK
             : COV_ECUDA;
}

cov_status cov_estimate_backward(const void *A, const void *G, cov_dtype dtype, int64_t N, int64_t M,
                                 int P, int Q, cov_norm norm, void *dA, void *workspace,
                                 size_t ws_bytes, cov_stream_t stream) {
  return cov_estimate_backward_ex(A, G, dtype, N, M, P, Q, norm, COV_BWD_AUTO, dA, workspace,
                                  ws_bytes, stream);
}

}  // extern "C"
