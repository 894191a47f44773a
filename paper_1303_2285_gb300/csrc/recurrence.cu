// The combination / diagonal-segment path (Sections 3.1-3.4, Algorithm 1),
// refined with the sliding-box recurrence: every distinct product of a
// unique combination is formed once, each combination's diagonal segments are
// seeded with a direct sum and walked along the diagonal, and one thread block
// writes each element of R. This file encodes the TMA map of A and launches
// the four kernels (rec_products.cu, rec_fringe.cu, rec_reduce.cu); see
// cov_internal.h for the notation and the split of the work.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>
#include <string.h>

#include "cov_internal.h"
#include "cov_launch.h"

namespace cov {

// ---------------------------------------------------------------------------
// TMA tensor map of A for the product kernel's tiles (host). A complex
// element is viewed as one 8-byte (complex64) or two 8-byte (complex128)
// FLOAT64 elements; the box is PITCH complex columns x STR rows; reads
// outside A are filled with zeros. Returns false when A cannot be described
// (base not 16-byte aligned or row pitch not a multiple of 16 bytes); the
// kernel then stages with cp.async.
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
  }
  return fn;
}

bool encode_tiled_2d(CUtensorMap &map, bool f64, const void *base, unsigned long long dim0,
                     unsigned long long dim1, unsigned long long row_bytes, unsigned box0,
                     unsigned box1) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)dim0, (cuuint64_t)dim1};
  cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
  cuuint32_t box[2] = {(cuuint32_t)box0, (cuuint32_t)box1};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r =
      enc(&map, f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
          const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static bool encode_tile_map_uncached(const RecParams &p, bool fp64, CUtensorMap &tmap);

// The last encoded map is reused when the same A, shape and tile are seen
// again (host-side cache; the encode call is not free).
static bool encode_tile_map(const RecParams &p, bool fp64, CUtensorMap &tmap) {
  static thread_local struct {
    const void *A;
    long long lda;
    int N, M, STR, PITCH, fp64, ok;
    CUtensorMap map;
  } c = {nullptr, 0, 0, 0, 0, 0, 0, 0, {}};
  if (c.A == p.A && c.lda == p.lda && c.N == p.N && c.M == p.M && c.STR == p.STR &&
      c.PITCH == p.PITCH && c.fp64 == (int)fp64) {
    tmap = c.map;
    return c.ok != 0;
  }
  const bool ok = encode_tile_map_uncached(p, fp64, tmap);
  c.A = p.A;
  c.lda = p.lda;
  c.N = p.N;
  c.M = p.M;
  c.STR = p.STR;
  c.PITCH = p.PITCH;
  c.fp64 = (int)fp64;
  c.ok = ok ? 1 : 0;
  c.map = tmap;
  return ok;
}

static bool encode_tile_map_uncached(const RecParams &p, bool fp64, CUtensorMap &tmap) {
  const int per = fp64 ? 2 : 1;  // FLOAT64 elements per complex value
  const size_t row_bytes = (size_t)p.lda * 8 * per;
  if (((uintptr_t)p.A & 15) != 0 || (row_bytes & 15) != 0) return false;
  if (p.STR > 256 || p.PITCH * per > 256) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)p.M * per, (cuuint64_t)p.N};
  cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
  cuuint32_t box[2] = {(cuuint32_t)(p.PITCH * per), (cuuint32_t)p.STR};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void *>(p.A), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------
// Launch sequence. Kernels 2-4 use programmatic dependent launch (their
// launch overlaps the previous kernel; each waits on its inputs in-kernel),
// except when stage events are recorded between the kernels.
// ---------------------------------------------------------------------------
cudaError_t launch_recurrence(const RecParams &p, bool fp64, int num_sms, cudaStream_t s,
                              StageEvents *ev) {
  CUtensorMap tmap;
  memset(&tmap, 0, sizeof(tmap));
  RecParams q = p;
  q.use_tma = 0;
  if (p.n_inner > 0 && encode_tile_map(p, fp64, tmap)) q.use_tma = 1;
  const bool inst = ev && ev->on;
  const int slot = inst ? (int)(ev->calls % ev->rounds) : 0;
  auto mark = [&](int k) -> cudaError_t {
    return inst ? cudaEventRecord(ev->ev[5 * slot + k], s) : cudaSuccess;
  };
  const bool pdl = !inst;
  cudaError_t e;
  if (q.fused && fused_supported(q, fp64)) {
    // one kernel: with stage events, event 0 before it and events 1-4 after
    if ((e = mark(0)) != cudaSuccess) return e;
    e = launch_fused(q, tmap, num_sms, s);
    if (e != cudaErrorNotSupported) {
      if (e != cudaSuccess) return e;
      for (int k = 1; k <= 4; ++k)
        if ((e = mark(k)) != cudaSuccess) return e;
      if (inst) ++ev->calls;
      return cudaSuccess;
    }
    cudaGetLastError();  // not co-resident here: the four kernels below
  }
  if ((e = mark(0)) != cudaSuccess) return e;
  // Without inner rows there is no product kernel; the fringe-row kernel,
  // which reads A before its dependency wait, is then launched without PDL
  // so that it cannot overlap the stream's earlier work.
  const bool products = q.n_inner > 0 && q.n_tasks > 0;
  if (products && (e = launch_products_any(q, tmap, fp64, num_sms, s)) != cudaSuccess) return e;
  if ((e = mark(1)) != cudaSuccess) return e;
  if ((e = launch_fringe(q, fp64, s, pdl && products)) != cudaSuccess) return e;
  if ((e = mark(2)) != cudaSuccess) return e;
  if ((e = launch_reduce(q, fp64, s, pdl)) != cudaSuccess) return e;
  if ((e = mark(3)) != cudaSuccess) return e;
  if ((e = launch_walk(q, fp64, s, pdl)) != cudaSuccess) return e;
  if ((e = mark(4)) != cudaSuccess) return e;
  if (inst) ++ev->calls;
  return cudaSuccess;
}

}  // namespace cov
