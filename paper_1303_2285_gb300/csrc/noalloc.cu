// An entry point of the combination path that allocates no device memory.
//
// Who needs it: callers that must not allocate device memory at call time.
// Examples are a plugin inside a host application whose own memory pool has
// already reserved the device memory, and a real-time radar / SAR processing
// loop whose device-memory budget is fixed at start-up so that no call can
// fail, stall or fragment memory mid-stream. Such callers cannot use
// cov_estimate (cudaMallocAsync) and may not own a buffer large enough to
// pass to cov_estimate_ex either.
//
// How: the scratch space of the combination path lives in a file-scope
// static __device__ array (kNoAllocScratchBytes). Every GPU that loads this
// library holds that array until the process exits. Host code cannot use the
// array's name as a device address (in host code it names a host-side
// stand-in), so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made
// while the device is current. Later calls reuse the cached address.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/cov.h"
#include "cov_internal.h"
#include "cov_launch.h"
#include "plan.h"

namespace {

constexpr size_t kNoAllocScratchBytes = COV_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};
int g_sms[kMaxDevices] = {0};

// Device address of g_noalloc_scratch and SM count of the current device,
// looked up on the first call for that device.
cov_status scratch_for_current_device(void **addr, int *sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return COV_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_addr[dev] == nullptr) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
      return COV_ECUDA;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      return COV_ECUDA;
    g_scratch_addr[dev] = p;
    g_sms[dev] = n;
  }
  *addr = g_scratch_addr[dev];
  *sms = g_sms[dev];
  return COV_OK;
}

}  // namespace

extern "C" cov_status cov_estimate_noalloc(const void *A, cov_dtype dtype, int64_t N, int64_t M,
                                           int64_t lda, int P, int Q, void *R, cov_norm norm,
                                           cov_stream_t stream) {
  using namespace cov;
  if (!A || !R || N < 1 || M < 1 || P < 1 || Q < 1 || P > N || Q > M || lda < M ||
      (dtype != COV_C64 && dtype != COV_C128) || (norm != COV_MEAN && norm != COV_SUM))
    return COV_EINVAL;
  if (!recurrence_ok(N, M, P, Q)) return COV_EUNSUPPORTED;
  const int elem = dtype == COV_C128 ? 16 : 8;
  if (((uintptr_t)A % (uintptr_t)(elem / 2)) != 0 || ((uintptr_t)R % (uintptr_t)(elem / 2)) != 0)
    return COV_EINVAL;
  void *base = nullptr;
  int sms = 0;
  const cov_status st = scratch_for_current_device(&base, &sms);
  if (st != COV_OK) return st;
  RecParams p;
  WsLayout ws;
  plan_recurrence(N, M, lda, P, Q, elem, sms, p, ws);
  if (ws.total > kNoAllocScratchBytes) return COV_EWORKSPACE;  // beyond the static maximum
  cudaStream_t s = (cudaStream_t)stream;
  char *w = (char *)base;
  p.A = A;
  p.R = R;
  p.mean = norm == COV_MEAN ? 1 : 0;
  p.status = (unsigned *)w;
  p.core_part = w + ws.core_off;
  p.colsum_part = w + ws.colsum_off;
  p.sin_part = w + ws.sin_off;
  p.rowval = w + ws.rowval_off;
  p.colval = w + ws.colval_off;
  // The status word and the fused kernel's barrier and task counters (the
  // first 16 bytes) must start at zero; every other scratch region is fully
  // written by the kernels before it is read.
  if (cudaMemsetAsync(w, 0, 16, s) != cudaSuccess) return COV_ECUDA;
  if (launch_recurrence(p, dtype == COV_C128, sms, s, nullptr) != cudaSuccess) return COV_ECUDA;
  return COV_OK;
}
