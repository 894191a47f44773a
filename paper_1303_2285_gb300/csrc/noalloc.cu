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
// stand-in), so the device address is looked up with cudaGetSymbolAddress,
// with the caller's device and context current, on the first call made in
// that context; later calls in the same context reuse it. The address
// belongs to a CUDA context, not to a device ordinal: a plugin that runs in
// its host application's own driver context gets that context's copy of the
// array, and a context created after cudaDeviceReset gets a fresh lookup
// (the cache is keyed by the context's process-unique ID).
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "../../include/cov.h"
#include "cov_internal.h"
#include "cov_launch.h"
#include "plan.h"

namespace {

constexpr size_t kNoAllocScratchBytes = COV_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

struct ScratchEntry {
  unsigned long long ctx_id;
  void *addr;
  int sms;
};

std::mutex g_setup_mutex;
std::vector<ScratchEntry> g_entries;

// The driver's cuCtxGetCurrent and cuCtxGetId (looked up once).
bool context_api(CtxGetCurrentFn *get_cur, CtxGetIdFn *get_id) {
  static CtxGetCurrentFn cur = nullptr;
  static CtxGetIdFn id = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      cur = (CtxGetCurrentFn)p;
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      id = (CtxGetIdFn)p;
    cudaGetLastError();
  }
  *get_cur = cur;
  *get_id = id;
  return cur != nullptr && id != nullptr;
}

// Device address of g_noalloc_scratch in the current context and the SM
// count of the current device, looked up on the first call in a context.
// On failure the runtime's last-error state is cleared, so that a caller's
// next cudaGetLastError does not report this library's failure as its own.
cov_status scratch_for_current_context(void **addr, int *sms) {
  CtxGetCurrentFn get_cur;
  CtxGetIdFn get_id;
  if (!context_api(&get_cur, &get_id)) return COV_ECUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return COV_ECUDA;
  }
  CUcontext ctx = nullptr;
  if (get_cur(&ctx) != CUDA_SUCCESS) return COV_ECUDA;
  if (ctx == nullptr) {
    // no context current yet: the runtime call binds the device's primary one
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return COV_ECUDA;
    }
    if (get_cur(&ctx) != CUDA_SUCCESS || ctx == nullptr) return COV_ECUDA;
  }
  unsigned long long id = 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return COV_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  for (const ScratchEntry &e : g_entries)
    if (e.ctx_id == id) {
      *addr = e.addr;
      *sms = e.sms;
      return COV_OK;
    }
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return COV_ECUDA;
  }
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return COV_ECUDA;
  }
  g_entries.push_back({id, p, n});
  *addr = p;
  *sms = n;
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
  const cov_status st = scratch_for_current_context(&base, &sms);
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

// The status word of the static scratch (its first 4 bytes), where the
// kernels of cov_estimate_noalloc record a bounded wait that gave up: read
// and cleared, as cov_check_device_status does for a caller's workspace.
extern "C" cov_status cov_noalloc_check_status(cov_stream_t stream) {
  void *base = nullptr;
  int sms = 0;
  const cov_status st = scratch_for_current_context(&base, &sms);
  if (st != COV_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned word = 0;
  if (cudaMemcpyAsync(&word, base, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess || cudaMemsetAsync(base, 0, 4, s) != cudaSuccess) {
    cudaGetLastError();
    return COV_ECUDA;
  }
  if (word == cov::kDevOk) return COV_OK;
  if (word == cov::kDevTimeout) return COV_ETIMEOUT;
  return COV_EDEVICE;
}
