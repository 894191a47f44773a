// The combination path (FP32) as one cooperative kernel.
//
// The four stages of the path (products over the inner rows, fringe-row
// products, reductions, seed-and-walk writer; see cov_internal.h) run in one
// launch of one CTA per SM, co-resident by construction (cooperative launch):
//   1. every CTA runs its share of the product tasks (producer warp + TMA
//      double buffer, as the stand-alone product kernel);
//   2. CTAs then take fringe-row tasks (side, column chunk, block of at most
//      one (row, lag) pair per thread) from a global counter, so the CTAs
//      that finish their product tasks first absorb this work and the tail
//      of stage 1;
//   3. grid barrier; the reduction warp tasks, spread over all warps;
//   4. grid barrier; the P x P blocks of R, one CTA at a time.
// This removes three kernel boundaries (each a launch, a ramp and a drain) of
// the four-kernel sequence. The grid barriers are a counter in the workspace
// header with bounded waits: a CTA that gives up records COV_ETIMEOUT and
// skips the remaining work; no wait is unbounded.
//
// Memory visibility: data produced by other CTAs (partials, RV, CV) is read
// only after a grid barrier (release fence before the arrival, acquire load
// of the counter), and no CTA reads those addresses earlier in the launch, so
// no stale copy can sit in its L1.
#include <cuda.h>
#include <cuda_runtime.h>

#include "cov_launch.h"
#include "rec_fringe.cuh"
#include "rec_products.cuh"
#include "rec_reduce.cuh"

namespace cov {

// Workspace header words used by the fused kernel (all zeroed per call).
constexpr int kCtlBarrier = 1;  // grid barrier arrivals
constexpr int kCtlFringe = 2;   // next fringe-row task

// Grid-wide barrier: arrival `target / gridDim.x` of every CTA. Returns false
// (and records COV_ETIMEOUT) if the other CTAs do not arrive within the limit.
// Release/acquire only: the CTA barrier orders the CTA's writes before thread
// 0's release pattern (fence.acq_rel + the arrival), whose acquire load of the
// counter is ordered before the CTA's later reads by the closing CTA barrier.
__device__ __forceinline__ bool grid_barrier(unsigned *counter, unsigned target,
                                             unsigned *status) {
  __syncthreads();
  int failed = 0;
  if (threadIdx.x == 0) {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(counter) : "memory");
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0;; ++it) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(counter) : "memory");
      if (v >= target) break;
      if ((it & 15) == 15 && global_ns() - t0 > kWaitLimitNs) {
        atomicCAS(status, kDevOk, kDevTimeout);
        failed = 1;
        break;
      }
      __nanosleep(32);
    }
  }
  return __syncthreads_or(failed) == 0;
}

template <int G, int PITCH, int NCW, int QMAX>
__global__ void __launch_bounds__((NCW + 1) * 32, 1)
    k_fused(const RecParams p, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(1024) unsigned char smem_f[];
  __shared__ int task_s;
  unsigned *ctl = p.status;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // ---- 1. products over the inner rows ------------------------------------
  const long long NT = p.n_tasks;
  const long long tb = NT * blockIdx.x / gridDim.x;
  const long long te = NT * (blockIdx.x + 1) / gridDim.x;
  bool ok = true;
  if (p.n_inner > 0) ok = products_phase<float, G, 16, PITCH, NCW>(p, tmap, smem_f, tb, te);
  ok = __syncthreads_and(ok) != 0;
  if (threadIdx.x == 0 && p.n_inner > 0 && tb < te) {
    // the barriers' memory is reused below
    const size_t bb = tile_buf_bytes<float, PITCH>(p.STR);
    uint64_t *bars = (uint64_t *)(smem_f + 2 * bb);
    for (int k = 0; k < 4; ++k)
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bars + k)) : "memory");
  }
  __syncthreads();

  // ---- 2. fringe rows x inner columns, tasks (side, chunk, pair block) ---
  // a task's (fringe row, row lag) pairs: at most one per thread, blocks of
  // equal size (finer tasks, four threads a pair, measured slower: their
  // extra shuffles and claims cost more than the shorter tail saves)
  const int npairs = (p.P - 1) * (2 * p.P - 1);
  const int npb = (npairs + (int)blockDim.x - 1) / (int)blockDim.x;
  const int n_ftasks = p.NFR > 0 ? 2 * p.NCH * npb : 0;
  float2 *S = (float2 *)smem_f;
  while (ok) {
    if (threadIdx.x == 0) task_s = (int)atomicAdd(&ctl[kCtlFringe], 1u);
    __syncthreads();
    const int task = task_s;
    __syncthreads();
    if (task >= n_ftasks) break;
    const int pb = task % npb, sc = task / npb;
    const int side = sc / p.NCH, cc = sc - side * p.NCH;
    fringe_stage<float>(p, S, side, cc);
    __syncthreads();
    const int t = (int)(((long long)npairs * pb) / npb) + threadIdx.x;
    if (t < (int)(((long long)npairs * (pb + 1)) / npb)) fringe_pair<float, QMAX, 8>(p, S, side, cc, t);
    __syncthreads();
  }

  // ---- 3. reductions (warp tasks) ------------------------------------------
  ok = grid_barrier(&ctl[kCtlBarrier], gridDim.x, p.status) && ok;
  if (ok) {
    // task w on warp w / gridDim.x of CTA w % gridDim.x: spread over all SMs
    const int total = reduce_tasks(p), nw = blockDim.x >> 5;
    for (int w = warp * (int)gridDim.x + (int)blockIdx.x; w < total; w += (int)gridDim.x * nw)
      reduce_task<float, QMAX>(p, w, lane);
  }

  // ---- 4. seed, walk and write the blocks of R -----------------------------
  ok = grid_barrier(&ctl[kCtlBarrier], 2 * gridDim.x, p.status) && ok;
  if (!ok) return;
  int nblk = 0;
  for (int dc = p.dc_lo; dc < p.dc_hi; ++dc) nblk += p.Q - dc;
  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
    int dc, bj;
    walk_block_of(p, b, dc, bj);
    walk_block<float>(p, dc, bj, smem_f);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <int G, int PITCH, int QMAX>
static cudaError_t launch_fused_t(const RecParams &p, const CUtensorMap &tmap, int num_sms,
                                  cudaStream_t s) {
  constexpr int NCW = 12;  // as the stand-alone product kernel
  auto kern = k_fused<G, PITCH, NCW, QMAX>;
  size_t smem = 2 * tile_buf_bytes<float, PITCH>(p.STR) + 64;
  const size_t fs = (size_t)(2 * p.P - 2) * p.FPITCH * sizeof(float2);
  const size_t ws = walk_smem_bytes<float>(p.P, p.NFR);
  if (fs > smem) smem = fs;
  if (ws > smem) smem = ws;
  cudaError_t e = ensure_smem_attr(kern, smem);
  if (e != cudaSuccess) return e;
  // one CTA per SM (the shared memory of the tile buffers), all co-resident
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, (NCW + 1) * 32, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorNotSupported;
  const int grid = num_sms;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((NCW + 1) * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, p, tmap);
}

// The pitch follows the tile width and Q (TC + 16 for Q <= 17, TC + 32
// above), QMAX the column-lag register count of the fringe tasks (>= Q).
template <int G, int PITCH>
static cudaError_t launch_fused_q(const RecParams &p, const CUtensorMap &tmap, int num_sms,
                                  cudaStream_t s) {
  if constexpr (PITCH == 64 || PITCH == 96) {
    return launch_fused_t<G, PITCH, 32>(p, tmap, num_sms, s);
  } else {
    switch (p.QMAXF) {
      case 4:
      case 8: return launch_fused_t<G, PITCH, 8>(p, tmap, num_sms, s);
      case 16: return launch_fused_t<G, PITCH, 16>(p, tmap, num_sms, s);
      case 32: return launch_fused_t<G, PITCH, 32>(p, tmap, num_sms, s);
    }
    return cudaErrorNotSupported;
  }
}

template <int G>
static cudaError_t launch_fused_g(const RecParams &p, const CUtensorMap &tmap, int num_sms,
                                  cudaStream_t s) {
  switch (p.PITCH) {
    case 48: return launch_fused_q<G, 48>(p, tmap, num_sms, s);
    case 64: return launch_fused_q<G, 64>(p, tmap, num_sms, s);
    case 80: return launch_fused_q<G, 80>(p, tmap, num_sms, s);
    case 96: return launch_fused_q<G, 96>(p, tmap, num_sms, s);
  }
  return cudaErrorNotSupported;
}

bool fused_supported(const RecParams &p, bool fp64) {
  return !fp64 && (p.G == 4 || p.G == 8 || p.G == 16) &&
         (p.PITCH == 48 || p.PITCH == 64 || p.PITCH == 80 || p.PITCH == 96);
}

cudaError_t launch_fused(const RecParams &p, const CUtensorMap &tmap, int num_sms, cudaStream_t s) {
  switch (p.G) {
    case 4: return launch_fused_g<4>(p, tmap, num_sms, s);
    case 8: return launch_fused_g<8>(p, tmap, num_sms, s);
    case 16: return launch_fused_g<16>(p, tmap, num_sms, s);
  }
  return cudaErrorNotSupported;
}

}  // namespace cov
