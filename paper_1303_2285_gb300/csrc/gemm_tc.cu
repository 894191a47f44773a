// Dense contraction form on tcgen05 tensor cores: R = X X^H / K with X the
// block-Hankel data matrix (column w = the column stack of window w; Eq. 2.2).
//
// Real form: Y = [Re X; Im X] (2PQ x K) and B = Y Y^T, so that
//   Re R[a][b] = B[a][b] + B[D+a][D+b],  Im R[a][b] = B[D+a][b] - B[a][D+b].
// B is symmetric; only its upper 128 x 128 tiles are formed. A CTA owns one
// tile and one range of the windows (split-K). Per K-step of 32 windows (one
// window row p, 32 consecutive q) the A region those windows read (P rows x
// 32+Q-1 columns) is staged by one TMA load into a 3-deep ring, two steps
// ahead; all threads then build the operand tiles in shared memory from it
// (K-major core-matrix layout, no swizzle) with each value split into TF32
// hi + lo; one thread issues the three products hi*hi + hi*lo + lo*hi as
// tcgen05.mma kind::tf32 (M = N = 128, K = 8) and commits them to an
// mbarrier, while the other threads build the next stage. Accumulation runs
// in TMEM: chunk accumulators of 4 K-steps alternate between two 128-column
// regions and are added (FP32, round to nearest, tcgen05.ld / st) into a
// third region, the running sum. A second kernel sums the K-split partials
// in a fixed order (FP64) and assembles R. Shapes whose region does not fit
// the ring build the operands from A in global memory instead.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/cov.h"
#include "cov_device.cuh"
#include "cov_launch.h"
#include "cov_internal.h"
#include "plan.h"

namespace cov {

constexpr int kGT = 128;         // tile rows / columns of B
constexpr int kGKW = 32;         // windows per K-step (TF32: 128-byte rows)
constexpr int kGThreads = 256;
constexpr int kGTileBytes = kGT * kGKW * 4;  // 16 KB per operand tile
constexpr unsigned long long kGWaitNs = 2000000000ull;
constexpr int kGRegStages = 3;             // A regions in flight
constexpr int kGRegMaxBytes = 16384;       // one region: P rows x RWf floats
constexpr unsigned kGRunCol = 256;         // TMEM columns of the running sum

struct GemmParams {
  const float2 *A;
  long long lda;
  int N, M, P, Q, D, W, Hn;
  int nt, ntiles, qsteps, nsplit;
  long long nsteps;
  float *part;  // [nsplit][ntiles][128][128]
  unsigned *status;
  float2 *R;
  long long K;
  int mean;
  int use_tma, RWf;  // A region per K-step: P rows x RWf floats, staged by TMA
};

__device__ __forceinline__ uint64_t smem_desc(unsigned addr) {
  // K-major, no swizzle: core matrices of 8 rows x 16 bytes; 128 B between
  // core matrices along K (leading), 1024 B along M/N (stride); version 1.
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((1024u >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ float tf32_rna(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// upper tile index t -> (ti, tj), ti <= tj
__device__ __forceinline__ void tile_of(int t, int nt, int &ti, int &tj) {
  int i = 0, rem = t;
  while (rem >= nt - i) {
    rem -= nt - i;
    ++i;
  }
  ti = i;
  tj = i + rem;
}

// One thread's four (row, 4-window chunk) items of an operand tile: rows are
// fixed for the whole kernel, so their (component, i, j) are decoded once.
struct GItem {
  int ok, comp, i, col, qoff, soff;  // col: A column of the chunk's first window; soff: tile offset
};

__device__ __forceinline__ void build_items(const GemmParams &p, int tile_row0, GItem (&it)[4]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int item = threadIdx.x + u * kGThreads;  // 1024 items: 128 rows x 8 chunks
    const int r8 = item & 7, chunk = (item >> 3) & 7, rg = item >> 6;
    const int row = rg * 8 + r8;
    const int r = tile_row0 + row;
    it[u].soff = rg * 256 + chunk * 32 + r8 * 4;  // (rg*1024 + chunk*128 + r8*16) bytes / 4
    it[u].ok = r < 2 * p.D;
    const int a = r % p.D;
    it[u].comp = r >= p.D ? 1 : 0;
    it[u].i = a % p.P;
    it[u].qoff = chunk * 4;            // first window of the chunk, relative to q0
    it[u].col = a / p.P + chunk * 4;   // A column of that window for element (i, j)
  }
}

__device__ __forceinline__ void fill_tile(const GemmParams &p, const GItem (&it)[4], int pw, int q0,
                                          float *hi, float *lo) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (it[u].ok) {
      const float2 *src = p.A + (long long)(pw + it[u].i) * p.lda + q0 + it[u].col;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (q0 + it[u].qoff + e < p.W) {  // window q must exist
          const float2 x = __ldg(src + e);
          v[e] = it[u].comp ? x.y : x.x;
        }
      }
    }
    float4 h, l;
    h.x = tf32_rna(v[0]);
    h.y = tf32_rna(v[1]);
    h.z = tf32_rna(v[2]);
    h.w = tf32_rna(v[3]);
    l.x = tf32_rna(v[0] - h.x);
    l.y = tf32_rna(v[1] - h.y);
    l.z = tf32_rna(v[2] - h.z);
    l.w = tf32_rna(v[3] - h.w);
    *(float4 *)(hi + it[u].soff) = h;
    *(float4 *)(lo + it[u].soff) = l;
  }
}

// The same operand tile from the staged A region: reg[r * RWf + 2c + comp]
// holds component comp of A[pw + r][q0 + c].
__device__ __forceinline__ void fill_tile_smem(const GemmParams &p, const GItem (&it)[4], int q0,
                                               const float *reg, float *hi, float *lo) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (it[u].ok) {
      const float *src = reg + it[u].i * p.RWf + 2 * it[u].col + it[u].comp;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (q0 + it[u].qoff + e < p.W) v[e] = src[2 * e];  // window q must exist
    }
    float4 h, l;
    h.x = tf32_rna(v[0]);
    h.y = tf32_rna(v[1]);
    h.z = tf32_rna(v[2]);
    h.w = tf32_rna(v[3]);
    l.x = tf32_rna(v[0] - h.x);
    l.y = tf32_rna(v[1] - h.y);
    l.z = tf32_rna(v[2] - h.z);
    l.w = tf32_rna(v[3] - h.w);
    *(float4 *)(hi + it[u].soff) = h;
    *(float4 *)(lo + it[u].soff) = l;
  }
}

__device__ __forceinline__ void mma_tf32(unsigned tmem, uint64_t ad, uint64_t bd, unsigned idesc,
                                         unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

// TMEM accumulators hold at most kGChunk K-steps: the tensor core's FP32
// accumulation is not round-to-nearest, so long chains drift. Chunks
// alternate between two accumulators; each finished chunk is added (FP32,
// round to nearest) into the running sum one chunk later, while the tensor
// core works on the other accumulator.
constexpr int kGChunk = 4;

#define COV_R32(r)                                                                              \
  "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),          \
      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), \
      "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),           \
      "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),           \
      "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
#define COV_W32(r)                                                                             \
  "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),      \
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),        \
      "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),      \
      "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),      \
      "r"(r[29]), "r"(r[30]), "r"(r[31])

__device__ __forceinline__ void tmem_ld32(unsigned taddr, unsigned (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : COV_R32(r)
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st32(unsigned taddr, const unsigned (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      COV_W32(r)
      : "memory");
}

// Adds TMEM accumulator `acc_col` (128 x 128 FP32) into the running sum
// (`first`: copies it): warp w takes lane quadrant w % 4 and column half w / 4.
__device__ __forceinline__ void flush_acc(unsigned tmem, unsigned acc_col, bool first) {
  const int warp = threadIdx.x >> 5;
  const int quad = warp & 3, half = warp >> 2;
  const unsigned lanes = (unsigned)(quad * 32) << 16;
#pragma unroll 1
  for (int c0 = half * 64; c0 < half * 64 + 64; c0 += 32) {
    unsigned r[32], s[32];
    tmem_ld32(tmem + lanes + acc_col + (unsigned)c0, r);
    if (!first) tmem_ld32(tmem + lanes + kGRunCol + (unsigned)c0, s);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (!first) {
#pragma unroll
      for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) + __uint_as_float(s[j]));
    }
    tmem_st32(tmem + lanes + kGRunCol + (unsigned)c0, r);
  }
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(kGThreads, 1)
    k_gemm_tf32x3(const GemmParams p, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(1024) unsigned char smem_g[];
  // two stages x [A_hi, A_lo, B_hi, B_lo], the A-region ring, then the
  // barriers and the TMEM address
  float *stage_base = (float *)smem_g;
  float *reg_base = (float *)(smem_g + 2 * 4 * kGTileBytes);
  uint64_t *bars = (uint64_t *)((unsigned char *)reg_base + kGRegStages * kGRegMaxBytes);
  uint64_t *mma_done = bars;        // [2] per smem stage
  uint64_t *chunk_done = bars + 2;  // [2] per TMEM accumulator
  uint64_t *reg_full = bars + 4;    // [3] per region stage
  unsigned *tmem_slot = (unsigned *)(bars + 4 + kGRegStages);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x % p.ntiles, split = blockIdx.x / p.ntiles;
  int ti, tj;
  tile_of(tile, p.nt, ti, tj);
  const bool diag = ti == tj;
  const long long s0 = p.nsteps * split / p.nsplit, s1 = p.nsteps * (split + 1) / p.nsplit;
  const long long nk = s1 - s0;
  const unsigned reg_bytes = (unsigned)(p.P * p.RWf * 4);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int b = 0; b < 4 + kGRegStages; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tmem_slot;

  // the A region of K-step k (TMA, complete_tx on reg_full[k % 3])
  auto issue_region = [&](long long k) {
    const long long step = s0 + k;
    const int pw = (int)(step / p.qsteps), q0 = (int)(step % p.qsteps) * kGKW;
    const int b = (int)(k % kGRegStages);
    mbar_arrive_expect_tx(&reg_full[b], reg_bytes);
    tma_load_2d((unsigned char *)reg_base + b * kGRegMaxBytes, &tmap, 2 * q0, pw, &reg_full[b]);
  };
  long long issued = 0;
  if (p.use_tma && tid == 0)
    for (; issued < 2 && issued < nk; ++issued) issue_region(issued);

  GItem ia[4], ib[4];
  build_items(p, ti * kGT, ia);
  build_items(p, tj * kGT, ib);
  // D = f32 (bit 4), A = B = tf32 (2), both K-major, N = 128, M = 128
  const unsigned idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
  bool ok = true;
  long long k = 0;
  for (; k < nk; ++k) {
    const long long step = s0 + k;
    const int st = (int)(k & 1);
    const long long chunk = k / kGChunk;
    const bool chunk_start = (k % kGChunk) == 0;
    bool w = true;
    if (k >= 2) w = mbar_wait(&mma_done[st], (unsigned)(((k >> 1) - 1) & 1), kGWaitNs);
    if (chunk_start && chunk >= 2) {
      // chunk - 2 used the accumulator this chunk is about to reuse: add it in
      const long long c = chunk - 2;
      w = w && mbar_wait(&chunk_done[c & 1], (unsigned)((c >> 1) & 1), kGWaitNs);
    }
    if (p.use_tma)
      w = w && mbar_wait(&reg_full[k % kGRegStages], (unsigned)((k / kGRegStages) & 1), kGWaitNs);
    // the CTA agrees on the outcome, so that a timeout leaves the loop in all
    // threads together
    if (__syncthreads_or(!w)) {
      ok = false;
      break;
    }
    if (chunk_start && chunk >= 2) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      flush_acc(tmem, (unsigned)((chunk - 2) & 1) * 128, chunk == 2);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    float *ahi = stage_base + st * 4 * (kGTileBytes / 4);
    float *alo = ahi + kGTileBytes / 4;
    float *bhi = alo + kGTileBytes / 4;
    float *blo = bhi + kGTileBytes / 4;
    const int pw = (int)(step / p.qsteps), q0 = (int)(step % p.qsteps) * kGKW;
    if (p.use_tma) {
      const float *reg = (const float *)((const unsigned char *)reg_base +
                                         (k % kGRegStages) * kGRegMaxBytes);
      fill_tile_smem(p, ia, q0, reg, ahi, alo);
      if (!diag) fill_tile_smem(p, ib, q0, reg, bhi, blo);
    } else {
      fill_tile(p, ia, pw, q0, ahi, alo);
      if (!diag) fill_tile(p, ib, pw, q0, bhi, blo);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned uah = smem_u32(ahi), ual = smem_u32(alo);
      const unsigned ubh = diag ? uah : smem_u32(bhi), ubl = diag ? ual : smem_u32(blo);
      const unsigned dacc = tmem + (unsigned)(chunk & 1) * 128;
#pragma unroll
      for (int s = 0; s < kGKW / 8; ++s) {
        const unsigned o = s * 256;  // two core matrices (8 TF32) along K per MMA
        const unsigned acc0 = (!chunk_start || s > 0) ? 1u : 0u;
        mma_tf32(dacc, smem_desc(uah + o), smem_desc(ubh + o), idesc, acc0);
        mma_tf32(dacc, smem_desc(uah + o), smem_desc(ubl + o), idesc, 1u);
        mma_tf32(dacc, smem_desc(ual + o), smem_desc(ubh + o), idesc, 1u);
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&mma_done[st]))
          : "memory");
      if ((k % kGChunk) == kGChunk - 1 || k == nk - 1)
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&chunk_done[chunk & 1]))
            : "memory");
      // the region two steps ahead reuses the buffer step k - 1 read, which
      // every thread finished before the barrier above
      if (p.use_tma && issued < nk && issued == k + 2) issue_region(issued++);
    }
  }
  // add in the last one or two chunks
  if (ok && nk > 0) {
    const long long last = (nk - 1) / kGChunk;
    for (long long c = (last >= 1 ? last - 1 : 0); c <= last; ++c) {
      const bool w = mbar_wait(&chunk_done[c & 1], (unsigned)((c >> 1) & 1), kGWaitNs);
      if (__syncthreads_or(!w)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      flush_acc(tmem, (unsigned)(c & 1) * 128, c == 0);
    }
  }
  if (p.use_tma) {
    // regions issued but not consumed (only after a timeout): let them land
    // before the CTA exits
    const long long n_issued = __shfl_sync(0xffffffffu, issued, 0);
    for (long long r = k; r < n_issued && warp == 0; ++r)
      mbar_wait(&reg_full[r % kGRegStages], (unsigned)((r / kGRegStages) & 1), kGWaitNs);
  }
  if (!ok && tid == 0) *p.status = kDevTimeout;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // partial tile (row-major 128 x 128 floats) from the running sum
  float *out = p.part + ((long long)split * p.ntiles + tile) * (kGT * kGT);
  {
    const int quad = warp & 3, half = warp >> 2;
    const int row = quad * 32 + lane;
#pragma unroll 1
    for (int c0 = half * 64; c0 < half * 64 + 64; c0 += 32) {
      unsigned r[32];
      if (nk > 0 && ok) {
        tmem_ld32(tmem + ((unsigned)(quad * 32) << 16) + kGRunCol + (unsigned)c0, r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) r[j] = 0u;
      }
      float4 *dst = (float4 *)(out + (long long)row * kGT + c0);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        dst[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                             __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
}

// B(r, c) from the upper tiles of split s (B is symmetric).
__device__ __forceinline__ float bval(const GemmParams &p, int s, int r, int c) {
  if (r > c) {
    const int t = r;
    r = c;
    c = t;
  }
  const int ti = r / kGT, tj = c / kGT;
  const int t = ti * p.nt - ti * (ti - 1) / 2 + (tj - ti);
  return p.part[((long long)s * p.ntiles + t) * (kGT * kGT) + (long long)(r % kGT) * kGT + (c % kGT)];
}

__global__ void __launch_bounds__(256) k_gemm_assemble(const GemmParams p) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long DD = (long long)p.D * p.D;
  if (e >= DD) return;
  const int a = (int)(e / p.D), b = (int)(e % p.D);
  double re = 0.0, im = 0.0;
  for (int s = 0; s < p.nsplit; ++s) {
    re += (double)bval(p, s, a, b) + (double)bval(p, s, p.D + a, p.D + b);
    im += (double)bval(p, s, p.D + a, b) - (double)bval(p, s, a, p.D + b);
  }
  if (p.mean) {
    re /= (double)p.K;
    im /= (double)p.K;
  }
  if (a == b) im = 0.0;
  p.R[e] = make_float2((float)re, (float)im);
}

}  // namespace cov

namespace cov {

bool gemm_shape_ok(long long N, long long M, int P, int Q) {
  return (long long)P * Q <= 1024 && N < (1LL << 30) && M < (1LL << 30);
}

static void gemm_plan(long long N, long long M, int P, int Q, int sms, GemmParams &g, size_t &ws) {
  memset(&g, 0, sizeof(g));
  g.N = (int)N;
  g.M = (int)M;
  g.P = P;
  g.Q = Q;
  g.D = P * Q;
  g.W = (int)(M - Q + 1);
  g.Hn = (int)(N - P + 1);
  g.K = (long long)g.W * g.Hn;
  g.nt = (2 * g.D + kGT - 1) / kGT;
  g.ntiles = g.nt * (g.nt + 1) / 2;
  g.qsteps = (g.W + kGKW - 1) / kGKW;
  g.nsteps = (long long)g.Hn * g.qsteps;
  int ns = sms / g.ntiles;
  if (ns < 1) ns = 1;
  if (ns > g.nsteps) ns = (int)g.nsteps;
  g.nsplit = ns;
  ws = kWsHeader + (((size_t)g.nsplit * g.ntiles * kGT * kGT * 4 + 255) & ~(size_t)255);
}

// The workspace is sized for up to kGMaxSms SMs (K-splits per tile follow the
// SM count), so that its size does not depend on the device.
constexpr int kGMaxSms = 160;

size_t gemm_workspace_size(long long N, long long M, int P, int Q) {
  GemmParams g;
  size_t ws;
  gemm_plan(N, M, P, Q, kGMaxSms, g, ws);
  return ws;
}

cudaError_t launch_gemm_tf32x3(const void *A, long long N, long long M, long long lda, int P, int Q,
                               void *R, int mean, void *workspace, size_t ws_bytes, int sms,
                               cudaStream_t s, bool *ws_ok) {
  GemmParams g;
  size_t need;
  gemm_plan(N, M, P, Q, sms < kGMaxSms ? sms : kGMaxSms, g, need);
  *ws_ok = workspace && ws_bytes >= gemm_workspace_size(N, M, P, Q) &&
           ((uintptr_t)workspace & 255) == 0;
  if (!*ws_ok) return cudaSuccess;
  g.A = (const float2 *)A;
  g.lda = lda;
  g.part = (float *)((char *)workspace + kWsHeader);
  g.status = (unsigned *)workspace;
  g.R = (float2 *)R;
  g.mean = mean;
  // the A region of a K-step (P rows, 32 + Q - 1 complex columns) by TMA when
  // it fits the ring and A meets TMA's alignment; else operands from global
  g.RWf = ((2 * (kGKW + Q - 1)) + 3) / 4 * 4;
  if (g.RWf % 32 == 0) g.RWf += 4;  // region rows of one warp's reads in different banks
  CUtensorMap tmap;
  memset(&tmap, 0, sizeof(tmap));
  g.use_tma = (size_t)P * g.RWf * 4 <= (size_t)kGRegMaxBytes && g.RWf <= 256 && P <= 256 &&
              ((uintptr_t)A & 15) == 0 && ((lda * 8) & 15) == 0 &&
              encode_tiled_2d(tmap, false, A, (unsigned long long)(2 * M), (unsigned long long)N,
                              (unsigned long long)(lda * 8), (unsigned)g.RWf, (unsigned)P)
                  ? 1 : 0;
  const size_t smem = 2 * 4 * kGTileBytes + (size_t)kGRegStages * kGRegMaxBytes + 128;
  static bool attr_done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !attr_done[dev]) {
    e = cudaFuncSetAttribute(k_gemm_tf32x3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_done[dev] = true;
  }
  if ((e = cudaMemsetAsync(workspace, 0, 4, s)) != cudaSuccess) return e;
  k_gemm_tf32x3<<<g.ntiles * g.nsplit, kGThreads, smem, s>>>(g, tmap);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const long long DD = (long long)g.D * g.D;
  k_gemm_assemble<<<(unsigned)((DD + 255) / 256), 256, 0, s>>>(g);
  return cudaGetLastError();
}

}  // namespace cov
