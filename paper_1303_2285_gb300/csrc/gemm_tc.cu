// Dense contraction form on tcgen05 tensor cores: R = X X^H / K with X the
// block-Hankel data matrix (column w = the column stack of window w; Eq. 2.2).
//
// Real form: Y = [Re X; Im X] (2PQ x K) and B = Y Y^T, so that
//   Re R[a][b] = B[a][b] + B[D+a][D+b],  Im R[a][b] = B[D+a][b] - B[a][D+b].
// B is symmetric; only its upper 128 x 128 tiles are formed. A CTA owns one
// tile and one range of the windows (split-K), and is warp-specialised:
//  - eight filler warps build the operand tiles of each K-step (16 windows:
//    one window row p, 16 consecutive q) in shared memory (K-major
//    core-matrix layout, no swizzle), each value split into TF32 hi + lo,
//    from the A region those windows read (P rows x 16+Q-1 columns), which a
//    TMA load stages into a ring of up to 12 slots, as many steps ahead; a
//    stage is handed over by one mbarrier arrival per warp;
//  - one thread of the ninth warp issues the three products hi*hi + hi*lo +
//    lo*hi as tcgen05.mma kind::tf32 (M = N = 128, K = 8) and commits each
//    stage back to its fillers, four stages deep.
// Accumulation runs in TMEM: chunk accumulators of 8 K-steps alternate
// between two 128-column regions; the filler warps add each finished chunk
// (FP32, round to nearest, tcgen05.ld / st) into a third region, the running
// sum, half a chunk later, before the accumulator is reused. A second kernel
// sums the K-split partials in a fixed order (FP64) and assembles R. Shapes
// whose region does not fit the ring build the operands from A in global
// memory instead.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/cov.h"
#include "cov_device.cuh"
#include "cov_launch.h"
#include "cov_internal.h"
#include "smem_attr.h"
#include "plan.h"

namespace cov {

constexpr int kGT = 128;         // tile rows / columns of B
constexpr int kGKW = 16;         // windows per K-step (TF32: 64-byte rows)
constexpr int kGStages = 4;      // operand stages in flight
constexpr int kGFillWarps = 8;   // operand builders; one more warp issues the MMAs
constexpr int kGFillThreads = kGFillWarps * 32;
constexpr int kGThreads = kGFillThreads + 32;
// Operand formats: TF32x3 (two TF32 parts per value, products hh + hl + lh,
// K = 8 per MMA) and BF16x3 (three BF16 parts hi, mid, lo; products hh +
// hm + mh + mm + hl + lh, K = 16 per MMA). A stage holds the parts of A and
// of B, each a 128 x 16 tile.
template <bool BF> struct GFmt {
  static constexpr int kElem = BF ? 2 : 4;
  static constexpr int kParts = BF ? 3 : 2;
  static constexpr int kTileBytes = kGT * kGKW * kElem;  // 4 KB (BF16), 8 KB (TF32)
  static constexpr int kStageBytes = 2 * kParts * kTileBytes;
  static constexpr unsigned kSBO = 8 * kGKW * kElem;      // bytes between 8-row groups
};
constexpr int kGStageBytesMax = GFmt<false>::kStageBytes;  // 32 KB
constexpr unsigned long long kGWaitNs = 2000000000ull;
constexpr int kGRegMaxStages = 12;         // A regions in flight (at most)
constexpr int kGRegRingBytes = 49152;      // the region ring
constexpr int kGRegMaxBytes = 16384;       // one region: P rows x RWf floats
constexpr unsigned kGRunCol = 256;         // TMEM columns of the running sum
constexpr int kGBars = 2 * kGStages + 2 + 2 * kGRegMaxStages + 1;
constexpr size_t kGSmemBytes = (size_t)kGStages * kGStageBytesMax + (size_t)kGRegRingBytes + 512;

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
  int RS, RSLOT;     // region slots in the ring (RS steps of prefetch) and slot bytes
};

__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned sbo) {
  // K-major, no swizzle: core matrices of 8 rows x 16 bytes; 128 B between
  // core matrices along K (leading), `sbo` bytes along M/N (stride: the core
  // matrices of a 16-window row group: 4 for TF32, 2 for BF16); version 1.
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
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

// One filler thread's two (row, 4-window chunk) items of an operand tile:
// rows are fixed for the whole kernel, so their (component, i, j) are decoded
// once.
struct GItem {
  int ok, comp, i, col, qoff, soff;  // col: A column of the chunk's first window; soff: tile byte offset
};

template <bool BF>
__device__ __forceinline__ void build_items(const GemmParams &p, int tile_row0, GItem (&it)[2]) {
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    // 512 items: 128 rows x 4 chunks; a warp's lanes take 32 consecutive rows
    // of one chunk (their region reads then meet at most two to a bank)
    const int item = threadIdx.x + u * kGFillThreads;
    const int r8 = item & 7, chunk = (item >> 5) & 3, rg = ((item >> 7) << 2) | ((item >> 3) & 3);
    const int row = rg * 8 + r8;
    const int r = tile_row0 + row;
    // K-major core matrices of 8 rows x 16 bytes: a 4-window chunk is one
    // core matrix column (TF32) or half of one (BF16)
    it[u].soff = BF ? rg * 256 + (chunk >> 1) * 128 + r8 * 16 + (chunk & 1) * 8
                    : rg * 512 + chunk * 128 + r8 * 16;
    it[u].ok = r < 2 * p.D;
    const int a = r % p.D;
    it[u].comp = r >= p.D ? 1 : 0;
    it[u].i = a % p.P;
    it[u].qoff = chunk * 4;            // first window of the chunk, relative to q0
    it[u].col = a / p.P + chunk * 4;   // A column of that window for element (i, j)
  }
}

// The split parts of four consecutive values into the part tiles at dst
// (part k at dst + k * tile bytes), at byte offset soff.
//  TF32: hi = the value rounded to TF32, lo = the rest rounded to TF32.
//  BF16: hi = RN_bf16(x), mid = RN_bf16(x - hi), lo = RN_bf16(x - hi - mid)
//        (each difference exact in FP32).
template <bool BF>
__device__ __forceinline__ void store_parts(const float (&v)[4], unsigned char *dst, int soff) {
  if constexpr (BF) {
    unsigned short h[4], m[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const __nv_bfloat16 bh = __float2bfloat16_rn(v[e]);
      const float r1 = v[e] - __bfloat162float(bh);
      const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
      const float r2 = r1 - __bfloat162float(bm);
      h[e] = __bfloat16_as_ushort(bh);
      m[e] = __bfloat16_as_ushort(bm);
      l[e] = __bfloat16_as_ushort(__float2bfloat16_rn(r2));
    }
    constexpr int T = GFmt<true>::kTileBytes;
    *(uint2 *)(dst + soff) = make_uint2(h[0] | ((unsigned)h[1] << 16), h[2] | ((unsigned)h[3] << 16));
    *(uint2 *)(dst + T + soff) = make_uint2(m[0] | ((unsigned)m[1] << 16), m[2] | ((unsigned)m[3] << 16));
    *(uint2 *)(dst + 2 * T + soff) =
        make_uint2(l[0] | ((unsigned)l[1] << 16), l[2] | ((unsigned)l[3] << 16));
  } else {
    float4 h, l;
    h.x = tf32_rna(v[0]);
    h.y = tf32_rna(v[1]);
    h.z = tf32_rna(v[2]);
    h.w = tf32_rna(v[3]);
    l.x = tf32_rna(v[0] - h.x);
    l.y = tf32_rna(v[1] - h.y);
    l.z = tf32_rna(v[2] - h.z);
    l.w = tf32_rna(v[3] - h.w);
    *(float4 *)(dst + soff) = h;
    *(float4 *)(dst + GFmt<false>::kTileBytes + soff) = l;
  }
}

template <bool BF>
__device__ __forceinline__ void fill_tile(const GemmParams &p, const GItem (&it)[2], int pw, int q0,
                                          unsigned char *dst) {
#pragma unroll
  for (int u = 0; u < 2; ++u) {
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
    store_parts<BF>(v, dst, it[u].soff);
  }
}

// The same operand tile from the staged A region: reg[r * RWf + 2c + comp]
// holds component comp of A[pw + r][q0 + c].
template <bool BF>
__device__ __forceinline__ void fill_tile_smem(const GemmParams &p, const GItem (&it)[2], int q0,
                                               const float *reg, unsigned char *dst) {
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (it[u].ok) {
      const float *src = reg + it[u].i * p.RWf + 2 * it[u].col + it[u].comp;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (q0 + it[u].qoff + e < p.W) v[e] = src[2 * e];  // window q must exist
    }
    store_parts<BF>(v, dst, it[u].soff);
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
// kind::f16 with A and B both BF16 (K = 16), FP32 accumulation
__device__ __forceinline__ void mma_bf16(unsigned tmem, uint64_t ad, uint64_t bd, unsigned idesc,
                                         unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

// TMEM accumulators hold at most kGChunk K-steps (128 windows): the tensor
// core's FP32 accumulation is not round-to-nearest, so long chains drift.
// Chunks alternate between two accumulators; each finished chunk is added
// (FP32, round to nearest) into the running sum while the tensor core works
// on the other accumulator.
constexpr int kGChunk = 8;

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
// (`first`: copies it): filler warp w takes lane quadrant w % 4 and column
// half w / 4.
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

template <bool BF>
__global__ void __launch_bounds__(kGThreads, 1)
    k_gemm_split(const GemmParams p, const __grid_constant__ CUtensorMap tmap) {
  using F = GFmt<BF>;
  extern __shared__ __align__(1024) unsigned char smem_g[];
  // operand stages x [A parts, B parts], the A-region ring, then the
  // barriers and the TMEM address
  unsigned char *stage_base = smem_g;
  unsigned char *reg_base = smem_g + kGStages * kGStageBytesMax;
  uint64_t *bars = (uint64_t *)(reg_base + kGRegRingBytes);
  uint64_t *full = bars;                          // [stages] built: one arrival per filler warp
  uint64_t *empty = full + kGStages;              // [stages] read by the tensor core (commit)
  uint64_t *chunk_done = empty + kGStages;        // [2] a chunk accumulator is complete (commit)
  uint64_t *reg_full = chunk_done + 2;              // [RS] A region landed (TMA)
  uint64_t *reg_empty = reg_full + kGRegMaxStages;  // [RS] A region read by every filler warp
  uint64_t *mma_fin = reg_empty + kGRegMaxStages;   // every issued MMA has completed
  unsigned *tmem_slot = (unsigned *)(bars + kGBars);
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
    for (int b = 0; b < kGStages; ++b) {
      mbar_init(&full[b], kGFillWarps);
      mbar_init(&empty[b], 1);
    }
    mbar_init(&chunk_done[0], 1);
    mbar_init(&chunk_done[1], 1);
    for (int b = 0; b < kGRegMaxStages; ++b) {
      mbar_init(&reg_full[b], 1);
      mbar_init(&reg_empty[b], kGFillWarps);
    }
    mbar_init(mma_fin, 1);
    fence_mbar_init();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tmem_slot;
  bool ok = true;

  if (warp < kGFillWarps) {
    // ---- filler warps ------------------------------------------------------
    // the A region of K-step k into ring slot b (TMA, complete_tx on reg_full)
    auto issue_region = [&](long long k, int b) {
      const long long step = s0 + k;
      const int rpw = (int)(step / p.qsteps), q0 = (int)(step % p.qsteps) * kGKW;
      mbar_arrive_expect_tx(&reg_full[b], reg_bytes);
      tma_load_2d(reg_base + b * p.RSLOT, &tmap, 2 * q0, rpw, &reg_full[b]);
    };
    long long issued = 0;  // thread 0 only
    if (p.use_tma && tid == 0)
      for (; issued < p.RS && issued < nk; ++issued) issue_region(issued, (int)issued);
    GItem ia[2], ib[2];
    build_items<BF>(p, ti * kGT, ia);
    build_items<BF>(p, tj * kGT, ib);
    long long flushed = 0;  // chunks added into the running sum
    // step k's ring slot and its phase parity, and its window row / column
    // step, kept incrementally (no divisions in the loop)
    int rslot = 0;
    unsigned rpar = 0;
    int pw = (int)(s0 / p.qsteps), qs = (int)(s0 % p.qsteps);
    long long k = 0;
    for (; k < nk; ++k) {
      const int st = (int)(k % kGStages);
      bool w = ok;
      // the tensor core has read this stage's previous operands
      if (w && k >= kGStages) w = mbar_wait(&empty[st], (unsigned)(((k / kGStages) - 1) & 1), kGWaitNs);
      if (w && p.use_tma) w = mbar_wait(&reg_full[rslot], rpar, kGWaitNs);
      // half a chunk into chunk c + 1, add chunk c into the running sum: its
      // accumulator is reused by chunk c + 2, whose first MMA waits for this
      // warp's arrival on the stage of step 8 (c + 2), issued after this
      if (w && (k % kGChunk) == kGChunk / 2 && k >= kGChunk + kGChunk / 2) {
        const long long c = flushed;  // == k / kGChunk - 1
        w = mbar_wait(&chunk_done[c & 1], (unsigned)((c >> 1) & 1), kGWaitNs);
        if (w) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          flush_acc(tmem, (unsigned)(c & 1) * 128, c == 0);
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          ++flushed;
        }
      }
      if (!__all_sync(0xffffffffu, w)) {
        ok = false;
        break;
      }
      unsigned char *apart = stage_base + st * F::kStageBytes;
      unsigned char *bpart = apart + F::kParts * F::kTileBytes;
      const int q0 = qs * kGKW;
      if (p.use_tma) {
        const float *reg = (const float *)(reg_base + rslot * p.RSLOT);
        fill_tile_smem<BF>(p, ia, q0, reg, apart);
        if (!diag) fill_tile_smem<BF>(p, ib, q0, reg, bpart);
      } else {
        fill_tile<BF>(p, ia, pw, q0, apart);
        if (!diag) fill_tile<BF>(p, ib, pw, q0, bpart);
      }
      // generic-proxy writes visible to the tensor core, then hand over
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&full[st]);
        if (p.use_tma) mbar_arrive(&reg_empty[rslot]);
      }
      // refill region k's slot with region k + RS once every filler warp has
      // read region k
      if (p.use_tma && tid == 0 && issued < nk) {
        if (mbar_wait(&reg_empty[rslot], rpar, kGWaitNs))
          issue_region(issued++, rslot);
        else
          ok = false;  // this warp leaves the loop at the next step
      }
      if (++rslot == p.RS) {
        rslot = 0;
        rpar ^= 1u;
      }
      if (++qs == p.qsteps) {
        qs = 0;
        ++pw;
      }
    }
    // add in the chunks not yet added
    if (ok && nk > 0) {
      const long long last = (nk - 1) / kGChunk;
      for (long long c = flushed; c <= last; ++c) {
        const bool w = mbar_wait(&chunk_done[c & 1], (unsigned)((c >> 1) & 1), kGWaitNs);
        if (!__all_sync(0xffffffffu, w)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        flush_acc(tmem, (unsigned)(c & 1) * 128, c == 0);
      }
    }
    if (p.use_tma && tid == 0) {
      // regions issued but not consumed (only after a timeout): let them land
      // before the CTA exits
      for (long long r = k; r < issued; ++r) {
        mbar_wait(&reg_full[rslot], rpar, kGWaitNs);
        if (++rslot == p.RS) {
          rslot = 0;
          rpar ^= 1u;
        }
      }
    }
  } else if (lane == 0) {
    // ---- MMA issuer -----------------------------------------------------------
    // D = f32 (bit 4), A = B = tf32 (2) or bf16 (1), both K-major, N = 128,
    // M = 128
    const unsigned fmt = BF ? 1u : 2u;
    const unsigned idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
    for (long long k = 0; k < nk; ++k) {
      const int st = (int)(k % kGStages);
      if (!mbar_wait(&full[st], (unsigned)((k / kGStages) & 1), kGWaitNs)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const long long chunk = k / kGChunk;
      const bool chunk_start = (k % kGChunk) == 0;
      const unsigned T = F::kTileBytes, sbo = F::kSBO;
      const unsigned ua0 = smem_u32(stage_base + st * F::kStageBytes);  // A part 0
      const unsigned ub0 = diag ? ua0 : ua0 + F::kParts * T;           // B part 0
      const unsigned dacc = tmem + (unsigned)(chunk & 1) * 128;
      if constexpr (BF) {
        // one K = 16 slice: hh + hm + mh + mm + hl + lh
        const unsigned acc0 = chunk_start ? 0u : 1u;
        mma_bf16(dacc, smem_desc(ua0, sbo), smem_desc(ub0, sbo), idesc, acc0);
        mma_bf16(dacc, smem_desc(ua0, sbo), smem_desc(ub0 + T, sbo), idesc, 1u);
        mma_bf16(dacc, smem_desc(ua0 + T, sbo), smem_desc(ub0, sbo), idesc, 1u);
        mma_bf16(dacc, smem_desc(ua0 + T, sbo), smem_desc(ub0 + T, sbo), idesc, 1u);
        mma_bf16(dacc, smem_desc(ua0, sbo), smem_desc(ub0 + 2 * T, sbo), idesc, 1u);
        mma_bf16(dacc, smem_desc(ua0 + 2 * T, sbo), smem_desc(ub0, sbo), idesc, 1u);
      } else {
#pragma unroll
        for (int s = 0; s < kGKW / 8; ++s) {
          const unsigned o = s * 256;  // two core matrices (8 TF32) along K per MMA
          const unsigned acc0 = (!chunk_start || s > 0) ? 1u : 0u;
          mma_tf32(dacc, smem_desc(ua0 + o, sbo), smem_desc(ub0 + o, sbo), idesc, acc0);
          mma_tf32(dacc, smem_desc(ua0 + o, sbo), smem_desc(ub0 + T + o, sbo), idesc, 1u);
          mma_tf32(dacc, smem_desc(ua0 + T + o, sbo), smem_desc(ub0 + o, sbo), idesc, 1u);
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&empty[st]))
          : "memory");
      if ((k % kGChunk) == kGChunk - 1 || k == nk - 1)
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&chunk_done[chunk & 1]))
            : "memory");
    }
    // every MMA issued (also after a timeout) completes before TMEM is read
    // back and freed
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(mma_fin))
        : "memory");
    if (!mbar_wait(mma_fin, 0u, kGWaitNs)) ok = false;
  }
  __syncwarp();  // each warp converged again before the CTA barriers below
  if (!ok) *p.status = kDevTimeout;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // partial tile (row-major 128 x 128 floats) from the running sum
  if (warp < kGFillWarps) {
    float *out = p.part + ((long long)split * p.ntiles + tile) * (kGT * kGT);
    const int quad = warp & 3, half = warp >> 2;
    const int row = quad * 32 + lane;
    const bool have = __all_sync(0xffffffffu, ok) && nk > 0;
#pragma unroll 1
    for (int c0 = half * 64; c0 < half * 64 + 64; c0 += 32) {
      unsigned r[32];
      if (have) {
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

template <bool BF>
static cudaError_t launch_gemm_split(const void *A, long long N, long long M, long long lda, int P,
                                     int Q, void *R, int mean, void *workspace, size_t ws_bytes,
                                     int sms, cudaStream_t s, bool *ws_ok) {
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
  // the A region of a K-step (P rows, 16 + Q - 1 complex columns) by TMA when
  // it fits the ring and A meets TMA's alignment; else operands from global
  g.RWf = ((2 * (kGKW + Q - 1)) + 3) / 4 * 4;
  if (g.RWf % 8 == 0) g.RWf += 4;  // = 4 mod 8: a warp's region reads two to a bank at most
  CUtensorMap tmap;
  memset(&tmap, 0, sizeof(tmap));
  g.use_tma = (size_t)P * g.RWf * 4 <= (size_t)kGRegMaxBytes && g.RWf <= 256 && P <= 256 &&
              ((uintptr_t)A & 15) == 0 && ((lda * 8) & 15) == 0 &&
              encode_tiled_2d(tmap, false, A, (unsigned long long)(2 * M), (unsigned long long)N,
                              (unsigned long long)(lda * 8), (unsigned)g.RWf, (unsigned)P)
                  ? 1 : 0;
  // ring slots: 128-byte aligned, as many as the ring holds (at most 12)
  g.RSLOT = (int)(((size_t)P * g.RWf * 4 + 127) & ~(size_t)127);
  g.RS = g.RSLOT > 0 ? kGRegRingBytes / g.RSLOT : 0;
  if (g.RS > kGRegMaxStages) g.RS = kGRegMaxStages;
  if (g.RS < 3) g.use_tma = 0;
  const size_t smem = kGSmemBytes;
  cudaError_t e = ensure_dyn_smem((const void *)k_gemm_split<BF>, smem, false);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(workspace, 0, 4, s)) != cudaSuccess) return e;
  k_gemm_split<BF><<<g.ntiles * g.nsplit, kGThreads, smem, s>>>(g, tmap);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const long long DD = (long long)g.D * g.D;
  k_gemm_assemble<<<(unsigned)((DD + 255) / 256), 256, 0, s>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tf32x3(const void *A, long long N, long long M, long long lda, int P, int Q,
                               void *R, int mean, void *workspace, size_t ws_bytes, int sms,
                               cudaStream_t s, bool *ws_ok) {
  return launch_gemm_split<false>(A, N, M, lda, P, Q, R, mean, workspace, ws_bytes, sms, s, ws_ok);
}

cudaError_t launch_gemm_bf16x3(const void *A, long long N, long long M, long long lda, int P, int Q,
                               void *R, int mean, void *workspace, size_t ws_bytes, int sms,
                               cudaStream_t s, bool *ws_ok) {
  return launch_gemm_split<true>(A, N, M, lda, P, Q, R, mean, workspace, ws_bytes, sms, s, ws_ok);
}

}  // namespace cov
