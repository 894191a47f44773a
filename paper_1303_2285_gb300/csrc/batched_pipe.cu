// The batched plan's stage form (Section 5.1: many covariance matrices
// computed concurrently): every member runs through the stages of the
// single-matrix combination path (Sections 3.1-3.4; see cov_internal.h),
// each stage one launch over all members, so that a batch of small matrices
// gets the single-matrix kernels' shared-memory tiles and register blocks:
//   1. products over the inner rows: one persistent CTA per SM takes chunks
//      of the members' product tasks (up to eight tiles of one member,
//      costliest first) from a counter until none is left, and runs the
//      product pipeline of rec_products.cuh on each (tiles
//      staged with cp.async by four producer warps, consumer warps taking
//      tasks) member by member; each member's lag group (4, 8 or 16) is
//      chosen by its own plan;
//   2. fringe rows x inner columns: the fringe-row CTAs of every member;
//   3. the reductions as thread tasks over all members (CV of each
//      combination, RV of each (combination, fringe row));
//   4. one thread per diagonal segment of every member seeds, walks, divides
//      by K and writes the outputs and their mirrors.
// Stages 3 and 4 number their tasks across the batch (a member's tasks are
// consecutive), so that a large member is spread over many CTAs.
// The stages exchange the single-matrix partial sums through each member's
// region of the workspace. The member plans are read from global memory as
// the kernels' read-only input, their workspace addresses resolved when the
// tables are uploaded. Members are grouped by the kernels' template
// parameters (tile pitch; column-lag register count), one launch per group.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>

#include "batched_pipe.h"
#include "plan.h"
#include "rec_fringe.cuh"
#include "rec_products.cuh"
#include "rec_reduce.cuh"

namespace cov {

// Never read: the tiles are staged with cp.async (use_tma = 0), so the
// product pipeline's tensor-map argument is not used.
__device__ CUtensorMap g_pipe_no_map;

// Index j with first[j] <= x < first[j + 1] (first non-decreasing, n + 1 entries).
__device__ __forceinline__ int find_member(const long long *first, int n, long long x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---- 1. products ------------------------------------------------------------
// Register block rows, consumer warps and producer warps (the tiles are
// staged with cp.async: several producer warps keep ahead of the consumers;
// 16 warps at 128 registers fill the register file)
template <typename T> struct PipeProd;
template <> struct PipeProd<float> { static constexpr int R = 16, NCW = 12, NPW = 4; };
template <> struct PipeProd<double> { static constexpr int R = 8, NCW = 12, NPW = 4; };

// Dynamic schedule: the class's product tasks are cut into chunks (a
// member's tasks of up to eight tiles), listed costliest first; each CTA takes
// the next chunk from a counter in the workspace header until none is left,
// and runs the product pipeline on it.
template <typename T, int PITCH>
__global__ void __launch_bounds__((PipeProd<T>::NCW + PipeProd<T>::NPW) * 32, 1)
    k_pipe_products(const RecParams *__restrict__ mp, const int *__restrict__ chunk_member,
                    const long long *__restrict__ chunk_range, int n_chunks, unsigned *counter) {
  constexpr int R = PipeProd<T>::R, NCW = PipeProd<T>::NCW, NPW = PipeProd<T>::NPW;
  extern __shared__ __align__(1024) unsigned char smem_pp[];
  __shared__ int cur;
  for (;;) {
    if (threadIdx.x == 0) cur = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int c = cur;
    __syncthreads();  // every thread has read cur before the next claim
    if (c >= n_chunks) return;
    const RecParams &p = mp[chunk_member[c]];
    const long long a = chunk_range[2 * c], b = chunk_range[2 * c + 1];
    bool ok = false;
    if (p.G == 4) {
      ok = products_phase<T, 4, R, PITCH, NCW, NPW>(p, g_pipe_no_map, smem_pp, a, b);
    } else if (p.G == 8) {
      ok = products_phase<T, 8, R, PITCH, NCW, NPW>(p, g_pipe_no_map, smem_pp, a, b);
    } else if constexpr (sizeof(T) == 4) {
      ok = products_phase<T, 16, R, PITCH, NCW, NPW>(p, g_pipe_no_map, smem_pp, a, b);
    }
    // every warp is done with the tiles and the barriers: invalidate them
    // before the next chunk's pipeline initialises its own
    ok = __syncthreads_and(ok) != 0;
    if (threadIdx.x == 0) {
      uint64_t *bars = (uint64_t *)(smem_pp + 2 * tile_buf_bytes<T, PITCH>(p.STR));
      for (int k = 0; k < 4; ++k)
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bars + k)) : "memory");
    }
    __syncthreads();
    if (!ok) return;  // a bounded wait gave up: the status word is set
  }
}

// ---- 2. fringe rows x inner columns -------------------------------------------
template <typename T, int QMAX>
__global__ void __launch_bounds__(256) k_pipe_fringe(const RecParams *__restrict__ mp,
                                                      const int *__restrict__ members,
                                                      const long long *__restrict__ first, int n) {
  using C2 = typename C2t<T>::type;
  extern __shared__ __align__(16) unsigned char smem_pf[];
  const int j = find_member(first, n, blockIdx.x);
  const RecParams &p = mp[members[j]];
  const int local = (int)(blockIdx.x - first[j]);
  const int npairs = (p.P - 1) * (2 * p.P - 1);
  const int nblk = (npairs + (int)blockDim.x - 1) / (int)blockDim.x;
  const int pb = local % nblk, rest = local / nblk;
  const int cc = rest % p.NCH, side = rest / p.NCH;
  fringe_stage<T>(p, (C2 *)smem_pf, side, cc);
  __syncthreads();
  const int t = pb * (int)blockDim.x + threadIdx.x;
  if (t < npairs) fringe_pair<T, QMAX, 8>(p, (const C2 *)smem_pf, side, cc, t);
}

// ---- 3. reductions, seed, walk and write ----------------------------------------
// Pairs (combination D, column offset j) that own outputs: j < Q - dc.
__host__ __device__ inline long long walk_pairs(int P, int Q) {
  long long n = 0;
  for (int dc = 0; dc < Q; ++dc) n += (long long)(dc == 0 ? P : 2 * P - 1) * (Q - dc);
  return n;
}
// Thread task: CV[D][j] of combination D for every column offset j (the
// inner-row box sums: core partials plus the fringe-column sums in the box;
// suffix and prefix running sums where a box holds Q - 1 fringe columns,
// window sums otherwise).
template <typename T>
__device__ __forceinline__ void cv_thread(const RecParams &p, int D) {
  using C2 = typename C2t<T>::type;
  const int Q = p.Q, NFC = p.NFC, n_rb = p.n_rb;
  int dr, dc;
  combo_of(p.P, D, dr, dc);
  const int J = Q - dc;
  Neu<T> cr, ci;
  {
    const int np = n_rb * p.n_cb;
    const C2 *cp = (const C2 *)p.core_part + (long long)D * np;
    for (int k = 0; k < np; ++k) {
      const C2 x = cp[k];
      cr.add(x.x);
      ci.add(x.y);
    }
  }
  const C2 *cs = (const C2 *)p.colsum_part + (long long)D * n_rb * NFC;
  auto colsum = [&](int fc) {
    Neu<T> a, b;
    for (int rb = 0; rb < n_rb; ++rb) {
      const C2 x = cs[(long long)rb * NFC + fc];
      a.add(x.x);
      b.add(x.y);
    }
    C2 v;
    v.x = a.value();
    v.y = b.value();
    return v;
  };
  // CV of the stage form: [j][D] (combination fastest)
  const long long cs_j = p.n_uc;
  C2 *cv = (C2 *)p.colval + D;
  if (NFC == 2 * (Q - 1)) {
    // suffix over the left fringe columns k >= j, kept in cv[j] ...
    T sr = T(0), si = T(0);
    for (int k = Q - 2; k >= 0; --k) {
      const C2 x = colsum(k);
      sr += x.x;
      si += x.y;
      if (k < J) {
        C2 o;
        o.x = sr;
        o.y = si;
        cv[k * cs_j] = o;
      }
    }
    // ... then the core and the prefix over the right ones k < j
    T pr = T(0), pi = T(0);
    for (int j = 0; j < J; ++j) {
      Neu<T> vr = cr, vi = ci;
      if (j < Q - 1) {
        vr.add(cv[j * cs_j].x);
        vi.add(cv[j * cs_j].y);
      }
      vr.add(pr);
      vi.add(pi);
      C2 o;
      o.x = vr.value();
      o.y = vi.value();
      cv[j * cs_j] = o;
      if (j < Q - 1) {
        const C2 x = colsum(Q - 1 + j);
        pr += x.x;
        pi += x.y;
      }
    }
  } else {
    for (int j = 0; j < J; ++j) {
      Neu<T> vr = cr, vi = ci;
      for (int k = j; k < j + p.HC; ++k) {
        const C2 x = colsum(k);
        vr.add(x.x);
        vi.add(x.y);
      }
      C2 o;
      o.x = vr.value();
      o.y = vi.value();
      cv[j * cs_j] = o;
    }
  }
}

// Thread task: RV of fringe row fr of combination D for every column offset
// j: the row's inner-column sum S_in (its chunk partials) plus its own
// fringe-column products (each formed once) inside the box of j. The stage
// form lays RV out as [j][fr][D] (combination fastest: consecutive threads
// store, and the walk's threads load, consecutive elements); js is the
// stride of j. The pointers are declared unaliased so that the loads of the
// running sums can be issued ahead of the stores of the outputs.
template <typename C2>
__device__ __forceinline__ void rv_scan(const C2 *__restrict__ An, const C2 *__restrict__ Ab,
                                        C2 *__restrict__ rv, C2 s_in, bool rowok, int Q, int J,
                                        int W, int dc, int M, long long js) {
  // suffix of the left fringe-column products (m = k >= j) ...
  C2 acc = czero<C2>();
#pragma unroll 4
  for (int k = Q - 2; k >= 0; --k) {
    if (rowok) cmac_conj(acc, An[k], Ab[k]);
    if (k < J) {
      C2 o;
      o.x = s_in.x + acc.x;
      o.y = s_in.y + acc.y;
      rv[k * js] = o;
    }
  }
  if (Q - 1 < J) rv[(Q - 1) * js] = s_in;
  // ... plus the prefix of the right ones (m = W + k, k < j)
  C2 pre = czero<C2>();
#pragma unroll 4
  for (int j = 1; j < J; ++j) {
    const int k = j - 1;
    if (rowok && W + k + dc < M) cmac_conj(pre, An[W + k], Ab[W + k]);
    C2 o = rv[j * js];
    o.x += pre.x;
    o.y += pre.y;
    rv[j * js] = o;
  }
}

template <typename T>
__device__ __forceinline__ void rv_thread(const RecParams &p, int D, int fr) {
  using C2 = typename C2t<T>::type;
  const int P = p.P, Q = p.Q, NFR = p.NFR, NFC = p.NFC, NCH = p.NCH;
  int dr, dc;
  combo_of(P, D, dr, dc);
  const int J = Q - dc;
  const int n = fringe_row(P, p.n_inner, fr);
  const bool rowok = n + dr >= 0 && n + dr < p.N;
  C2 s_in = czero<C2>();
  {
    const C2 *sp = (const C2 *)p.sin_part + (long long)D * NCH * NFR + fr;
    for (int cc = 0; cc < NCH; ++cc) {
      const C2 x = sp[(long long)cc * NFR];
      s_in.x += x.x;
      s_in.y += x.y;
    }
  }
  const C2 *A = (const C2 *)p.A;
  const C2 *An = A + (long long)n * p.lda;
  const C2 *Ab = A + (long long)(rowok ? n + dr : n) * p.lda + dc;
  const long long js = (long long)NFR * p.n_uc;
  C2 *rv = (C2 *)p.rowval + (long long)fr * p.n_uc + D;
  if (NFC == 2 * (Q - 1)) {
    rv_scan<C2>(An, Ab, rv, s_in, rowok, Q, J, p.M - Q + 1, dc, p.M, js);
  } else {
    C2 pr[2 * kMaxPQ];
    for (int k = 0; k < NFC; ++k) {
      const int m = fringe_col(Q, p.n_innerc, k);
      C2 v = czero<C2>();
      if (rowok && m + dc < p.M) cmac_conj(v, __ldg(An + m), __ldg(Ab + m));
      pr[k] = v;
    }
    for (int j = 0; j < J; ++j) {
      C2 w = czero<C2>();
      for (int k = j; k < j + p.HC; ++k) {
        w.x += pr[k].x;
        w.y += pr[k].y;
      }
      C2 o;
      o.x = s_in.x + w.x;
      o.y = s_in.y + w.y;
      rv[j * js] = o;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_pipe_reduce(const RecParams *__restrict__ mp,
                                                      const int *__restrict__ members,
                                                      const long long *__restrict__ first, int n,
                                                      long long total) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int j = find_member(first, n, t);
  const RecParams &p = mp[members[j]];
  const long long u = t - first[j];  // [0, n_uc): CV tasks; then RV tasks, combination fastest
  if (u < p.n_uc)
    cv_thread<T>(p, (int)u);
  else
    rv_thread<T>(p, (int)((u - p.n_uc) % p.n_uc), (int)((u - p.n_uc) / p.n_uc));
}

template <typename T>
__global__ void __launch_bounds__(256) k_pipe_walk(const RecParams *__restrict__ mp,
                                                    const int *__restrict__ members,
                                                    const long long *__restrict__ first, int n,
                                                    long long total) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int j = find_member(first, n, t);
  const RecParams &p = mp[members[j]];
  // the member's segments: chunk c, then by column lag dc, column offset
  // j < Q - dc, and the lag's combinations fastest (only the pairs (D, j)
  // that own outputs)
  const long long u = t - first[j];
  const long long per_chunk = walk_pairs(p.P, p.Q);
  const int c = (int)(u / per_chunk);
  long long r = u - c * per_chunk;
  int dc = 0;
  for (;; ++dc) {
    const long long nd = (long long)(dc == 0 ? p.P : 2 * p.P - 1) * (p.Q - dc);
    if (r < nd) break;
    r -= nd;
  }
  const int ncomb = dc == 0 ? p.P : 2 * p.P - 1;
  const int jj = (int)(r / ncomb), k = (int)(r % ncomb);
  const int D = first_combo(p.P, dc) + k;
  const int dr = dc == 0 ? k : k - (p.P - 1);
  const int adr = dr < 0 ? -dr : dr;
  const int I = p.P - adr, i0 = dr < 0 ? -dr : 0;
  const int is = i0 + c * p.L;
  if (is >= i0 + I) return;
  const int ie = (i0 + I) < (is + p.L) ? (i0 + I) : (is + p.L);
  using C2 = typename C2t<T>::type;
  const long long n_uc = p.n_uc;
  const C2 *RV = (const C2 *)p.rowval + (long long)jj * p.NFR * n_uc + D;  // [j][fr][D]
  const C2 cv = ((const C2 *)p.colval)[jj * n_uc + D];                      // [j][D]
  walk_segment_rv<T>(p, RV, n_uc, cv, (C2 *)p.R, dr, dc, jj, is, ie);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

bool pipe_members_ok(const cov_desc *descs, int count) {
  for (int i = 0; i < count; ++i) {
    const cov_desc &d = descs[i];
    if (!d.A || !d.R || d.N < 1 || d.M < 1 || d.P < 1 || d.Q < 1 || d.P > d.N || d.Q > d.M ||
        d.lda < d.M || !recurrence_ok(d.N, d.M, d.P, d.Q) || (((uintptr_t)d.A) & 7) != 0 ||
        (((uintptr_t)d.R) & 7) != 0)
      return false;
  }
  return true;
}

void pipe_plan_build(PipePlan &pp, const cov_desc *descs, int count, int elem, int mean,
                     size_t off, int sms) {
  pp.elem = elem;
  pp.params.resize(count);
  pp.products.clear();
  pp.fringe.clear();
  pp.finish.clear();
  std::map<int, PipeClass> prod, fr, fin;
  std::vector<size_t> region(count);
  std::vector<WsLayout> lay(count);
  for (int k = 0; k < count; ++k) {
    const cov_desc &d = descs[k];
    RecParams &p = pp.params[k];
    // the plan's defaults, four stages, no tuning cache; one walk segment
    // per diagonal (the walk's threads are many already; fewer seeds);
    // FP32 fringe-row chunks of 128 columns (a small member's inner columns
    // in one or two chunks: fewer CTAs and partial sums)
    const Tuning t = {0, 0, kMaxPQ, 4, 0, elem == 8 ? 128 : 0};
    plan_recurrence(d.N, d.M, d.lda, d.P, d.Q, elem, 0, p, lay[k], &t);
    p.A = d.A;
    p.R = d.R;
    p.mean = mean;
    p.use_tma = 0;
    p.fused = 0;
    region[k] = lay[k].total - lay[k].core_off;
    if (p.n_inner > 0 && p.n_tasks > 0) prod[p.PITCH].members.push_back(k);
    if (p.NFR > 0 && p.NCH > 0) fr[p.QMAXF].members.push_back(k);
    fin[0].members.push_back(k);  // reductions
    fin[1].members.push_back(k);  // walk
  }
  const int fpb = elem == 16 ? 32 : 256;
  int slot = 0;  // the counter word of each product launch in the workspace header
  for (auto &kv : prod) {
    PipeClass &c = kv.second;
    c.key = kv.first;
    int str = 0;
    // chunks of one member's tasks: up to eight tiles, and small enough for
    // about four chunks an SM (a batch of a few large members is cut
    // finer); cost = tasks x (a task's rows, the member's mean over its row
    // blocks, times its lags, plus its epilogue); costliest first
    struct Chunk {
      int k;
      long long a, b, cost;
    };
    std::vector<Chunk> ch;
    long long class_tasks = 0;
    for (int k : c.members) class_tasks += pp.params[k].n_tasks;
    const long long fine = std::max(1LL, class_tasks / (4LL * (sms > 0 ? sms : 1)));
    for (int k : c.members) {
      const RecParams &p = pp.params[k];
      const long long w = (long long)((p.n_inner + p.n_rb - 1) / p.n_rb) * p.G + 48;
      const long long step = std::min(8 * p.tasks_per_tile, fine);
      for (long long a = 0; a < p.n_tasks; a += step) {
        const long long b = std::min(p.n_tasks, a + step);
        ch.push_back({k, a, b, (b - a) * w});
      }
      str = std::max(str, p.STR);
    }
    std::stable_sort(ch.begin(), ch.end(), [](const Chunk &x, const Chunk &y) { return x.cost > y.cost; });
    c.members.clear();
    c.first.clear();
    for (const Chunk &x : ch) {
      c.members.push_back(x.k);
      c.first.push_back(x.a);
      c.first.push_back(x.b);
    }
    c.total = (long long)ch.size();
    c.counter = 4 * (1 + slot++);
    c.smem = 2 * ((((size_t)str * c.key * elem) + 1023) & ~(size_t)1023) + 64;
    pp.products.push_back(c);
  }
  for (auto &kv : fr) {
    PipeClass &c = kv.second;
    c.key = kv.first;
    c.first.assign(1, 0);
    size_t smem = 0;
    for (int k : c.members) {
      const RecParams &p = pp.params[k];
      const long long npairs = (long long)(p.P - 1) * (2 * p.P - 1);
      c.first.push_back(c.first.back() + 2LL * p.NCH * ((npairs + fpb - 1) / fpb));
      smem = std::max(smem, (size_t)(2 * p.P - 2) * p.FPITCH * elem);
    }
    c.total = c.first.back();
    c.smem = smem;
    pp.fringe.push_back(c);
  }
  for (auto &kv : fin) {  // key 0: reduction tasks; key 1: walk segments
    PipeClass &c = kv.second;
    c.key = kv.first;
    c.first.assign(1, 0);
    for (int k : c.members) {
      const RecParams &p = pp.params[k];
      const long long nt = c.key == 0 ? (long long)p.n_uc * (1 + p.NFR)
                                      : walk_pairs(p.P, p.Q) * ((p.P + p.L - 1) / p.L);
      c.first.push_back(c.first.back() + nt);
    }
    c.total = c.first.back();
    pp.finish.push_back(c);
  }
  // layout: the member plans, the class arrays, then each member's region;
  // the plans' pointer fields hold workspace offsets (status: offset 0)
  pp.off_params = al256(off);
  off = al256(pp.off_params + sizeof(RecParams) * count);
  for (auto *v : {&pp.products, &pp.fringe, &pp.finish})
    for (PipeClass &c : *v) {
      c.off_members = off;
      off = al256(off + sizeof(int) * c.members.size());
      c.off_first = off;
      off = al256(off + sizeof(long long) * c.first.size());
    }
  for (int k = 0; k < count; ++k) {
    RecParams &p = pp.params[k];
    const WsLayout &w = lay[k];
    p.status = nullptr;
    p.core_part = (void *)(uintptr_t)off;
    p.colsum_part = (void *)(uintptr_t)(off + (w.colsum_off - w.core_off));
    p.sin_part = (void *)(uintptr_t)(off + (w.sin_off - w.core_off));
    p.rowval = (void *)(uintptr_t)(off + (w.rowval_off - w.core_off));
    p.colval = (void *)(uintptr_t)(off + (w.colval_off - w.core_off));
    off = al256(off + region[k]);
  }
  pp.total = off;
}

cudaError_t pipe_upload(const PipePlan &pp, char *ws, cudaStream_t s) {
  // the member plans with their workspace offsets resolved against this
  // workspace (the kernels read them as they are)
  std::vector<RecParams> &abs = pp.resolved;
  abs = pp.params;
  for (RecParams &p : abs) {
    p.status = (unsigned *)(ws + (uintptr_t)p.status);
    p.core_part = ws + (uintptr_t)p.core_part;
    p.colsum_part = ws + (uintptr_t)p.colsum_part;
    p.sin_part = ws + (uintptr_t)p.sin_part;
    p.rowval = ws + (uintptr_t)p.rowval;
    p.colval = ws + (uintptr_t)p.colval;
  }
  cudaError_t e = cudaMemcpyAsync(ws + pp.off_params, abs.data(), sizeof(RecParams) * abs.size(),
                                  cudaMemcpyHostToDevice, s);
  for (const auto *v : {&pp.products, &pp.fringe, &pp.finish})
    for (const PipeClass &c : *v) {
      if (e == cudaSuccess && !c.members.empty())
        e = cudaMemcpyAsync(ws + c.off_members, c.members.data(), sizeof(int) * c.members.size(),
                            cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess && !c.first.empty())
        e = cudaMemcpyAsync(ws + c.off_first, c.first.data(), sizeof(long long) * c.first.size(),
                            cudaMemcpyHostToDevice, s);
    }
  return e;
}

template <typename T, int PITCH>
static cudaError_t launch_pipe_products(const PipeClass &c, char *ws, const RecParams *mp, int sms,
                                        cudaStream_t s) {
  auto kern = k_pipe_products<T, PITCH>;
  cudaError_t e = ensure_dyn_smem((const void *)kern, c.smem, true);
  if (e != cudaSuccess) return e;
  long long grid = sms;
  if (grid > c.total) grid = c.total;
  kern<<<(unsigned)grid, (PipeProd<T>::NCW + PipeProd<T>::NPW) * 32, c.smem, s>>>(
      mp, (const int *)(ws + c.off_members), (const long long *)(ws + c.off_first), (int)c.total,
      (unsigned *)(ws + c.counter));
  return cudaGetLastError();
}

template <typename T, int QMAX>
static cudaError_t launch_pipe_fringe(const PipeClass &c, char *ws, const RecParams *mp,
                                      cudaStream_t s) {
  auto kern = k_pipe_fringe<T, QMAX>;
  cudaError_t e = ensure_dyn_smem((const void *)kern, c.smem, true);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)c.total, sizeof(T) == 8 ? 32 : 256, c.smem, s>>>(
      mp, (const int *)(ws + c.off_members), (const long long *)(ws + c.off_first),
      (int)c.members.size());
  return cudaGetLastError();
}

template <typename T>
static cudaError_t pipe_launch_t(const PipePlan &pp, char *ws, int sms, cudaStream_t s) {
  const RecParams *mp = (const RecParams *)(ws + pp.off_params);
  cudaError_t e = cudaSuccess;
  for (const PipeClass &c : pp.products) {
    if (c.total <= 0) continue;
    switch (c.key) {
      case 48: e = launch_pipe_products<T, 48>(c, ws, mp, sms, s); break;
      case 64: e = launch_pipe_products<T, 64>(c, ws, mp, sms, s); break;
      case 80: e = launch_pipe_products<T, 80>(c, ws, mp, sms, s); break;
      case 96: e = launch_pipe_products<T, 96>(c, ws, mp, sms, s); break;
      default: e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  }
  for (const PipeClass &c : pp.fringe) {
    if (c.total <= 0) continue;
    switch (c.key) {
      case 4: e = launch_pipe_fringe<T, 4>(c, ws, mp, s); break;
      case 8: e = launch_pipe_fringe<T, 8>(c, ws, mp, s); break;
      case 16: e = launch_pipe_fringe<T, 16>(c, ws, mp, s); break;
      case 32: e = launch_pipe_fringe<T, 32>(c, ws, mp, s); break;
      default: e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  }
  for (const PipeClass &c : pp.finish) {
    if (c.total <= 0) continue;
    const unsigned grid = (unsigned)((c.total + 255) / 256);
    const int *mem = (const int *)(ws + c.off_members);
    const long long *first = (const long long *)(ws + c.off_first);
    if (c.key == 0)
      k_pipe_reduce<T><<<grid, 256, 0, s>>>(mp, mem, first, (int)c.members.size(), c.total);
    else
      k_pipe_walk<T><<<grid, 256, 0, s>>>(mp, mem, first, (int)c.members.size(), c.total);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t pipe_launch(const PipePlan &pp, char *ws, int sms, cudaStream_t s) {
  return pp.elem == 16 ? pipe_launch_t<double>(pp, ws, sms, s) : pipe_launch_t<float>(pp, ws, sms, s);
}

}  // namespace cov
