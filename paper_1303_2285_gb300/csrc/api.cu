// C ABI of the library (see include/cov.h): argument checks, algorithm
// selection, workspace layout and kernel launches. No entry point computes
// anything on the host; every result comes from this library's kernels.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "../../include/cov.h"
#include "cov_internal.h"
#include "cov_launch.h"
#include "plan.h"

using namespace cov;

namespace {

int device_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  static int cache[64] = {0};
  if (dev >= 0 && dev < 64 && cache[dev] > 0) return cache[dev];
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (dev >= 0 && dev < 64) cache[dev] = sms;
  return sms;
}

bool shape_ok(int64_t N, int64_t M, int P, int Q) {
  return N >= 1 && M >= 1 && P >= 1 && Q >= 1 && P <= N && Q <= M && N < (1LL << 30) &&
         M < (1LL << 30) && (int64_t)P * Q <= (1LL << 15);
}

StageEvents g_stage_events = {nullptr, 0, 0, false};
cudaEvent_t g_stage_store[5 * 4096];

// Plans (cached tuning unless `tune` is given) and launches the combination
// path on the caller's workspace.
cov_status run_recurrence(const void *A, int elem, int64_t N, int64_t M, int64_t lda, int P, int Q,
                          void *R, cov_norm norm, void *workspace, size_t ws_bytes, int sms,
                          cudaStream_t s, const Tuning *tune, StageEvents *marks, int dc_lo = 0,
                          int dc_hi = -1) {
  RecParams p;
  WsLayout ws;
  plan_recurrence(N, M, lda, P, Q, elem, sms, p, ws, tune);
  if (dc_hi >= 0) restrict_to_lags(p, dc_lo, dc_hi);
  if (!workspace || ws_bytes < ws.total || ((uintptr_t)workspace & 255) != 0)
    return COV_EWORKSPACE;
  char *w = (char *)workspace;
  p.A = A;
  p.R = R;
  p.mean = norm == COV_MEAN ? 1 : 0;
  p.status = (unsigned *)w;
  p.core_part = w + ws.core_off;
  p.colsum_part = w + ws.colsum_off;
  p.sin_part = w + ws.sin_off;
  p.rowval = w + ws.rowval_off;
  p.colval = w + ws.colval_off;
  // status word and the fused kernel's barrier and task counters start at 0
  if (cudaMemsetAsync(w, 0, 16, s) != cudaSuccess) return COV_ECUDA;
  if (p.dc_lo >= p.dc_hi) return COV_OK;  // empty shard
  if (launch_recurrence(p, elem == 16, sms, s, marks) != cudaSuccess) return COV_ECUDA;
  return COV_OK;
}

cov_algo resolve_algo(cov_algo algo, int64_t N, int64_t M, int P, int Q) {
  if (algo != COV_AUTO) return algo;
  return recurrence_ok(N, M, P, Q) ? COV_RECURRENCE : COV_DIRECT;
}

}  // namespace

extern "C" {

const char *cov_status_string(cov_status s) {
  switch (s) {
    case COV_OK: return "COV_OK";
    case COV_EINVAL: return "COV_EINVAL: invalid argument";
    case COV_ECUDA: return "COV_ECUDA: CUDA call or launch failed";
    case COV_EWORKSPACE: return "COV_EWORKSPACE: workspace missing, too small or misaligned";
    case COV_ETIMEOUT: return "COV_ETIMEOUT: a bounded device wait gave up";
    case COV_EUNSUPPORTED: return "COV_EUNSUPPORTED: not supported by the selected algorithm";
    case COV_EDEVICE: return "COV_EDEVICE: device-side check failed";
  }
  return "unknown cov_status";
}

int cov_version(void) { return 100; }

cov_status cov_plan_info(int64_t N, int64_t M, int P, int Q, cov_plan_info_t *out) {
  if (!out || !shape_ok(N, M, P, Q)) return COV_EINVAL;
  memset(out, 0, sizeof(*out));
  const long long D = (long long)P * Q;
  out->K = n_positions(N, M, P, Q);
  out->n_combinations = n_unique_combinations(P, Q);
  out->distinct_products = distinct_products(N, M, P, Q);
  out->r_elements = D * D;
  out->naive_macs = out->K * (D * (D + 1) / 2);
  out->recurrence_ok = recurrence_ok(N, M, P, Q) ? 1 : 0;
  if (out->recurrence_ok) {
    RecParams p;
    WsLayout ws;
    plan_recurrence(N, M, M, P, Q, 8, device_sms(), p, ws);
    out->n_groups = p.ngroups;
    out->n_tasks = p.n_tasks;
    // products of the inner-row kernel: inner rows x all columns, valid lags
    long long inner = 0, fringe = 0;
    for (int dc = 0; dc < Q; ++dc) {
      const int lo = dc == 0 ? 0 : -(P - 1);
      for (int dr = lo; dr <= P - 1; ++dr) {
        const long long cols_all = M - dc;                  // columns with a valid partner
        const long long cols_inner = p.n_innerc;            // inner columns
        inner += (long long)p.n_inner * cols_all;
        long long rows_f = 0;                               // fringe rows with a valid partner
        for (int k = 0; k < p.NFR; ++k) {
          const long long n = fringe_row(P, p.n_inner, k);
          if (n + dr >= 0 && n + dr < N) ++rows_f;
        }
        long long cols_f = 0;                               // fringe columns with a valid partner
        for (int k = 0; k < p.NFC; ++k)
          if (fringe_col(Q, p.n_innerc, k) + dc < M) ++cols_f;
        fringe += rows_f * cols_inner;                       // lane-strided inner columns
        fringe += rows_f * cols_f;                           // its own fringe-column products
      }
    }
    out->products_inner = inner;
    out->products_fringe = fringe;
  }
  return COV_OK;
}

cov_status cov_workspace_size(cov_dtype dtype, int64_t N, int64_t M, int P, int Q,
                              cov_algo algo, size_t *bytes) {
  if (!bytes || !shape_ok(N, M, P, Q) || (dtype != COV_C64 && dtype != COV_C128))
    return COV_EINVAL;
  algo = resolve_algo(algo, N, M, P, Q);
  switch (algo) {
    case COV_RECURRENCE: {
      if (!recurrence_ok(N, M, P, Q)) return COV_EUNSUPPORTED;
      RecParams p;
      WsLayout ws;
      plan_recurrence(N, M, M, P, Q, dtype == COV_C128 ? 16 : 8, device_sms(), p, ws);
      *bytes = ws.total;
      return COV_OK;
    }
    case COV_DIRECT:
      *bytes = kWsHeader;
      return COV_OK;
    case COV_GEMM_TF32X3:
    case COV_GEMM_BF16X3:
      if (dtype != COV_C64 || !gemm_shape_ok(N, M, P, Q)) return COV_EUNSUPPORTED;
      *bytes = gemm_workspace_size(N, M, P, Q);
      return COV_OK;
    default:
      return COV_EUNSUPPORTED;
  }
}

cov_status cov_estimate_ex(const void *A, cov_dtype dtype, int64_t N, int64_t M, int64_t lda,
                           int P, int Q, void *R, cov_algo algo, cov_norm norm, void *workspace,
                           size_t ws_bytes, cov_stream_t stream) {
  if (!A || !R || !shape_ok(N, M, P, Q) || lda < M || (dtype != COV_C64 && dtype != COV_C128) ||
      (norm != COV_MEAN && norm != COV_SUM))
    return COV_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  algo = resolve_algo(algo, N, M, P, Q);
  const int elem = dtype == COV_C128 ? 16 : 8;
  if (((uintptr_t)A % (uintptr_t)(elem / 2)) != 0 || ((uintptr_t)R % (uintptr_t)(elem / 2)) != 0)
    return COV_EINVAL;
  switch (algo) {
    case COV_RECURRENCE: {
      if (!recurrence_ok(N, M, P, Q)) return COV_EUNSUPPORTED;
      if (!workspace || ((uintptr_t)workspace & 255) != 0) return COV_EWORKSPACE;
      const int sms = device_sms();
      if (sms <= 0) return COV_ECUDA;
      return run_recurrence(A, elem, N, M, lda, P, Q, R, norm, workspace, ws_bytes, sms, s,
                            nullptr, &g_stage_events);
    }
    case COV_DIRECT: {
      if (workspace && ((uintptr_t)workspace & 255) == 0 && ws_bytes >= 4)
        if (cudaMemsetAsync(workspace, 0, 4, s) != cudaSuccess) return COV_ECUDA;
      DirectParams d;
      d.A = A;
      d.R = R;
      d.lda = lda;
      d.N = (int)N;
      d.M = (int)M;
      d.P = P;
      d.Q = Q;
      d.K = n_positions(N, M, P, Q);
      d.mean = norm == COV_MEAN ? 1 : 0;
      if (launch_direct(d, dtype == COV_C128, s) != cudaSuccess) return COV_ECUDA;
      return COV_OK;
    }
    case COV_GEMM_TF32X3:
    case COV_GEMM_BF16X3: {
      if (dtype != COV_C64 || !gemm_shape_ok(N, M, P, Q)) return COV_EUNSUPPORTED;
      const int sms = device_sms();
      if (sms <= 0) return COV_ECUDA;
      bool ws_ok = false;
      const cudaError_t e =
          algo == COV_GEMM_BF16X3
              ? launch_gemm_bf16x3(A, N, M, lda, P, Q, R, norm == COV_MEAN ? 1 : 0, workspace,
                                   ws_bytes, sms, s, &ws_ok)
              : launch_gemm_tf32x3(A, N, M, lda, P, Q, R, norm == COV_MEAN ? 1 : 0, workspace,
                                   ws_bytes, sms, s, &ws_ok);
      if (e != cudaSuccess) return COV_ECUDA;
      return ws_ok ? COV_OK : COV_EWORKSPACE;
    }
    default:
      return COV_EUNSUPPORTED;
  }
}

cov_status cov_estimate(const void *A, cov_dtype dtype, int64_t N, int64_t M, int P, int Q,
                        void *R, cov_stream_t stream) {
  size_t bytes = 0;
  cov_status st = cov_workspace_size(dtype, N, M, P, Q, COV_AUTO, &bytes);
  if (st != COV_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  void *ws = nullptr;
  if (bytes > 0 && cudaMallocAsync(&ws, bytes, s) != cudaSuccess) return COV_ECUDA;
  st = cov_estimate_ex(A, dtype, N, M, M, P, Q, R, COV_AUTO, COV_MEAN, ws, bytes, stream);
  if (ws && cudaFreeAsync(ws, s) != cudaSuccess && st == COV_OK) st = COV_ECUDA;
  return st;
}

cov_status cov_estimate_c64(const cov_c64_t *A, int64_t N, int64_t M, int P, int Q, cov_c64_t *R,
                            cov_stream_t stream) {
  return cov_estimate(A, COV_C64, N, M, P, Q, R, stream);
}

cov_status cov_estimate_c128(const cov_c128_t *A, int64_t N, int64_t M, int P, int Q,
                             cov_c128_t *R, cov_stream_t stream) {
  return cov_estimate(A, COV_C128, N, M, P, Q, R, stream);
}

cov_status cov_set_stage_events(void *const *events, int n_events) {
  if (!events) {
    g_stage_events.on = false;
    return COV_OK;
  }
  if (n_events < 5 || n_events % 5 != 0 || n_events > 5 * 4096) return COV_EINVAL;
  for (int k = 0; k < n_events; ++k) {
    if (!events[k]) return COV_EINVAL;
    g_stage_store[k] = (cudaEvent_t)events[k];
  }
  g_stage_events.ev = g_stage_store;
  g_stage_events.rounds = n_events / 5;
  g_stage_events.calls = 0;
  g_stage_events.on = true;
  return COV_OK;
}

cov_status cov_check_device_status(void *workspace, cov_stream_t stream) {
  if (!workspace) return COV_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned word = 0;
  if (cudaMemcpyAsync(&word, workspace, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return COV_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return COV_ECUDA;
  if (cudaMemsetAsync(workspace, 0, 4, s) != cudaSuccess) return COV_ECUDA;
  if (word == kDevOk) return COV_OK;
  if (word == kDevTimeout) return COV_ETIMEOUT;
  return COV_EDEVICE;
}

cov_status cov_partition_lags(int64_t N, int64_t M, int P, int Q, int n_ranks, int32_t *dc_begin,
                              int64_t *rank_cost) {
  if (!dc_begin || !shape_ok(N, M, P, Q) || n_ranks < 1 || n_ranks > 65536) return COV_EINVAL;
  if (!recurrence_ok(N, M, P, Q)) return COV_EUNSUPPORTED;
  std::vector<int> b(n_ranks + 1);
  std::vector<long long> c(n_ranks);
  partition_lags(N, M, P, Q, n_ranks, b.data(), c.data());
  for (int r = 0; r <= n_ranks; ++r) dc_begin[r] = b[r];
  if (rank_cost)
    for (int r = 0; r < n_ranks; ++r) rank_cost[r] = c[r];
  return COV_OK;
}

cov_status cov_estimate_shard(const void *A, cov_dtype dtype, int64_t N, int64_t M, int64_t lda,
                              int P, int Q, int dc_lo, int dc_hi, void *R, cov_norm norm,
                              void *workspace, size_t ws_bytes, cov_stream_t stream) {
  if (!A || !R || !shape_ok(N, M, P, Q) || lda < M || (dtype != COV_C64 && dtype != COV_C128) ||
      (norm != COV_MEAN && norm != COV_SUM) || dc_lo < 0 || dc_hi < dc_lo || dc_hi > Q)
    return COV_EINVAL;
  if (!recurrence_ok(N, M, P, Q)) return COV_EUNSUPPORTED;
  const int elem = dtype == COV_C128 ? 16 : 8;
  if (((uintptr_t)A % (uintptr_t)(elem / 2)) != 0 || ((uintptr_t)R % (uintptr_t)(elem / 2)) != 0)
    return COV_EINVAL;
  if (!workspace || ((uintptr_t)workspace & 255) != 0) return COV_EWORKSPACE;
  const int sms = device_sms();
  if (sms <= 0) return COV_ECUDA;
  return run_recurrence(A, elem, N, M, lda, P, Q, R, norm, workspace, ws_bytes, sms,
                        (cudaStream_t)stream, nullptr, nullptr, dc_lo, dc_hi);
}

// autotune candidates
static const int kTuneG[3] = {4, 8, 16};
static const int kTuneTRB[9] = {16, 24, 32, 48, 64, 96, 128, 160, 192};
static const int kTuneTC[2] = {64, 32};
static const int kTuneL[5] = {2, 4, 8, 16, 32};

cov_status cov_autotune_workspace_size(cov_dtype dtype, int64_t N, int64_t M, int P, int Q,
                                       size_t *bytes) {
  if (!bytes || !shape_ok(N, M, P, Q) || (dtype != COV_C64 && dtype != COV_C128)) return COV_EINVAL;
  if (!recurrence_ok(N, M, P, Q)) return COV_EUNSUPPORTED;
  const int elem = dtype == COV_C128 ? 16 : 8;
  const int sms = device_sms();
  RecParams p;
  WsLayout ws;
  plan_recurrence(N, M, M, P, Q, elem, sms, p, ws, nullptr);
  size_t mx = ws.total;
  for (int gi = 0; gi < 3; ++gi)
    for (int ti = 0; ti < 9; ++ti)
      for (int ci = 0; ci < 2; ++ci) {
        const Tuning c = {kTuneG[gi], kTuneTRB[ti], 8, 0, kTuneTC[ci]};
        plan_recurrence(N, M, M, P, Q, elem, sms, p, ws, &c);
        if (ws.total > mx) mx = ws.total;
      }
  *bytes = mx;
  return COV_OK;
}

static bool tuning_valid(const cov_tuning_t &t, int elem) {
  const bool g_ok = t.lag_group == 4 || t.lag_group == 8 || (t.lag_group == 16 && elem == 8);
  const bool k_ok = t.kernels == 0 || t.kernels == 4 || (t.kernels == 1 && elem == 8);
  const bool c_ok = t.tile_cols == 0 || t.tile_cols == 32 || t.tile_cols == 64;
  return g_ok && k_ok && c_ok && t.rows_per_task >= 8 && t.rows_per_task <= 256 &&
         t.rows_per_task % 8 == 0 && t.reseed_interval >= 1 && t.reseed_interval <= kMaxPQ;
}

cov_status cov_tuning_get(cov_dtype dtype, int64_t N, int64_t M, int P, int Q, cov_tuning_t *out,
                          int *cached) {
  if (!out || !shape_ok(N, M, P, Q) || (dtype != COV_C64 && dtype != COV_C128)) return COV_EINVAL;
  if (!recurrence_ok(N, M, P, Q)) return COV_EUNSUPPORTED;
  const int elem = dtype == COV_C128 ? 16 : 8;
  const int sms = device_sms();
  Tuning t;
  if (cached) *cached = lookup_tuning(elem, N, M, P, Q, sms, t) ? 1 : 0;
  RecParams p;
  WsLayout ws;
  plan_recurrence(N, M, M, P, Q, elem, sms, p, ws);
  out->lag_group = p.G;
  out->rows_per_task = p.TRB;
  out->reseed_interval = p.L;
  out->kernels = p.fused ? 1 : 4;
  out->tile_cols = p.TC;
  return COV_OK;
}

cov_status cov_tuning_set(cov_dtype dtype, int64_t N, int64_t M, int P, int Q,
                          const cov_tuning_t *t) {
  if (!shape_ok(N, M, P, Q) || (dtype != COV_C64 && dtype != COV_C128)) return COV_EINVAL;
  if (!recurrence_ok(N, M, P, Q)) return COV_EUNSUPPORTED;
  const int elem = dtype == COV_C128 ? 16 : 8;
  if (t && !tuning_valid(*t, elem)) return COV_EINVAL;
  if (t) {
    const Tuning k = {t->lag_group, t->rows_per_task, t->reseed_interval, t->kernels,
                      t->tile_cols};
    store_tuning(elem, N, M, P, Q, device_sms(), &k);
  } else {
    store_tuning(elem, N, M, P, Q, device_sms(), nullptr);
  }
  return COV_OK;
}

void cov_tuning_clear(void) { clear_tuning(); }

cov_status cov_tuning_save(const char *path) {
  if (!path) return COV_EINVAL;
  return save_tuning(path) == 0 ? COV_OK : COV_EINVAL;
}

cov_status cov_tuning_load(const char *path, int *n_loaded) {
  if (!path) return COV_EINVAL;
  const int n = load_tuning(path);
  if (n_loaded) *n_loaded = n < 0 ? 0 : n;
  return n < 0 ? COV_EINVAL : COV_OK;
}

cov_status cov_autotune(const void *A, cov_dtype dtype, int64_t N, int64_t M, int64_t lda, int P,
                        int Q, void *R, void *workspace, size_t ws_bytes, int reps,
                        cov_stream_t stream, cov_tuning_t *best, float *best_ms) {
  if (!A || !R || !shape_ok(N, M, P, Q) || lda < M || (dtype != COV_C64 && dtype != COV_C128) ||
      reps < 1 || reps > 1000)
    return COV_EINVAL;
  if (!recurrence_ok(N, M, P, Q)) return COV_EUNSUPPORTED;
  const int elem = dtype == COV_C128 ? 16 : 8;
  if (((uintptr_t)A % (uintptr_t)(elem / 2)) != 0 || ((uintptr_t)R % (uintptr_t)(elem / 2)) != 0)
    return COV_EINVAL;
  if (!workspace || ((uintptr_t)workspace & 255) != 0) return COV_EWORKSPACE;
  const int sms = device_sms();
  if (sms <= 0) return COV_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return COV_ECUDA;
  }
  // Times one candidate; returns its mean milliseconds per call, or a negative
  // value when it does not fit the workspace or repeats a planned config.
  std::vector<Tuning> seen;
  cov_status err = COV_OK;
  auto time_one = [&](const Tuning &cand) -> float {
    RecParams p;
    WsLayout ws;
    plan_recurrence(N, M, lda, P, Q, elem, sms, p, ws, &cand);
    if (ws.total > ws_bytes) return -1.f;
    const Tuning eff = {p.G, p.TRB, p.L, p.fused ? 1 : 4, p.TC};
    for (const Tuning &k : seen)
      if (k.G == eff.G && k.TRB == eff.TRB && k.L == eff.L && k.K == eff.K && k.TC == eff.TC)
        return -1.f;
    seen.push_back(eff);
    cov_status st = run_recurrence(A, elem, N, M, lda, P, Q, R, COV_MEAN, workspace, ws_bytes,
                                   sms, s, &eff, nullptr);
    if (st == COV_OK && cudaEventRecord(e0, s) != cudaSuccess) st = COV_ECUDA;
    for (int r = 0; r < reps && st == COV_OK; ++r)
      st = run_recurrence(A, elem, N, M, lda, P, Q, R, COV_MEAN, workspace, ws_bytes, sms, s,
                          &eff, nullptr);
    if (st == COV_OK && cudaEventRecord(e1, s) != cudaSuccess) st = COV_ECUDA;
    if (st == COV_OK && cudaEventSynchronize(e1) != cudaSuccess) st = COV_ECUDA;
    float ms = 0.f;
    if (st == COV_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = COV_ECUDA;
    if (st == COV_OK) st = cov_check_device_status(workspace, stream);
    if (st != COV_OK) {
      err = st;
      return -1.f;
    }
    return ms / (float)reps;
  };
  RecParams p0;
  WsLayout ws0;
  plan_recurrence(N, M, lda, P, Q, elem, sms, p0, ws0, nullptr);
  Tuning bestt = {0, 0, 0, 0, 0};
  float bestv = -1.f;
  // stage 1: lags per group, rows per task and tile width (the product kernel)
  for (int gi = 0; gi < 3 && err == COV_OK; ++gi) {
    if (kTuneG[gi] == 16 && elem == 16) continue;
    for (int ci = 0; ci < 2 && err == COV_OK; ++ci)
      for (int ti = 0; ti < 9 && err == COV_OK; ++ti) {
        const Tuning c = {kTuneG[gi], kTuneTRB[ti], p0.L, 0, kTuneTC[ci]};
        const float v = time_one(c);
        if (v > 0.f && (bestv < 0.f || v < bestv)) {
          bestv = v;
          bestt = seen.back();
        }
      }
  }
  // stage 2: the walk's re-seed interval at the best stage-1 knobs
  for (int li = 0; li < 5 && err == COV_OK && bestv > 0.f; ++li) {
    const Tuning c = {bestt.G, bestt.TRB, kTuneL[li], bestt.K, bestt.TC};
    const float v = time_one(c);
    if (v > 0.f && v < bestv) {
      bestv = v;
      bestt = seen.back();
    }
  }
  // stage 3: the other kernel form (FP32 only)
  if (err == COV_OK && bestv > 0.f && elem == 8) {
    const Tuning c = {bestt.G, bestt.TRB, bestt.L, bestt.K == 1 ? 4 : 1, bestt.TC};
    const float v = time_one(c);
    if (v > 0.f && v < bestv) {
      bestv = v;
      bestt = seen.back();
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != COV_OK) return err;
  if (bestv < 0.f) return COV_EWORKSPACE;  // no candidate fits the workspace
  store_tuning(elem, N, M, P, Q, sms, &bestt);
  if (best) {
    best->lag_group = bestt.G;
    best->rows_per_task = bestt.TRB;
    best->reseed_interval = bestt.L;
    best->kernels = bestt.K;
    best->tile_cols = bestt.TC;
  }
  if (best_ms) *best_ms = bestv;
  return COV_OK;
}

}  // extern "C"
