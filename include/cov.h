/*
 * cov.h -- C ABI of the GB300 (sm_103a) covariance-method library.
 *
 * The library computes the estimated covariance matrix of the covariance
 * method (arXiv 1303.2285, Section 2.2, Eq. 2.1-2.2): for an N x M complex
 * input A and a P x Q sliding window, each window position (p, q) is
 * column-stacked into the PQ-vector x (x[i + P*j] = A[p+i][q+j], 0-based),
 * and
 *
 *     R = (1/K) * sum over all K = (N-P+1)(M-Q+1) positions of x * x^H
 *
 * (COV_MEAN; COV_SUM returns the plain sum of Eq. 2.2). R is PQ x PQ and
 * Hermitian; the library writes both triangles, with the lower one the exact
 * conjugate of the upper one and a zero imaginary part on the diagonal.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Complex numbers are interleaved (re, im): COV_C64 = two floats (8 bytes),
 *   COV_C128 = two doubles (16 bytes).
 * - A is row-major with leading dimension lda >= M (in complex elements);
 *   R is row-major PQ x PQ, dense (leading dimension PQ).
 * - All data pointers (A, R, G, dA, workspace, descriptor tables) are DEVICE
 *   pointers owned by the caller, unless a parameter says "host". The library
 *   keeps no reference to them after the call returns, never frees them, and
 *   overwrites (never accumulates into) its outputs.
 * - Calls are asynchronous and ordered on `stream` (a cudaStream_t; NULL is
 *   the legacy default stream). The returned status covers host-side argument
 *   checks and launch errors only. A kernel that gives up a bounded wait
 *   records COV_ETIMEOUT (or COV_EDEVICE) in the workspace's status word; read
 *   it with cov_check_device_status.
 * - No entry point falls back to a CPU implementation: every result is
 *   computed by this library's CUDA kernels.
 * - Entry points that take (workspace, ws_bytes) never allocate device
 *   memory. cov_estimate allocates a stream-ordered workspace
 *   (cudaMallocAsync / cudaFreeAsync) on `stream`.
 */
#ifndef COV_H
#define COV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *cov_stream_t; /* same type as cudaStream_t */

typedef enum {
  COV_OK = 0,
  COV_EINVAL = 1,       /* null pointer, size out of range, P > N, lda < M, ... */
  COV_ECUDA = 2,        /* a CUDA runtime call or a kernel launch failed */
  COV_EWORKSPACE = 3,   /* workspace missing, too small or not 256-byte aligned */
  COV_ETIMEOUT = 4,     /* a bounded device-side wait gave up */
  COV_EUNSUPPORTED = 5, /* valid arguments the selected algorithm cannot take */
  COV_EDEVICE = 6       /* a device-side consistency check failed */
} cov_status;

typedef enum { COV_C64 = 0, COV_C128 = 1 } cov_dtype;

typedef enum { COV_MEAN = 0, COV_SUM = 1 } cov_norm;

typedef enum {
  /* COV_RECURRENCE where it applies, else COV_DIRECT. */
  COV_AUTO = 0,
  /* The combination / diagonal-segment method (Sections 3.1-3.4,
   * Algorithm 1): every distinct product A[n][m] * conj(A[n+dr][m+dc]) of a
   * unique combination (Eq. 3.3) is formed once; each combination's diagonal
   * segments are seeded with a direct box sum and walked along the diagonal
   * by adding the entering row of products and subtracting the leaving one;
   * exactly one thread block writes each element of R. FP32 with compensated
   * running sums for COV_C64, FP64 for COV_C128. Needs P, Q <= 32
   * (COV_EUNSUPPORTED otherwise); every N >= P, M >= Q is taken, also
   * where no row (N < 2P-1) or no column (M < 2Q-1) lies in every box. */
  COV_RECURRENCE = 1,
  /* Dense form R = X X^H on the block-Hankel data matrix X (PQ x K, Eq. 2.2)
   * on tcgen05 tensor cores, with split operands and FP32 accumulation.
   * COV_C64 only. TF32X3: x = hi + lo in TF32, products hh + hl + lh.
   * BF16X3: x = hi + mid + lo in BF16, products hh + hm + mh + mm + hl + lh
   * (the terms down to 2^-16 of |x y|). */
  COV_GEMM_TF32X3 = 2,
  COV_GEMM_BF16X3 = 3,
  /* Plain per-element sums of Eq. 2.2 in FP64 (the straightforward serial
   * algorithm of Section 2.4, one thread per element of R). Output rounded to
   * the input's type. */
  COV_DIRECT = 4
} cov_algo;

/* Human-readable name of a status code (static string). A property of the
 * library; the paper has no counterpart. */
const char *cov_status_string(cov_status s);

/* Library version as 10000*major + 100*minor + patch (no paper counterpart). */
int cov_version(void);

/* ---------------------------------------------------------------------------
 * Plan-layer queries. Host only: no GPU, no CUDA call.
 * ------------------------------------------------------------------------- */
typedef struct {
  int64_t K;                 /* window positions (N-P+1)(M-Q+1) */
  int64_t n_combinations;    /* |UC| = PQ + (P-1)(Q-1), Eq. 3.4 */
  int64_t distinct_products; /* UM = sum over UC of (N-|dr|)(M-|dc|), Eq. 3.5-3.6 */
  int64_t r_elements;        /* (PQ)^2 elements written */
  int64_t naive_macs;        /* K * PQ(PQ+1)/2: products of the direct method */
  int32_t recurrence_ok;     /* 1 if COV_RECURRENCE accepts the shape */
  int32_t n_groups;          /* lag groups of the product kernel */
  int64_t n_tasks;           /* warp tasks of the product kernel */
  int64_t products_inner;    /* products formed by the inner-row kernel */
  int64_t products_fringe;   /* products formed by the fringe-row kernel */
} cov_plan_info_t;

/* Fills *out for an N x M input and P x Q window (cf. Eq. 3.4-3.6, 4.1).
 * COV_EINVAL on a bad shape or null out. */
cov_status cov_plan_info(int64_t N, int64_t M, int P, int Q, cov_plan_info_t *out);

/* Bytes of device workspace cov_estimate_ex needs for this problem (0 is
 * possible). Host only. COV_EINVAL on a bad shape, COV_EUNSUPPORTED if the
 * algorithm cannot take it. For COV_RECURRENCE the workspace holds the
 * partial sums of each unique combination's products (Eq. 3.3-3.6: per
 * combination, per row block and column block of A) and the box-row and
 * box-column sums the diagonal walk of Section 3.3 reads. */
cov_status cov_workspace_size(cov_dtype dtype, int64_t N, int64_t M, int P, int Q,
                              cov_algo algo, size_t *bytes);

/* ---------------------------------------------------------------------------
 * One input matrix.
 * ------------------------------------------------------------------------- */

/* Full control. A: device, N x M (leading dimension lda). R: device, PQ x PQ.
 * workspace: device, >= cov_workspace_size bytes, 256-byte aligned (may be
 * NULL when that size is 0). The workspace is scratch: its contents on entry
 * are ignored and on exit are unspecified, except its first 4 bytes (the
 * status word, see cov_check_device_status). Calls that share a workspace
 * must be ordered on one stream. Section 2.2, Eq. 2.1-2.2. */
cov_status cov_estimate_ex(const void *A, cov_dtype dtype, int64_t N, int64_t M,
                           int64_t lda, int P, int Q, void *R, cov_algo algo,
                           cov_norm norm, void *workspace, size_t ws_bytes,
                           cov_stream_t stream);

/* Convenience form: COV_AUTO, COV_MEAN, lda = M. Allocates its workspace
 * with cudaMallocAsync on `stream` and frees it with cudaFreeAsync. */
cov_status cov_estimate(const void *A, cov_dtype dtype, int64_t N, int64_t M, int P,
                        int Q, void *R, cov_stream_t stream);

/* Interleaved complex elements of the typed entry points (the layout of
 * CUDA's float2 and double2). */
typedef struct {
  float re, im;
} cov_c64_t;
typedef struct {
  double re, im;
} cov_c128_t;

/* Typed short forms of Eq. 2.1-2.2 (Section 2.2): R (PQ x PQ, device) = the
 * mean over all window positions of x x^H for the N x M input A (device,
 * leading dimension M), COV_AUTO. The same call as cov_estimate with
 * COV_C64 / COV_C128: the workspace comes from the stream-ordered allocator
 * (cudaMallocAsync / cudaFreeAsync on `stream`, served by the stream's
 * memory pool). Callers that must not allocate use cov_estimate_ex with a
 * workspace of their own, or cov_estimate_noalloc. COV_EINVAL on a null
 * pointer or a bad shape (N, M, P, Q < 1, P > N, Q > M). */
cov_status cov_estimate_c64(const cov_c64_t *A, int64_t N, int64_t M, int P, int Q, cov_c64_t *R,
                            cov_stream_t stream);
cov_status cov_estimate_c128(const cov_c128_t *A, int64_t N, int64_t M, int P, int Q,
                             cov_c128_t *R, cov_stream_t stream);

/* Size of the static device scratch array behind cov_estimate_noalloc. */
#define COV_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)

/* Same computation as cov_estimate_ex with COV_RECURRENCE, for callers that
 * must not allocate device memory during a call: for example a plugin whose
 * host application's memory pool already holds the device memory, or a
 * real-time radar / SAR processing loop whose device-memory budget is fixed
 * at start-up so that no call can fail, stall or fragment memory mid-stream.
 * The paper has no counterpart; this is a property of the library.
 *
 * The scratch space is a static device array of COV_NOALLOC_SCRATCH_BYTES
 * (16 MiB) inside this library, which every GPU that loads the library holds
 * until the process exits. The caller still passes A and R (device, as for
 * cov_estimate_ex). Nothing is allocated or freed: no cudaMalloc, cudaFree
 * or allocating library routine is called.
 * - The first call made in a given CUDA context (the device's primary
 *   context, or a driver context the caller made current) looks up the
 *   array's device address in that context (cudaGetSymbolAddress) and caches
 *   it under the context's ID; make that first call before any stream
 *   capture. A new context (for example after cudaDeviceReset) gets a new
 *   lookup on its first call.
 * - Problems whose scratch need exceeds COV_NOALLOC_SCRATCH_BYTES (see
 *   cov_workspace_size with COV_RECURRENCE) are rejected with COV_EWORKSPACE
 *   before any work is queued; COV_EUNSUPPORTED for shapes COV_RECURRENCE
 *   does not take.
 * - All calls on a device share the one array, which keeps the previous
 *   call's contents (each call clears what must start at zero). Calls whose
 *   work overlaps on the GPU (different streams, or different host threads
 *   without ordering) race on the array: order them on one stream. */
cov_status cov_estimate_noalloc(const void *A, cov_dtype dtype, int64_t N, int64_t M,
                                int64_t lda, int P, int Q, void *R, cov_norm norm,
                                cov_stream_t stream);

/* The status word of cov_estimate_noalloc's static scratch array (in the
 * current context): reads it, clears it and returns COV_OK, COV_ETIMEOUT (a
 * kernel of the last call gave up a bounded wait; R is then incomplete) or
 * COV_EDEVICE; COV_ECUDA if the copy fails. Synchronises `stream`. Each
 * cov_estimate_noalloc call clears the word first, so check it after the
 * call whose result is to be trusted and before the next one. Allocates
 * nothing. No paper counterpart. */
cov_status cov_noalloc_check_status(cov_stream_t stream);

/* Reads (and then clears) the status word a previous call left at the start
 * of `workspace`. Synchronises `stream`. Returns COV_OK, COV_ETIMEOUT or
 * COV_EDEVICE; COV_ECUDA if the copy itself fails. */
cov_status cov_check_device_status(void *workspace, cov_stream_t stream);

/* Measured rate of the FMA pipe the combination path runs on (instrumentation,
 * not in the paper): COV_C64 times paired FP32 FMAs (fma.rn.f32x2, as the
 * product kernels issue them), COV_C128 FP64 FMAs, in a kernel of independent
 * FMA chains on every SM, `reps` (1..100) timed launches after one warm-up;
 * *fma_per_s = lane FMAs per second of the fastest launch (2 FLOP each).
 * Synchronises `stream`; no device memory is used. */
cov_status cov_measure_fma_rate(cov_dtype dtype, int reps, double *fma_per_s,
                                cov_stream_t stream);

/* Failure-detection self-test (not in the paper). Launches one warp that
 * waits, through the library's bounded mbarrier wait, on a barrier nothing
 * completes; after limit_us microseconds (1 .. 1,000,000) the wait gives up,
 * the kernel records COV_ETIMEOUT in the status word at the start of
 * `workspace` (device, >= 4 bytes, 256-byte aligned) and returns normally,
 * so cov_check_device_status then reports COV_ETIMEOUT and the context stays
 * usable. COV_EINVAL for a limit out of range. */
cov_status cov_selftest_timeout(void *workspace, size_t ws_bytes, uint32_t limit_us,
                                cov_stream_t stream);

/* Instrumentation (not in the paper). With events != NULL, following
 * cov_estimate_ex calls of COV_RECURRENCE record five events each on their
 * stream: before the first kernel and after each of the four kernels
 * (products over inner rows, fringe rows, reductions, walk-and-write), so
 * that cudaEventElapsedTime between consecutive events times one kernel. The
 * events (cudaEvent_t handles owned by the caller; n_events a multiple of 5,
 * at most 5*4096) are used in rounds: the c-th call after this one uses
 * events[5*(c mod n_events/5) ...]. NULL switches this off. Process-wide
 * host state; not thread safe. COV_EINVAL on a bad count or a null handle. */
cov_status cov_set_stage_events(void *const *events, int n_events);

/* ---------------------------------------------------------------------------
 * Tuned knobs of COV_RECURRENCE (not in the paper, whose Section 5 fixes the
 * work decomposition by hand). Three knobs change speed, never the set of
 * products computed:
 *   lag_group       lags (combinations) that share one pass over a tile:
 *                   4, 8 or 16 (16 only for COV_C64);
 *   rows_per_task   inner rows of one product task: a multiple of 8 in
 *                   [8, 256] (clamped by the planner to what shared memory
 *                   holds);
 *   reseed_interval outputs walked from one direct seed along a diagonal,
 *                   1..32 (1 = every output seeded directly);
 *   kernels         1 = the four stages in one cooperative kernel with grid
 *                   barriers (COV_C64 only), 4 = four kernels chained by
 *                   programmatic dependent launch (the only form for
 *                   COV_C128), 0 = the default (COV_C64: 1 while
 *                   |UC| * 2(P-1) <= 32768, else 4);
 *   tile_cols       columns of A per shared-memory tile of the product
 *                   kernel: 32 or 64 (a narrower tile holds more rows, so
 *                   rows_per_task can be larger), 0 = the default (32 where
 *                   a 64-column tile would hold fewer than 96 rows besides
 *                   its halo, else 64).
 * A process-wide host cache maps (dtype, N, M, P, Q, SM count of the current
 * device) to knobs; planning (cov_workspace_size, cov_estimate_ex,
 * cov_estimate, cov_estimate_noalloc) uses the cached knobs for that key, else
 * the defaults. The workspace size can change with the knobs: query
 * cov_workspace_size again after changing the cache. Cache calls are
 * thread safe; host only; no device work except in cov_autotune.
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t lag_group;
  int32_t rows_per_task;
  int32_t reseed_interval;
  int32_t kernels;
  int32_t tile_cols;
} cov_tuning_t;

/* Knobs planning would use for this shape now (*out); *cached (optional)
 * = 1 if they come from the cache. COV_EUNSUPPORTED for shapes
 * COV_RECURRENCE does not take. */
cov_status cov_tuning_get(cov_dtype dtype, int64_t N, int64_t M, int P, int Q,
                          cov_tuning_t *out, int *cached);
/* Stores knobs (HOST struct, copied) for this shape; t == NULL removes the
 * entry. COV_EINVAL for knobs outside the ranges above. */
cov_status cov_tuning_set(cov_dtype dtype, int64_t N, int64_t M, int P, int Q,
                          const cov_tuning_t *t);
void cov_tuning_clear(void);
/* Writes the cache to a text file (one line per entry: dtype-bytes N M P Q
 * SMs and the five knobs; lines with the first four knobs only are read with
 * tile_cols = 0) / merges such a file into it (*n_loaded = entries read).
 * COV_EINVAL if the file cannot be written or read or has a malformed line. */
cov_status cov_tuning_save(const char *path);
cov_status cov_tuning_load(const char *path, int *n_loaded);
/* Upper bound of the workspace any cov_autotune candidate for this shape
 * needs; a smaller workspace makes cov_autotune skip the candidates that do
 * not fit. */
cov_status cov_autotune_workspace_size(cov_dtype dtype, int64_t N, int64_t M, int P, int Q,
                                       size_t *bytes);
/* Times COV_RECURRENCE candidates on the caller's data with CUDA events on
 * `stream` (one warm-up and `reps` timed calls each, 1 <= reps <= 1000):
 * first lag_group x tile_cols x rows_per_task, then reseed_interval at the
 * best of those, then (COV_C64) one kernel against four; stores the fastest in the cache and returns it in *best (optional)
 * with its mean milliseconds per call in *best_ms (optional). Overwrites R
 * (with the correct mean-normalised estimate) and the workspace; synchronises
 * `stream`; not capturable. A candidate whose device status word reports a
 * failure ends the search with that status. */
cov_status cov_autotune(const void *A, cov_dtype dtype, int64_t N, int64_t M, int64_t lda,
                        int P, int Q, void *R, void *workspace, size_t ws_bytes, int reps,
                        cov_stream_t stream, cov_tuning_t *best, float *best_ms);

/* ---------------------------------------------------------------------------
 * Many input matrices of uneven N, M, P, Q in one launch sequence
 * (Section 5.1: computing several matrices concurrently to keep all cores
 * busy). The plan is built on the host once; the device work is a single
 * persistent pass per phase, capturable in one CUDA graph.
 * ------------------------------------------------------------------------- */
typedef struct {
  const void *A; /* device, N x M, leading dimension lda */
  void *R;       /* device, PQ x PQ */
  int64_t lda;
  int32_t N, M, P, Q;
} cov_desc;

typedef struct cov_batched_plan cov_batched_plan;

/* Apertures of one image (the image-processing use of Section 2.3: one
 * covariance matrix per overlapping aperture). Fills descs[k] (HOST, up to
 * max_count entries) for the ap_n x ap_m apertures at rows a*step_r and
 * columns b*step_c of the H x W image (device, leading dimension ld), in
 * row-major order of (a, b): A points into the image in place (lda = ld; no
 * copies), R = R + k * (PQ)^2 complex elements (device, caller-owned,
 * count * (PQ)^2 elements). *count = the number of apertures; with
 * descs == NULL only *count is set. Host only; pass the result to
 * cov_batched_plan_create. */
cov_status cov_aperture_descs(const void *image, cov_dtype dtype, int64_t H, int64_t W, int64_t ld,
                              int ap_n, int ap_m, int step_r, int step_c, int P, int Q, void *R,
                              cov_desc *descs, int max_count, int *count);

/* The same apertures computed in one launch, strip by strip (Section 2.3;
 * Eq. 2.1-2.2 per aperture, through the combinations of Eq. 3.3 and the
 * diagonal walk of Eq. 3.7-3.8): a CTA takes one row of apertures and the
 * neighbours in it whose columns fit a 64-column strip of the image, so that
 * a product under several of them is formed once. image: device, H x W,
 * leading dimension ld, COV_C64, 8-byte aligned, read only. R: device,
 * caller-owned, 8-byte aligned, count * (PQ)^2 complex elements with count
 * and the order of cov_aperture_descs (aperture (a, b) at a * nc + b);
 * overwritten. Needs no workspace and never allocates. COV_EINVAL on the
 * argument errors of cov_aperture_descs, a null R or a misaligned pointer;
 * COV_EUNSUPPORTED for COV_C128, P or Q above 16, ap_n or ap_m above 64.
 * Stream-ordered; FP32 products and sums, 1/K as the FP32 reciprocal. */
cov_status cov_estimate_apertures(const void *image, cov_dtype dtype, int64_t H, int64_t W,
                                  int64_t ld, int ap_n, int ap_m, int step_r, int step_c, int P,
                                  int Q, void *R, cov_norm norm, cov_stream_t stream);

/* Validates `count` descriptors (HOST array, copied) and builds the task
 * schedule. COV_RECURRENCE (or COV_AUTO) only; every member must satisfy the
 * COV_RECURRENCE shape rule (P, Q <= 32), A and R 8-byte aligned. COV_C64
 * plans offer every form whose limits the members meet (below); COV_C128
 * plans the stage form only. On success *plan owns
 * host memory until cov_batched_plan_destroy. The schedule is balanced for
 * the SM count of the device current at creation (152, GB300's, when no
 * device is visible); cov_batched_upload, cov_estimate_batched and
 * cov_batched_autotune return COV_EUNSUPPORTED on a device with another SM
 * count (re-create the plan there). This departs from a device-side
 * descriptor table read at launch: the plan keeps the descriptors on the
 * host, where the schedule is built once, and uploads its tables. */
cov_status cov_batched_plan_create(const cov_desc *descs, int count, cov_dtype dtype,
                                   cov_algo algo, cov_norm norm, cov_batched_plan **plan);
cov_status cov_batched_workspace_size(const cov_batched_plan *plan, size_t *bytes);
/* Copies the plan's tables into `workspace` (stream-ordered). Must precede the
 * first cov_estimate_batched on that workspace (the tables hold addresses in
 * it); not needed again while the workspace is only used by this plan. */
cov_status cov_batched_upload(const cov_batched_plan *plan, void *workspace,
                              size_t ws_bytes, cov_stream_t stream);
/* Launches the batched computation (kernel launches only; capturable). */
cov_status cov_estimate_batched(const cov_batched_plan *plan, void *workspace,
                                size_t ws_bytes, cov_stream_t stream);
void cov_batched_plan_destroy(cov_batched_plan *plan);

/* Tuned knobs of a batched plan (the segment length and task shape the
 * autotuner picks):
 *   form            0: one CTA per member in flight (COV_C64; members with
 *                      P, Q <= 16, N >= 2P-1, M >= 2Q-1, M <= 512);
 *                   3: the stages of the single-matrix combination path,
 *                      each one launch over all members: products over the
 *                      inner rows (persistent CTAs sharing the concatenated
 *                      task list), fringe rows, then one CTA per member for
 *                      the reductions and the seed-and-walk writer; the
 *                      members' partial sums live in the workspace (offered
 *                      while they fit in 4 GiB, and always where no other
 *                      form takes the members);
 *                   1: one warp per member (only when every member has
 *                      M <= 32, N*M <= 1024 and P, Q <= 16);
 *                   2: one CTA per small member in flight, every output a
 *                      separable box sum of its combination's product image
 *                      (column sums walked down the diagonal, window sums
 *                      across the lanes), the upper triangle staged in
 *                      shared memory and R written in whole rows (only when
 *                      every member has M <= 32, N*M <= 1024, P, Q <= 16
 *                      and PQ <= 100: the apertures of Section 2.3);
 *   reseed_interval form 0: the walk down each diagonal segment starts from
 *                   a direct-sum seed every this many outputs (Section 4.3's
 *                   segments cut shorter: more parallel seeds, fewer
 *                   additions in a chain); 0 = one seed per segment; <= 16;
 *   row_ranges      form 0: at most this many row ranges (1, 2 or 4) per
 *                   column block of the inner-row product tasks.
 * A new plan starts at form = 2 where offered, else 1, else 3, else 0,
 * reseed_interval 0, row_ranges 4. */
typedef struct {
  int32_t form;
  int32_t reseed_interval;
  int32_t row_ranges;
} cov_batched_tuning_t;

/* Host only. COV_EINVAL on null arguments. */
cov_status cov_batched_get_tuning(const cov_batched_plan *plan, cov_batched_tuning_t *t);
/* Host only: sets the knobs and rebuilds the schedule when the form changes
 * (upload again before the next cov_estimate_batched). COV_EINVAL on a value
 * outside the ranges above, or a form the plan does not offer. */
cov_status cov_batched_set_tuning(cov_batched_plan *plan, const cov_batched_tuning_t *t);
/* Times the candidate knob settings (forms 2, 1 and 3 where offered; form 0
 * with reseed_interval 0, 2, 4 and row_ranges 2, 4) on the plan's own members,
 * `reps` launches each after one warm-up on `stream`, keeps the fastest and
 * uploads its tables into `workspace`. Writes every member's R (the last
 * setting's result, all settings compute the same R up to rounding);
 * synchronises the stream. COV_EWORKSPACE / COV_EINVAL as
 * cov_estimate_batched; COV_ECUDA on a failed launch or event. */
cov_status cov_batched_autotune(cov_batched_plan *plan, void *workspace, size_t ws_bytes, int reps,
                                cov_stream_t stream);

/* ---------------------------------------------------------------------------
 * Downstream use of the estimates: minimum-variance (Capon) spectra. Section
 * 2.3 cites the covariance method as the input of the Minimum Variance
 * Method in SAR imaging (one estimate per aperture of an image) and of the
 * Capon estimator. For each of `count` matrices R_k (device, COV_C64, D x D,
 * contiguous, R_k at R + k D^2 complex elements) and each of F steering
 * vectors a_f (device, F x D complex64, row f = a_f):
 *     P_k(f) = 1 / (a_f^H (R_k + d_k I)^{-1} a_f),  d_k = loading trace(R_k) / D,
 * computed by an FP32 Cholesky factorisation of R_k + d_k I in shared memory
 * (one CTA per matrix) and forward substitution, P = 1 / ||L^{-1} a||^2.
 * out: device, count x F floats. A matrix whose factorisation meets a
 * non-positive pivot (R_k + d_k I not positive definite) gets NaN outputs.
 * 1 <= D <= 128, loading >= 0; COV_EINVAL otherwise. Stream-ordered.
 * ------------------------------------------------------------------------- */
cov_status cov_capon_spectrum(const void *R, int count, int D, const void *steer, int F,
                              float loading, float *out, cov_stream_t stream);

/* ---------------------------------------------------------------------------
 * Adjoint (not in the paper; the derivative of Eq. 2.2).
 * Given G = dL/dR (PQ x PQ, device, convention dL/dRe + i dL/dIm), writes
 * dA = dL/dA (N x M, device, leading dimension M, same convention):
 *     H = (G + G^H) / K  (G + G^H for COV_SUM),  Y = H X,
 *     dA[n][m] = sum over windows w containing (n, m) of Y[(n-p) + P(m-q), w],
 * with X recomputed from A (never stored) and a gather-form col2im (one
 * writer per element of dA, no atomics). COV_C64 (FP32) and, in the dense
 * form only, COV_C128 (FP64; COV_BWD_AUTO picks it, COV_BWD_STENCIL is
 * COV_EUNSUPPORTED; shapes whose H rows and A patch exceed shared memory,
 * about PQ > 280, are COV_EUNSUPPORTED).
 * ------------------------------------------------------------------------- */
/* Two forms of the same dA (equal up to rounding):
 *   COV_BWD_DENSE    the formula above (H X, (PQ)^2 complex MACs per window);
 *   COV_BWD_STENCIL  dA[n][m] = sum over combinations Delta = (dr, dc), both
 *                    signs, of T_Delta * A[n+dr][m+dc], where T_Delta sums
 *                    H[a][a+Delta] over the window offsets a that a valid
 *                    window places on (n, m) (a rectangle, so T takes
 *                    (2P-1)(2Q-1) values per Delta: the paper's combination
 *                    structure, Sections 3.1-3.3, applied to the adjoint):
 *                    (2P-1)(2Q-1) complex MACs per element of dA. Needs
 *                    N >= 2P-1, M >= 2Q-1 and (2P-1)(2Q-1) <= 2048;
 *   COV_BWD_AUTO     the stencil where it applies, else dense.
 * The workspace depends on the form. */
typedef enum { COV_BWD_AUTO = 0, COV_BWD_DENSE = 1, COV_BWD_STENCIL = 2 } cov_bwd_form;

cov_status cov_backward_workspace_size(cov_dtype dtype, int64_t N, int64_t M, int P,
                                       int Q, size_t *bytes);
cov_status cov_backward_workspace_size_ex(cov_dtype dtype, int64_t N, int64_t M, int P,
                                          int Q, cov_bwd_form form, size_t *bytes);
/* COV_BWD_AUTO. */
cov_status cov_estimate_backward(const void *A, const void *G, cov_dtype dtype,
                                 int64_t N, int64_t M, int P, int Q, cov_norm norm,
                                 void *dA, void *workspace, size_t ws_bytes,
                                 cov_stream_t stream);
cov_status cov_estimate_backward_ex(const void *A, const void *G, cov_dtype dtype,
                                    int64_t N, int64_t M, int P, int Q, cov_norm norm,
                                    cov_bwd_form form, void *dA, void *workspace,
                                    size_t ws_bytes, cov_stream_t stream);
/* A batch of `batch` (1..65535) equal-shape COV_C64 members in one launch
 * sequence, stencil form only: member k reads A + k*stride_A (N x M,
 * leading dimension M), G + k*stride_G (PQ x PQ) and writes
 * dA + k*stride_dA (strides in complex elements, at least one member's
 * size). The workspace holds every member's weight table
 * (cov_backward_strided_workspace_size). COV_EUNSUPPORTED where the stencil
 * form does not apply. */
cov_status cov_backward_strided_workspace_size(int batch, int64_t N, int64_t M, int P, int Q,
                                               size_t *bytes);
cov_status cov_estimate_backward_strided(const void *A, int64_t stride_A, const void *G,
                                         int64_t stride_G, void *dA, int64_t stride_dA,
                                         int batch, int64_t N, int64_t M, int P, int Q,
                                         cov_norm norm, void *workspace, size_t ws_bytes,
                                         cov_stream_t stream);

/* ---------------------------------------------------------------------------
 * Sharding across GPUs (one process per GPU). Section 4.2 gives every
 * combination Delta = (dr, dc) its own set of outputs of R (Eq. 3.7-3.8), so
 * disjoint sets of combinations write disjoint parts of R and need no
 * reduction; Section 5.1 balances the work by the combinations' costs. The
 * shard unit here is a column lag dc: all combinations (dr, dc) of that dc,
 * which own exactly the P x P blocks (a, b) of R with |b - a| = dc (block
 * (a, b) = rows a*P .. a*P+P-1, columns b*P .. b*P+P-1). Every rank needs the
 * whole of A. Host-only planning; the data exchange (gathering the blocks) is
 * the caller's.
 * ------------------------------------------------------------------------- */

/* Splits the column lags [0, Q) into n_ranks contiguous ranges: rank r owns
 * [dc_begin[r], dc_begin[r+1]) (dc_begin: HOST array of n_ranks + 1 entries;
 * empty ranges when n_ranks > Q). The split minimises the largest rank cost,
 * cost = distinct products of the rank's combinations plus a fixed share per
 * combination; rank_cost (HOST, n_ranks, optional) receives them.
 * COV_EUNSUPPORTED for shapes COV_RECURRENCE does not take. */
cov_status cov_partition_lags(int64_t N, int64_t M, int P, int Q, int n_ranks, int32_t *dc_begin,
                              int64_t *rank_cost);
/* COV_RECURRENCE restricted to the column lags [dc_lo, dc_hi): writes exactly
 * the blocks (a, b) of R with dc_lo <= |b - a| < dc_hi (both triangles, same
 * values as cov_estimate_ex) and leaves every other element of R untouched.
 * Same workspace as cov_estimate_ex with COV_RECURRENCE; an empty range queues
 * nothing but the status-word reset. */
cov_status cov_estimate_shard(const void *A, cov_dtype dtype, int64_t N, int64_t M, int64_t lda,
                              int P, int Q, int dc_lo, int dc_hi, void *R, cov_norm norm,
                              void *workspace, size_t ws_bytes, cov_stream_t stream);
/* The exchange of a sharded estimate: the blocks of R a column-lag range
 * [dc_lo, dc_hi) owns (above), packed contiguously so that ranks can gather
 * them with one collective (no reduction: Section 4.2 gives each block one
 * owner). Layout: lag by lag; within lag dc, for a = 0 .. Q-dc-1, block
 * (a, a + dc) and then, for dc > 0, block (a + dc, a); each block P x P
 * row-major. cov_shard_packed_size (host) gives its bytes; cov_shard_pack
 * copies those blocks of R (device, PQ x PQ) into `packed` (device) and
 * cov_shard_unpack writes them back into R, leaving every other element of R
 * untouched. Stream-ordered kernels; an empty range queues nothing.
 * COV_EINVAL for a bad dtype, shape or range, or a null pointer. */
cov_status cov_shard_packed_size(cov_dtype dtype, int P, int Q, int dc_lo, int dc_hi,
                                 size_t *bytes);
cov_status cov_shard_pack(const void *R, cov_dtype dtype, int P, int Q, int dc_lo, int dc_hi,
                          void *packed, cov_stream_t stream);
cov_status cov_shard_unpack(const void *packed, cov_dtype dtype, int P, int Q, int dc_lo,
                            int dc_hi, void *R, cov_stream_t stream);
/* Batched workload (Section 5.1, several matrices at once): assigns each of
 * `count` matrices (HOST descriptors; only the sizes are read) to one of
 * n_ranks ranks, longest processing time first by the same cost the batched
 * plan uses; rank_of (HOST, count) and rank_cost (HOST, n_ranks, optional). */
cov_status cov_partition_matrices(const cov_desc *descs, int count, int n_ranks, int32_t *rank_of,
                                  int64_t *rank_cost);
/* Adjoint: rank r owns the rows [row_begin[r], row_begin[r+1]) of dA (equal
 * bands; row_begin HOST, n_ranks + 1 entries) and needs the rows
 * [halo_lo[r], halo_hi[r]) of A (the band widened by P - 1 rows each way,
 * clipped; HOST, n_ranks each, optional). Because dA is linear in G, the band
 * equals those rows of cov_estimate_backward on that sub-image with COV_SUM
 * and G scaled by 1/K of the full image (COV_MEAN) or unscaled (COV_SUM). */
cov_status cov_partition_rows(int64_t N, int P, int n_ranks, int64_t *row_begin, int64_t *halo_lo,
                              int64_t *halo_hi);

#ifdef __cplusplus
}
#endif

#endif /* COV_H */
