/*
 * CPU oracle for the sliding-window covariance method (arXiv 1303.2285).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it. It shares no code, header or constant with the CUDA
 * library.
 *
 * Everything here is the plain definition written out, in FP64, with a fixed
 * loop order and no floating-point contraction (built with -ffp-contract=off):
 *
 *   Section 2.2, Eq. 2.1: the P x Q window S^{p,q} with upper-left corner
 *   (p, q) is column-stacked into x, x[i + P*j] = A[p+i][q+j] (0-based).
 *   Section 2.2, Eq. 2.2: C = sum over window positions of x * x^H.
 *   Section 1: the estimate averages over all window positions, so
 *   R = C / K with K = (N-P+1)(M-Q+1) (every valid position; see the
 *   readings of the paper in the design notes).
 *   Section 3.2: C is Hermitian, so only b >= a is summed; the lower triangle
 *   is the conjugate, and the diagonal is real (x_a * conj(x_a) = |x_a|^2).
 *
 * Complex numbers are interleaved (re, im) doubles. A is row-major with a
 * leading dimension lda >= M (in complex elements). R is row-major PQ x PQ.
 */
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* x[i + P*j] = A[p+i][q+j]: the column stack of window (p, q), Eq. 2.1. */
static void gather_window(const double *A, long lda, int P, int Q, long p,
                          long q, double *x) {
  for (int j = 0; j < Q; ++j)
    for (int i = 0; i < P; ++i) {
      const double *s = A + 2 * ((p + i) * lda + (q + j));
      x[2 * (i + P * j)] = s[0];
      x[2 * (i + P * j) + 1] = s[1];
    }
}

/*
 * Full estimate R (Eq. 2.2, averaged when mean != 0). Output rows a are split
 * across nthreads; each element still sums the windows in the same order
 * (p outer, q inner), so the result does not depend on nthreads.
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int cov_oracle_window(const double *A, long N, long M, long lda, int P, int Q,
                      int mean, int nthreads, double *R) {
  if (!A || !R || N < 1 || M < 1 || P < 1 || Q < 1 || P > N || Q > M ||
      lda < M)
    return -1;
  const long D = (long)P * Q;
  const long K = (N - P + 1) * (M - Q + 1);
  double *S = (double *)calloc((size_t)(2 * D * D), sizeof(double));
  if (!S) return -1;
  if (nthreads < 1) nthreads = 1;
  int failed = 0;
#pragma omp parallel num_threads(nthreads)
  {
    int t = 0, nt = 1;
#ifdef _OPENMP
    t = omp_get_thread_num();
    nt = omp_get_num_threads();
#endif
    double *x = (double *)malloc((size_t)(2 * D) * sizeof(double));
    if (!x) {
#pragma omp atomic write
      failed = 1;
    } else {
      for (long p = 0; p + P <= N; ++p)
        for (long q = 0; q + Q <= M; ++q) {
          gather_window(A, lda, P, Q, p, q, x);
          for (long a = t; a < D; a += nt) {
            const double ar = x[2 * a], ai = x[2 * a + 1];
            double *row = S + 2 * a * D;
            for (long b = a; b < D; ++b) {
              const double br = x[2 * b], bi = x[2 * b + 1];
              /* x_a * conj(x_b) */
              row[2 * b] += ar * br + ai * bi;
              row[2 * b + 1] += ai * br - ar * bi;
            }
          }
        }
      free(x);
    }
  }
  if (failed) {
    free(S);
    return -1;
  }
  for (long a = 0; a < D; ++a) {
    for (long b = a; b < D; ++b) {
      double re = S[2 * (a * D + b)], im = S[2 * (a * D + b) + 1];
      if (mean) {
        re = re / (double)K;
        im = im / (double)K;
      }
      if (a == b) im = 0.0;
      R[2 * (a * D + b)] = re;
      R[2 * (a * D + b) + 1] = im;
      R[2 * (b * D + a)] = re;
      R[2 * (b * D + a) + 1] = (a == b) ? 0.0 : -im;
    }
  }
  free(S);
  return 0;
}

/*
 * One element R[a][b], summed over the windows in the same order as
 * cov_oracle_window, so it reproduces that element bit for bit. Used to check
 * sampled outputs of full-size problems, where the full oracle is too slow.
 */
int cov_oracle_element(const double *A, long N, long M, long lda, int P, int Q,
                       int mean, long a, long b, double *out) {
  const long D = (long)P * Q;
  if (!A || !out || N < 1 || M < 1 || P < 1 || Q < 1 || P > N || Q > M ||
      lda < M || a < 0 || b < 0 || a >= D || b >= D)
    return -1;
  const int swap = b < a;
  const long aa = swap ? b : a, bb = swap ? a : b;
  const long ia = aa % P, ja = aa / P, ib = bb % P, jb = bb / P;
  const long K = (N - P + 1) * (M - Q + 1);
  double re = 0.0, im = 0.0;
  for (long p = 0; p + P <= N; ++p)
    for (long q = 0; q + Q <= M; ++q) {
      const double *xa = A + 2 * ((p + ia) * lda + (q + ja));
      const double *xb = A + 2 * ((p + ib) * lda + (q + jb));
      re += xa[0] * xb[0] + xa[1] * xb[1];
      im += xa[1] * xb[0] - xa[0] * xb[1];
    }
  if (mean) {
    re = re / (double)K;
    im = im / (double)K;
  }
  if (aa == bb) im = 0.0;
  out[0] = re;
  out[1] = swap ? -im : im;
  return 0;
}

/*
 * Adjoint of the estimate (not in the paper; the derivative of Eq. 2.2).
 * With G = dL/dR in the convention G = dL/dRe(R) + i dL/dIm(R), and the same
 * convention for dA:
 *   dL/dx_w = H x_w,  H = (G + G^H) / K  (or G + G^H in sum mode),
 *   dA[n][m] = sum over windows w that contain (n, m) of (H x_w)[a],
 *   a = (n - p) + P (m - q).
 * Plain loops: for each window, gather x, form y = H x, add y back into dA.
 */
int cov_oracle_backward(const double *A, const double *G, long N, long M,
                        long lda, int P, int Q, int mean, double *dA) {
  if (!A || !G || !dA || N < 1 || M < 1 || P < 1 || Q < 1 || P > N ||
      Q > M || lda < M)
    return -1;
  const long D = (long)P * Q;
  const long K = (N - P + 1) * (M - Q + 1);
  double *H = (double *)malloc((size_t)(2 * D * D) * sizeof(double));
  double *x = (double *)malloc((size_t)(2 * D) * sizeof(double));
  double *y = (double *)malloc((size_t)(2 * D) * sizeof(double));
  if (!H || !x || !y) {
    free(H);
    free(x);
    free(y);
    return -1;
  }
  for (long a = 0; a < D; ++a)
    for (long b = 0; b < D; ++b) {
      /* H[a][b] = G[a][b] + conj(G[b][a]) */
      double re = G[2 * (a * D + b)] + G[2 * (b * D + a)];
      double im = G[2 * (a * D + b) + 1] - G[2 * (b * D + a) + 1];
      if (mean) {
        re = re / (double)K;
        im = im / (double)K;
      }
      H[2 * (a * D + b)] = re;
      H[2 * (a * D + b) + 1] = im;
    }
  for (long n = 0; n < N; ++n)
    memset(dA + 2 * n * lda, 0, (size_t)(2 * M) * sizeof(double));
  for (long p = 0; p + P <= N; ++p)
    for (long q = 0; q + Q <= M; ++q) {
      gather_window(A, lda, P, Q, p, q, x);
      for (long a = 0; a < D; ++a) {
        double re = 0.0, im = 0.0;
        for (long b = 0; b < D; ++b) {
          const double hr = H[2 * (a * D + b)], hi = H[2 * (a * D + b) + 1];
          re += hr * x[2 * b] - hi * x[2 * b + 1];
          im += hr * x[2 * b + 1] + hi * x[2 * b];
        }
        y[2 * a] = re;
        y[2 * a + 1] = im;
      }
      for (int j = 0; j < Q; ++j)
        for (int i = 0; i < P; ++i) {
          double *d = dA + 2 * ((p + i) * lda + (q + j));
          d[0] += y[2 * (i + P * j)];
          d[1] += y[2 * (i + P * j) + 1];
        }
    }
  free(H);
  free(x);
  free(y);
  return 0;
}

/* Number of OpenMP threads available (1 when built without OpenMP). */
int cov_oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
