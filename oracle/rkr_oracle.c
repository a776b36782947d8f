/*
 * rkr_oracle.c -- plain FP64 CPU oracle for reverse k-ranks queries.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header
 * or constant with the CUDA path, and the CUDA path never calls it.
 *
 * Canonical score (the paper fixes no precision; this is the reading used on
 * both sides): s(u, x) = sum over k = 0 .. d-1, left to right, of
 * (double)u[k] * (double)x[k], with one rounding to double after each addition.
 * The product of two floats is exact in double, so a fused multiply-add gives
 * the same value.  Ranks compare canonical scores with strict ">" (Def. 1).
 *
 * Build: gcc -O2 -std=c11 -fPIC -shared -ffp-contract=off -pthread (no fast-math).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- threads */

typedef void (*range_fn)(void *ctx, int64_t lo, int64_t hi);

typedef struct {
  range_fn fn;
  void *ctx;
  int64_t lo, hi;
} range_job;

static void *range_entry(void *arg) {
  range_job *j = (range_job *)arg;
  j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}

/* Split [0, count) into nthreads contiguous ranges and run fn on each. */
static void parallel_for(int64_t count, int32_t nthreads, range_fn fn, void *ctx) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (count < 2 * nthreads) nthreads = 1;
  if (nthreads == 1) {
    fn(ctx, 0, count);
    return;
  }
  pthread_t tid[256];
  range_job jobs[256];
  int started[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].fn = fn;
    jobs[t].ctx = ctx;
    jobs[t].lo = count * t / nthreads;
    jobs[t].hi = count * (t + 1) / nthreads;
    started[t] = pthread_create(&tid[t], NULL, range_entry, &jobs[t]) == 0;
    if (!started[t]) fn(ctx, jobs[t].lo, jobs[t].hi);
  }
  for (int t = 0; t < nthreads; ++t)
    if (started[t]) pthread_join(tid[t], NULL);
}

/* ------------------------------------------------------- canonical scores */

/* s(a, b): the canonical inner product (left-to-right FP64 sum). */
double rkro_dot(const float *a, const float *b, int32_t d) {
  double acc = 0.0;
  for (int32_t k = 0; k < d; ++k) acc = acc + (double)a[k] * (double)b[k];
  return acc;
}

/* ||x|| = sqrt of the left-to-right FP64 sum of squares (Alg. 1, norm step). */
void rkro_norms(const float *X, int64_t m, int32_t d, double *out) {
  for (int64_t i = 0; i < m; ++i) out[i] = sqrt(rkro_dot(X + i * d, X + i * d, d));
}

typedef struct {
  const float *U, *X;
  int64_t nx;
  int32_t d;
  double *out;
} scores_ctx;

static void scores_range(void *p, int64_t lo, int64_t hi) {
  scores_ctx *c = (scores_ctx *)p;
  for (int64_t i = lo; i < hi; ++i)
    for (int64_t j = 0; j < c->nx; ++j)
      c->out[i * c->nx + j] = rkro_dot(c->U + i * c->d, c->X + j * c->d, c->d);
}

/* out[i * nx + j] = s(U_i, X_j) for every pair. */
void rkro_scores(const float *U, int64_t n, const float *X, int64_t nx, int32_t d,
                 int32_t nthreads, double *out) {
  scores_ctx c = {U, X, nx, d, out};
  parallel_for(n, nthreads, scores_range, &c);
}

/* ------------------------------------------------------------ exact ranks */

/* Def. 1 written out: rank = 1 + #{p in P : s(u,p) > s(u,q)}.  O(n nq m d). */
void rkro_ranks_literal(const float *U, int64_t n, const float *P, int64_t m, const float *Q,
                        int64_t nq, int32_t d, int32_t *out) {
  for (int64_t i = 0; i < n; ++i) {
    const float *u = U + i * d;
    for (int64_t q = 0; q < nq; ++q) {
      double theta = rkro_dot(u, Q + q * d, d);
      int64_t above = 0;
      for (int64_t p = 0; p < m; ++p)
        if (rkro_dot(u, P + p * d, d) > theta) ++above;
      out[i * nq + q] = (int32_t)(1 + above);
    }
  }
}

static int cmp_double_desc(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x < y) - (x > y);
}

typedef struct {
  const float *U, *P, *Q;
  int64_t m, nq;
  int32_t d;
  int32_t *out;
} ranks_ctx;

/* Same count as Def. 1, reached by sorting u's scores over P once:
 * the number of scores strictly above theta is the first index whose score
 * is <= theta in descending order. */
static void ranks_range(void *p, int64_t lo, int64_t hi) {
  ranks_ctx *c = (ranks_ctx *)p;
  double *sc = (double *)malloc((size_t)(c->m > 0 ? c->m : 1) * sizeof(double));
  if (!sc) return;
  for (int64_t i = lo; i < hi; ++i) {
    const float *u = c->U + i * c->d;
    for (int64_t j = 0; j < c->m; ++j) sc[j] = rkro_dot(u, c->P + j * c->d, c->d);
    qsort(sc, (size_t)c->m, sizeof(double), cmp_double_desc);
    for (int64_t q = 0; q < c->nq; ++q) {
      double theta = rkro_dot(u, c->Q + q * c->d, c->d);
      int64_t a = 0, b = c->m; /* first index with sc[idx] <= theta */
      while (a < b) {
        int64_t mid = a + (b - a) / 2;
        if (sc[mid] > theta) a = mid + 1; else b = mid;
      }
      c->out[i * c->nq + q] = (int32_t)(1 + a);
    }
  }
  free(sc);
}

void rkro_ranks(const float *U, int64_t n, const float *P, int64_t m, const float *Q, int64_t nq,
                int32_t d, int32_t nthreads, int32_t *out) {
  ranks_ctx c = {U, P, Q, m, nq, d, out};
  parallel_for(n, nthreads, ranks_range, &c);
}

/* ------------------------------------------------ pre-processing (Alg. 1) */

typedef struct {
  const float *U, *P;
  int64_t m;
  int32_t d;
  double *fmin, *fmax;
} fb_ctx;

static void fbounds_range(void *p, int64_t lo, int64_t hi) {
  fb_ctx *c = (fb_ctx *)p;
  for (int64_t i = lo; i < hi; ++i) {
    const float *u = c->U + i * c->d;
    double mx = -INFINITY, mn = INFINITY;
    for (int64_t j = 0; j < c->m; ++j) {
      double s = rkro_dot(u, c->P + j * c->d, c->d);
      if (s > mx) mx = s;
      if (s < mn) mn = s;
    }
    c->fmax[i] = mx;
    c->fmin[i] = mn;
  }
}

/* f_max(u,P) and f_min(u,P): max and min of s(u,p) over P (Section 4.2, step 2). */
void rkro_fbounds_exact(const float *U, int64_t n, const float *P, int64_t m, int32_t d,
                        int32_t nthreads, double *fmin, double *fmax) {
  fb_ctx c = {U, P, m, d, fmin, fmax};
  parallel_for(n, nthreads, fbounds_range, &c);
}

/* t_{u,j} for j = 1..tau (stored at index j-1):
 * t = f_min + (j - 1) * ((f_max - f_min) / (tau - 1)), evaluated in that order
 * (Section 4.2, step 2).  Each operation rounds to double. */
void rkro_thresholds(double fmin, double fmax, int32_t tau, double *t) {
  double delta = (fmax - fmin) / (double)(tau - 1);
  for (int32_t j = 0; j < tau; ++j) {
    double step = (double)j * delta;
    t[j] = fmin + step;
  }
}

typedef struct {
  const float *U, *S;
  int32_t d;
  const int32_t *samp_count;
  const int64_t *weight;
  int32_t omega, tau;
  const double *fmin, *fmax;
  uint32_t *N;
} table_ctx;

/* Rank-table numerators (Alg. 1, step 3; Eq. 1).
 * For user i and column j, T-hat_{i,j} = 1 + N_{i,j} / s with
 * N_{i,j} = sum over buckets l of weight_l * A_l[j], where A_l[j] counts the
 * samples p of bucket l with s(u_i, p) > t_{i,j}, and weight_l is |P_l| (s of
 * |P_l| items sampled) or s (bucket small enough that all of it was taken).
 * The counting loop for one sample stops at the first threshold it does not
 * exceed, because the thresholds are non-decreasing in j. */
static void table_range(void *p, int64_t lo, int64_t hi) {
  table_ctx *c = (table_ctx *)p;
  double *t = (double *)malloc((size_t)c->tau * sizeof(double));
  int64_t *A = (int64_t *)malloc((size_t)c->tau * sizeof(int64_t));
  uint64_t *acc = (uint64_t *)malloc((size_t)c->tau * sizeof(uint64_t));
  if (!t || !A || !acc) { free(t); free(A); free(acc); return; }
  for (int64_t i = lo; i < hi; ++i) {
    const float *u = c->U + i * c->d;
    rkro_thresholds(c->fmin[i], c->fmax[i], c->tau, t);
    memset(acc, 0, (size_t)c->tau * sizeof(uint64_t));
    const float *samp = c->S;
    for (int32_t l = 0; l < c->omega; ++l) {
      memset(A, 0, (size_t)c->tau * sizeof(int64_t));
      for (int32_t q = 0; q < c->samp_count[l]; ++q) {
        double sc = rkro_dot(u, samp, c->d);
        samp += c->d;
        for (int32_t j = 0; j < c->tau; ++j) {
          if (sc > t[j]) A[j] += 1;
          else break;
        }
      }
      for (int32_t j = 0; j < c->tau; ++j) acc[j] += (uint64_t)c->weight[l] * (uint64_t)A[j];
    }
    for (int32_t j = 0; j < c->tau; ++j) c->N[i * c->tau + j] = (uint32_t)acc[j];
  }
  free(t); free(A); free(acc);
}

/* S holds the sampled item rows bucket after bucket (samp_count[l] rows for
 * bucket l).  N is n x tau, row-major. */
void rkro_rank_table(const float *U, int64_t n, int32_t d, const float *S,
                     const int32_t *samp_count, const int64_t *weight, int32_t omega,
                     const double *fmin, const double *fmax, int32_t tau, int32_t nthreads,
                     uint32_t *N) {
  table_ctx c = {U, S, d, samp_count, weight, omega, tau, fmin, fmax, N};
  parallel_for(n, nthreads, table_range, &c);
}
