/*
 * Oracle: plain, slow CPU FP64 reference for the Salem-Said matrix-condensation
 * log-determinant with max-abs pivoting inside the pivot row.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library. It shares no code with the CUDA path
 * and the CUDA path never calls it.
 *
 * What it computes (Dong, Barnett, Dhall, "Parallel Matrix Condensation for
 * Calculating Log-Determinant of Large Matrix"):
 *
 *  - Eq. (2): B is the (m-1)x(m-1) matrix of 2x2 minors built around the pivot
 *    a_kl; row k and column l are dropped and the other rows and columns keep
 *    their order (the index shift past k and l in the four cases of Eq. (2)).
 *  - Eq. (3), Sec. 2.3: a_kl is factored out of the pivot ROW, so the pivot
 *    becomes 1 and every minor reduces to  a_ij - a_il * (a_kj / a_kl).
 *    det A = a_kl * det A*, and det A* = (-1)^(k+l) det B*. The factor (-1)^(k+l)
 *    is the Laplace-expansion sign of the eliminated entry; the printed Eq. (1)
 *    leaves it out (a 3x3 permutation matrix with k = 1, l = 2 has det B = 1 but
 *    det A = -1).
 *  - Sec. 2.2: the pivot column l is the column of largest |a_kj| in row k.
 *    Ties go to the first such column; with order-preserving deletion that is the
 *    smallest original column label.
 *  - Fig. 6 with one process: the pivot row k is always the first row of the
 *    current matrix, the running sum is log|a_kl|, and the final 1x1 matrix
 *    contributes its own log|a|.
 *
 * Rounding: the factored row is an IEEE divide  r_j = a_kj / a_kl  and each
 * minor is one fused multiply-add  fma(-a_il, r_j, a_ij). The file must be built
 * with -ffp-contract=off so that no other expression is contracted. The sum of
 * log|a_kl| is compensated (Neumaier's variant of Kahan summation).
 *
 * Other choices the paper names (oracle_logdet_ex):
 *  - Sec. 1: earlier work picks the pivot column differently: the smallest column
 *    index with a nonzero entry (rule 2), or the nonzero entry whose value is
 *    closest to 1 (rule 1; closeness is measured on |a_kj|, as in the Sec. 2.2
 *    example of entries 1e-10 and 2.01); ties go to the first such column.
 *  - Sec. 1 and Sec. 2.3: a_kl may be factored out of column l instead of row k:
 *    c_i = a_il / a_kl and each minor is fma(-c_i, a_kj, a_ij).
 *
 * Conventions where the paper is silent: n == 0 gives (sign 1, logabs 0); a
 * pivot row that is all zero gives (0, -inf) and stops; a NaN anywhere in a
 * pivot row gives (NaN, NaN) and stops.
 *
 * The rank-1 loop over rows may be split over POSIX threads (nthreads > 1). Each
 * row is still computed by exactly the same operations, so the result does not
 * depend on the thread count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_BAD_ARG 1
#define ORACLE_NO_MEMORY 2

/* Neumaier-compensated running sum. */
typedef struct {
  double s, c;
} csum_t;

static void csum_add(csum_t *acc, double x) {
  double t = acc->s + x;
  if (fabs(acc->s) >= fabs(x))
    acc->c += (acc->s - t) + x;
  else
    acc->c += (x - t) + acc->s;
  acc->s = t;
}

/* Pivot column of row 0 of the m x m matrix W (Sec. 2.2): first index of the
 * largest |w_0j|. Returns -1 when the row holds a NaN. */
static int64_t pivot_column(const double *W, int64_t m) {
  int64_t l = 0;
  double best = fabs(W[0]);
  for (int64_t j = 0; j < m; ++j) {
    if (isnan(W[j])) return -1;
    if (fabs(W[j]) > best) {
      best = fabs(W[j]);
      l = j;
    }
  }
  return l;
}

/* Pivot column of row 0 under the rules of earlier work (Sec. 1): rule 1 the
 * first nonzero entry closest to 1 in absolute value (smallest | |w| - 1 |),
 * rule 2 the first nonzero entry. Column 0 when the row is all zero (the caller
 * then sees a zero pivot); -1 when the row holds a NaN. */
static int64_t pivot_column_rule(const double *W, int64_t m, int rule) {
  int64_t l = -1;
  double best = 0.0;
  for (int64_t j = 0; j < m; ++j)
    if (isnan(W[j])) return -1;
  for (int64_t j = 0; j < m; ++j) {
    if (W[j] == 0.0) continue;
    if (rule == 2) return j;
    const double d = fabs(fabs(W[j]) - 1.0);
    if (l < 0 || d < best) {
      best = d;
      l = j;
    }
  }
  return l < 0 ? 0 : l;
}

/* Eq. (2) with the row-factored pivot of Eq. (3): rows i0..i1-1 (i >= 1) of the
 * new matrix. W is m x m (leading dimension m), r is the factored pivot row,
 * Wn is (m-1) x (m-1). Row 0 (the pivot row k) and column l are dropped,
 * the rest keep their order. */
static void condense_rows(const double *W, int64_t m, int64_t l, const double *r,
                          double *Wn, int64_t i0, int64_t i1) {
  for (int64_t i = i0; i < i1; ++i) {
    const double *wi = W + i * m;
    double *out = Wn + (i - 1) * (m - 1);
    const double a_il = wi[l];
    int64_t jj = 0;
    for (int64_t j = 0; j < m; ++j) {
      if (j == l) continue;
      out[jj++] = fma(-a_il, r[j], wi[j]);
    }
  }
}

/* Eq. (2) with the pivot factored out of COLUMN l instead (Sec. 2.3): the
 * multiplier c_i = a_il / a_kl, and each minor is fma(-c_i, a_kj, a_ij); row 0
 * of W is the unfactored pivot row. */
static void condense_rows_colf(const double *W, int64_t m, int64_t l, double p, double *Wn,
                               int64_t i0, int64_t i1) {
  for (int64_t i = i0; i < i1; ++i) {
    const double *wi = W + i * m;
    double *out = Wn + (i - 1) * (m - 1);
    const double c_i = wi[l] / p;
    int64_t jj = 0;
    for (int64_t j = 0; j < m; ++j) {
      if (j == l) continue;
      out[jj++] = fma(-c_i, W[j], wi[j]);
    }
  }
}

/* ---- a small fixed thread team for the row loop ---- */
typedef struct {
  const double *W;
  double *Wn;
  const double *r;
  int64_t m, l;
  double p;
  int colf; /* 1: column-factored minors (condense_rows_colf) */
} job_t;

static void job_rows(const job_t *job, int64_t i0, int64_t i1) {
  if (job->colf)
    condense_rows_colf(job->W, job->m, job->l, job->p, job->Wn, i0, i1);
  else
    condense_rows(job->W, job->m, job->l, job->r, job->Wn, i0, i1);
}

typedef struct team team_t;
typedef struct {
  team_t *team;
  int id;
} worker_arg_t;

struct team {
  int nthreads;
  int quit;
  job_t job;
  pthread_barrier_t start, done;
  pthread_t *threads;
  worker_arg_t *args;
};

static void team_rows(const job_t *job, int id, int nthreads, int64_t *i0, int64_t *i1) {
  int64_t rows = job->m - 1; /* rows 1..m-1 */
  int64_t per = rows / nthreads, extra = rows % nthreads;
  int64_t a = 1 + id * per + (id < extra ? id : extra);
  int64_t b = a + per + (id < extra ? 1 : 0);
  *i0 = a;
  *i1 = b;
}

static void *team_worker(void *p) {
  worker_arg_t *wa = (worker_arg_t *)p;
  team_t *t = wa->team;
  for (;;) {
    pthread_barrier_wait(&t->start);
    if (t->quit) break;
    int64_t i0, i1;
    team_rows(&t->job, wa->id, t->nthreads, &i0, &i1);
    job_rows(&t->job, i0, i1);
    pthread_barrier_wait(&t->done);
  }
  return NULL;
}

static int team_start(team_t *t, int nthreads) {
  memset(t, 0, sizeof(*t));
  t->nthreads = nthreads;
  if (nthreads <= 1) return 0;
  if (pthread_barrier_init(&t->start, NULL, (unsigned)nthreads)) return -1;
  if (pthread_barrier_init(&t->done, NULL, (unsigned)nthreads)) return -1;
  t->threads = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  t->args = (worker_arg_t *)calloc((size_t)nthreads, sizeof(worker_arg_t));
  if (!t->threads || !t->args) return -1;
  for (int i = 1; i < nthreads; ++i) {
    t->args[i].team = t;
    t->args[i].id = i;
    if (pthread_create(&t->threads[i], NULL, team_worker, &t->args[i])) return -1;
  }
  return 0;
}

static void team_run(team_t *t, const job_t *job) {
  if (t->nthreads <= 1) {
    job_rows(job, 1, job->m);
    return;
  }
  t->job = *job;
  pthread_barrier_wait(&t->start);
  int64_t i0, i1;
  team_rows(job, 0, t->nthreads, &i0, &i1);
  job_rows(job, i0, i1);
  pthread_barrier_wait(&t->done);
}

static void team_stop(team_t *t) {
  if (t->nthreads <= 1) return;
  t->quit = 1;
  pthread_barrier_wait(&t->start);
  for (int i = 1; i < t->nthreads; ++i) pthread_join(t->threads[i], NULL);
  pthread_barrier_destroy(&t->start);
  pthread_barrier_destroy(&t->done);
  free(t->threads);
  free(t->args);
}

/*
 * sign(det A) and log|det A| by the condensation sweep (Eqs. (2)-(3), Sec. 2.2,
 * Fig. 6 with one process).
 *
 *   A          n x n, row-major, leading dimension lda >= n (read only)
 *   max_steps  < 0: run to the end. >= 0: stop after that many condensation
 *              steps (a bounded sample for timing; sign/logabs are then partial)
 *   nthreads   threads for the row loop (>= 1)
 *   rule       pivot column: 0 max |a_kj| (Sec. 2.2, the paper's), 1 the nonzero
 *              |a_kj| closest to 1, 2 the first nonzero (earlier work, Sec. 1)
 *   colf       0: a_kl factored out of row k; 1: out of column l (Sec. 2.3)
 *   sign       out: +1, -1, 0 (singular) or NaN
 *   logabs     out: log|det A|, -inf when singular, NaN on NaN input
 *   piv_label  out (may be NULL): n entries, original column label of the pivot
 *              of each step (the last entry is the final 1x1); -1 where no step ran
 *   piv_value  out (may be NULL): n entries, the signed pivot a_kl of each step
 *   steps_done out (may be NULL): number of pivots taken
 * Returns 0, or 1 for bad arguments, 2 when host memory runs out.
 */
int oracle_logdet_ex(const double *A, int64_t n, int64_t lda, int64_t max_steps, int nthreads,
                     int rule, int colf, double *sign, double *logabs, int64_t *piv_label,
                     double *piv_value, int64_t *steps_done) {
  if (n < 0 || lda < n || (n > 0 && !A) || !sign || !logabs || nthreads < 1) return ORACLE_BAD_ARG;
  if (rule < 0 || rule > 2 || colf < 0 || colf > 1) return ORACLE_BAD_ARG;
  for (int64_t s = 0; s < n; ++s) {
    if (piv_label) piv_label[s] = -1;
    if (piv_value) piv_value[s] = 0.0;
  }
  if (steps_done) *steps_done = 0;
  *sign = 1.0;
  *logabs = 0.0;
  if (n == 0) return ORACLE_OK;

  double *W = (double *)malloc((size_t)n * (size_t)n * sizeof(double));
  double *Wn = (double *)malloc((size_t)n * (size_t)n * sizeof(double));
  double *r = (double *)malloc((size_t)n * sizeof(double));
  int64_t *label = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  if (!W || !Wn || !r || !label) {
    free(W); free(Wn); free(r); free(label);
    return ORACLE_NO_MEMORY;
  }
  for (int64_t i = 0; i < n; ++i) memcpy(W + i * n, A + i * lda, (size_t)n * sizeof(double));
  for (int64_t j = 0; j < n; ++j) label[j] = j;

  team_t team;
  if (team_start(&team, nthreads)) {
    free(W); free(Wn); free(r); free(label);
    return ORACLE_NO_MEMORY;
  }

  double sgn = 1.0;
  csum_t acc = {0.0, 0.0};
  int64_t m = n, step = 0;
  int done = 0;
  while (!done) {
    if (max_steps >= 0 && step >= max_steps) break;
    int64_t l = rule == 0 ? pivot_column(W, m) : pivot_column_rule(W, m, rule);
    if (l < 0) { /* NaN in the pivot row */
      sgn = NAN;
      acc.s = NAN;
      acc.c = 0.0;
      break;
    }
    double p = W[l];
    if (piv_label) piv_label[step] = label[l];
    if (piv_value) piv_value[step] = p;
    ++step;
    if (p == 0.0) { /* the whole pivot row is zero: det A = 0 */
      sgn = 0.0;
      acc.s = -INFINITY;
      acc.c = 0.0;
      break;
    }
    /* det A = a_kl det A* (Eq. (3)); det A* = (-1)^(k+l) det B*, with k = 1 and
     * 1-based l = l + 1, so the Laplace sign is (-1)^l for 0-based l. */
    if (p < 0.0) sgn = -sgn;
    if (l & 1) sgn = -sgn;
    csum_add(&acc, log(fabs(p)));
    if (m == 1) {
      done = 1;
      break;
    }
    if (!colf)
      for (int64_t j = 0; j < m; ++j) r[j] = W[j] / p; /* pivot row factored (Sec. 2.3) */
    job_t job = {W, Wn, r, m, l, p, colf};
    team_run(&team, &job);
    for (int64_t j = l; j + 1 < m; ++j) label[j] = label[j + 1]; /* drop column l */
    double *tmp = W;
    W = Wn;
    Wn = tmp;
    --m;
  }
  team_stop(&team);
  *sign = sgn;
  *logabs = acc.s + acc.c;
  if (steps_done) *steps_done = step;
  free(W); free(Wn); free(r); free(label);
  return ORACLE_OK;
}

/* The paper's method: max-abs pivot column, pivot factored out of the row. */
int oracle_logdet(const double *A, int64_t n, int64_t lda, int64_t max_steps, int nthreads,
                  double *sign, double *logabs, int64_t *piv_label, double *piv_value,
                  int64_t *steps_done) {
  return oracle_logdet_ex(A, n, lda, max_steps, nthreads, 0, 0, sign, logabs, piv_label,
                          piv_value, steps_done);
}

/*
 * One condensation step of Eq. (2) around an arbitrary pivot (k, l) (0-based),
 * with a_kl factored out of row k (Eq. (3), Sec. 2.3). Sec. 2.1 notes that both
 * k and l may be chosen freely.
 *
 *   A  m x m, row-major, leading dimension lda (read only), m >= 2
 *   B  out: (m-1) x (m-1), leading dimension m-1; B_ij = a_ij - a_il * a_kj / a_kl
 *      with row k and column l dropped and the other indices shifted as in Eq. (2)
 *   factor out: a_kl * (-1)^(k+l), so that det A = factor * det B
 * Returns 0, or 1 for bad arguments (including a_kl == 0).
 */
int oracle_condense_once(const double *A, int64_t m, int64_t lda, int64_t k, int64_t l,
                         double *B, double *factor) {
  if (m < 2 || lda < m || !A || !B || !factor || k < 0 || k >= m || l < 0 || l >= m)
    return ORACLE_BAD_ARG;
  double p = A[k * lda + l];
  if (p == 0.0 || isnan(p)) return ORACLE_BAD_ARG;
  double *r = (double *)malloc((size_t)m * sizeof(double));
  if (!r) return ORACLE_NO_MEMORY;
  for (int64_t j = 0; j < m; ++j) r[j] = A[k * lda + j] / p;
  int64_t ii = 0;
  for (int64_t i = 0; i < m; ++i) {
    if (i == k) continue;
    const double a_il = A[i * lda + l];
    int64_t jj = 0;
    for (int64_t j = 0; j < m; ++j) {
      if (j == l) continue;
      B[ii * (m - 1) + jj] = fma(-a_il, r[j], A[i * lda + j]);
      ++jj;
    }
    ++ii;
  }
  free(r);
  *factor = ((k + l) & 1) ? -p : p;
  return ORACLE_OK;
}
