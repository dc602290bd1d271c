/*
 * simplex_oracle.c -- plain FP64 dense-tableau two-phase simplex.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the CPU oracle that the CUDA solver
 * is checked against.  It shares no code, header, table or helper with the
 * CUDA path; only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg may load it.
 *
 * What it computes (Section 3, Eq. 1-3): for each LP
 *     maximize  sum_j c_j x_j   s.t.  sum_j a_ij x_j <= b_i (i = 1..m),  x_j >= 0,
 * the status (optimal / infeasible / unbounded / iteration limit), an optimal
 * vertex x*, the optimum c^T x*, the duals y and the final basis.
 *
 * How (Section 3 and Section 3.1, in the paper's order):
 *   - slack form (Eq. 4): one slack x_{n+i} per row; the initial basis is the
 *     slacks.  Rows whose b_i is negative make that basis infeasible; they are
 *     negated and get one artificial variable each, and Phase I maximizes
 *     w = -(sum of artificials) (Section 3: the auxiliary LP whose objective is
 *     the sum of the artificial variables; feasible iff its optimum is 0).
 *   - the tableau (Section 3.1, Fig. 1) has the m constraint rows, the
 *     objective row, and here one more row for the Phase-I objective; its
 *     columns are the n structurals, the m slacks, the artificials and the
 *     right-hand side b.  The basic-variable index column of the paper is kept
 *     as the int array `basis`.
 *   - Step 1 (entering): the objective row stores r_j = z_j - c_j (it starts
 *     as -c).  The entering column is the most negative r_j below -eps_d, the
 *     paper's "largest coefficient" rule (LPC, Section 4.2) with the row's sign
 *     flipped.  Ties go to the lowest variable index.  No eligible column:
 *     optimal.  Under the paper's "random positive coefficient" rule (RPC,
 *     Section 4.2) the entering variable is a uniformly random eligible one:
 *     the eligible variable j with the smallest (key, j), where the key of j
 *     at pivot `it` of LP `lp` is the upper 32 bits of the first output of
 *     SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) started from the state
 *     seed ^ (lp << 40) ^ (it << 20) ^ j.  The random draw is thus a
 *     counter-based function of the LP, the pivot and the variable.  Under
 *     steepest-edge pricing (the paper has only LPC and RPC; this is the
 *     textbook rule of Goldfarb and Reid, Math. Programming 12, 1977, with the
 *     exact weights of the tableau) the entering column maximizes
 *     r_j^2 / gamma_j, gamma_j = 1 + sum_i t_ij^2 over the constraint rows in
 *     use: the squared length of the edge the pivot moves along, in the space
 *     of all variables (the entering variable moves by 1, the basic variable
 *     of row i by -t_ij).  The sum runs over the rows in order with one fused
 *     multiply-add per row; ties go to the lowest variable index.
 *   - Step 2 (leaving): among rows with pivot-column entry t_ie > eps_p, the
 *     minimum ratio b_i / t_ie.  Ties go to the lowest basic-variable index.
 *     No eligible row: unbounded.
 *   - Step 3 (pivot): the pivot row is divided by the pivot element, then
 *     every other row i has t_ie times the new pivot row subtracted
 *     (Section 4.3, the row update of Listing 1).
 *   - anti-cycling (the paper is silent): after m + n consecutive degenerate
 *     pivots (step length <= eps_p) Step 1 switches to the lowest-index
 *     eligible column (Bland's rule) until a pivot with a positive step.
 *   - after Phase I, artificials still basic at zero level are pivoted out on
 *     the largest |t_ij| > eps_p of a non-artificial column; a row with no such
 *     entry is redundant and is dropped from later ratio tests.  Artificial
 *     columns never enter.
 *
 * Parity unpinned parts: none; the tests pin the statuses and optima against
 * brute-force vertex enumeration, certificates (strong duality, KKT, Farkas
 * and ray) and an independent LP solver.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_OPTIMAL = 0, OR_INFEASIBLE = 1, OR_UNBOUNDED = 2, OR_ITER_LIMIT = 3, OR_NUMERIC = 4 };

typedef struct {
  int m, n, k;          /* rows, structurals, artificials */
  int ncol;             /* n + m + k (variables), RHS at column ncol */
  int ld;               /* ncol + 1 */
  double *T;            /* (m + 2) x ld, row-major; row m = objective, row m+1 = Phase-I objective */
  int *basis;           /* basis[i] = variable basic in row i */
  int *isbasic;         /* isbasic[j] = 1 if variable j is basic */
  int *dropped;         /* dropped[i] = 1 if row i was found redundant after Phase I */
} tableau;

#define TE(t, i, j) ((t)->T[(size_t)(i) * (t)->ld + (j)])

enum { OR_RULE_LPC = 0, OR_RULE_RPC = 1, OR_RULE_SE = 2 };
typedef struct {
  int rule;              /* OR_RULE_LPC, OR_RULE_RPC or OR_RULE_SE */
  uint64_t seed;         /* RPC: generator seed */
  uint64_t lp;           /* RPC: index of the LP in its batch */
} pivot_rule;

/* SplitMix64: advance the state by the golden-ratio increment and return the
 * mixed output (the generator of Steele, Lea and Flood, OOPSLA 2014). */
uint64_t oracle_splitmix64_next(uint64_t *state) {
  uint64_t z = (*state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

/* RPC key of variable j at pivot `it`. */
static uint32_t rpc_key(const pivot_rule *pr, uint64_t it, uint64_t j) {
  uint64_t st = pr->seed ^ (pr->lp << 40) ^ (it << 20) ^ j;
  return (uint32_t)(oracle_splitmix64_next(&st) >> 32);
}

/* Steepest-edge weight of column j: 1 + sum of t_ij^2 over the constraint
 * rows in use, in row order. */
static double se_weight(const tableau *t, int j) {
  double g = 1.0;
  for (int i = 0; i < t->m; ++i) {
    if (t->dropped[i]) continue;
    g = fma(TE(t, i, j), TE(t, i, j), g);
  }
  return g;
}

/* Step 3: pivot on (l, e). */
static void pivot(tableau *t, int l, int e) {
  const int rows = t->m + 2, ld = t->ld;
  double *pr = &t->T[(size_t)l * ld];
  const double pe = pr[e];
  for (int j = 0; j < ld; ++j) pr[j] = pr[j] / pe;
  for (int i = 0; i < rows; ++i) {
    if (i == l) continue;
    double *ri = &t->T[(size_t)i * ld];
    const double f = ri[e];
    if (f == 0.0) continue;
    for (int j = 0; j < ld; ++j) ri[j] = ri[j] - f * pr[j];
  }
  t->isbasic[t->basis[l]] = 0;
  t->basis[l] = e;
  t->isbasic[e] = 1;
}

/* Step 1 on objective row `orow` at pivot `it`; returns the entering column
 * or -1 (optimal). */
static int entering(const tableau *t, int orow, double eps_d, int bland, const pivot_rule *pr, int it) {
  const int nonart = t->n + t->m;
  int best = -1;
  double bv = 0.0;
  uint32_t bk = 0;
  for (int j = 0; j < nonart; ++j) {
    if (t->isbasic[j]) continue;
    const double r = TE(t, orow, j);
    if (!(r < -eps_d)) continue;
    if (bland) return j;                  /* lowest eligible index */
    if (pr->rule == OR_RULE_RPC) {        /* smallest (key, j): j increases, so ties keep the lower j */
      const uint32_t key = rpc_key(pr, (uint64_t)it, (uint64_t)j);
      if (best < 0 || key < bk) { best = j; bk = key; }
    } else if (pr->rule == OR_RULE_SE) {  /* largest r_j^2 / gamma_j; ties keep the lower j */
      const double score = (r * r) / se_weight(t, j);
      if (best < 0 || score > bv) { best = j; bv = score; }
    } else if (best < 0 || r < bv) {
      best = j; bv = r;
    }
  }
  return best;
}

/* Step 2 for entering column e; returns the leaving row or -1 (unbounded). */
static int leaving(const tableau *t, int e, double eps_p, double *theta) {
  int best = -1;
  double br = 0.0;
  for (int i = 0; i < t->m; ++i) {
    if (t->dropped[i]) continue;
    const double a = TE(t, i, e);
    if (!(a > eps_p)) continue;
    const double ratio = TE(t, i, t->ncol) / a;
    if (best < 0 || ratio < br || (ratio == br && t->basis[i] < t->basis[best])) {
      best = i; br = ratio;
    }
  }
  *theta = br;
  return best;
}

/* Steps 1-3 iterated on objective row `orow` until a halt condition. */
static int run_phase(tableau *t, int orow, int max_iter, int *iters, double eps_p, double eps_d,
                     int *last_e, const pivot_rule *pr) {
  int degenerate_run = 0, bland = 0;
  for (;;) {
    const int e = entering(t, orow, eps_d, bland, pr, *iters);
    if (e < 0) return OR_OPTIMAL;
    double theta;
    const int l = leaving(t, e, eps_p, &theta);
    *last_e = e;
    if (l < 0) return OR_UNBOUNDED;
    if (*iters >= max_iter) return OR_ITER_LIMIT;
    pivot(t, l, e);
    ++*iters;
    if (theta <= eps_p) {
      if (++degenerate_run >= t->m + t->n) bland = 1;
    } else {
      degenerate_run = 0;
      bland = 0;
    }
  }
}

/*
 * Solve one LP.  A is m x n row-major.  Outputs: x[n], y[m], *obj, basis[m]
 * (variable index per row: 0..n-1 structural, n..n+m-1 slack, -1 for a
 * dropped redundant row), *iters, and cert[n + m]:
 *   unbounded  -> cert[0..n-1] = a ray d >= 0 with A d <= 0 and c^T d > 0
 *   infeasible -> cert[0..m-1] = a Farkas vector u >= 0 with A^T u >= 0, b^T u < 0
 * Any output pointer may be NULL.  Returns the status.
 */
static int solve_one_rule(int m, int n, const double *A, const double *b, const double *c,
                          int max_iter, double eps_p, double eps_d, double feas_tol,
                          double *x, double *y, double *obj, int *basis_out, int *iters_out,
                          double *cert, const pivot_rule *pr) {
  tableau t;
  int k = 0;
  for (int i = 0; i < m; ++i) k += (b[i] < 0.0);
  t.m = m; t.n = n; t.k = k;
  t.ncol = n + m + k;
  t.ld = t.ncol + 1;
  t.T = (double *)calloc((size_t)(m + 2) * t.ld, sizeof(double));
  t.basis = (int *)malloc(sizeof(int) * (m > 0 ? m : 1));
  t.isbasic = (int *)calloc((size_t)t.ncol + 1, sizeof(int));
  t.dropped = (int *)calloc((size_t)(m > 0 ? m : 1), sizeof(int));
  if (!t.T || !t.basis || !t.isbasic || !t.dropped) {
    free(t.T); free(t.basis); free(t.isbasic); free(t.dropped);
    return OR_NUMERIC;
  }
  if (max_iter <= 0) max_iter = 50 * (m + n);

  /* Slack form (Eq. 4) with artificials on rows whose b_i < 0. */
  int a = 0;
  double bmax = 0.0;
  for (int i = 0; i < m; ++i) {
    const double s = (b[i] < 0.0) ? -1.0 : 1.0;
    for (int j = 0; j < n; ++j) TE(&t, i, j) = s * A[(size_t)i * n + j];
    TE(&t, i, n + i) = s;
    TE(&t, i, t.ncol) = s * b[i];
    if (fabs(b[i]) > bmax) bmax = fabs(b[i]);
    if (s < 0.0) {
      TE(&t, i, n + m + a) = 1.0;
      t.basis[i] = n + m + a;
      ++a;
    } else {
      t.basis[i] = n + i;
    }
    t.isbasic[t.basis[i]] = 1;
  }
  /* Objective row: r = -c on the structurals, value 0. */
  for (int j = 0; j < n; ++j) TE(&t, m, j) = -c[j];
  /* Phase-I row: maximize w = -sum(artificials), written in the non-basic variables. */
  for (int i = 0; i < m; ++i) {
    if (t.basis[i] < n + m) continue;
    for (int j = 0; j < n + m; ++j) TE(&t, m + 1, j) -= TE(&t, i, j);
    TE(&t, m + 1, t.ncol) -= TE(&t, i, t.ncol);
  }

  int iters = 0, status = OR_OPTIMAL, last_e = -1;
  if (k > 0) {
    status = run_phase(&t, m + 1, max_iter, &iters, eps_p, eps_d, &last_e, pr);
    if (status == OR_UNBOUNDED) status = OR_NUMERIC;   /* the auxiliary LP is bounded */
    if (status == OR_OPTIMAL) {
      const double w = TE(&t, m + 1, t.ncol);           /* = -(sum of artificials) */
      if (-w > feas_tol * (1.0 + bmax)) {
        status = OR_INFEASIBLE;
        if (cert) {                                      /* Farkas vector from the Phase-I row */
          for (int i = 0; i < m; ++i) cert[i] = TE(&t, m + 1, n + i);
        }
      } else {
        /* Drive zero-level artificials out of the basis. */
        for (int i = 0; i < m; ++i) {
          if (t.basis[i] < n + m) continue;
          int best = -1;
          double bv = eps_p;
          for (int j = 0; j < n + m; ++j) {
            if (t.isbasic[j]) continue;
            const double v = fabs(TE(&t, i, j));
            if (v > bv) { bv = v; best = j; }
          }
          if (best >= 0) { pivot(&t, i, best); ++iters; }
          else t.dropped[i] = 1;
        }
      }
    }
  }
  if (status == OR_OPTIMAL) status = run_phase(&t, m, max_iter, &iters, eps_p, eps_d, &last_e, pr);

  if (status == OR_UNBOUNDED && cert) {
    /* The entering column with no eligible row gives the ray. */
    const int e = last_e;
    for (int j = 0; j < n + m; ++j) cert[j] = 0.0;
    if (e >= 0) {
      cert[e] = 1.0;
      for (int i = 0; i < m; ++i)
        if (!t.dropped[i] && t.basis[i] < n + m) cert[t.basis[i]] = -TE(&t, i, e);
    }
  }

  if (x) for (int j = 0; j < n; ++j) x[j] = 0.0;
  if (y) for (int i = 0; i < m; ++i) y[i] = 0.0;
  if (status == OR_OPTIMAL) {
    if (x)
      for (int i = 0; i < m; ++i)
        if (t.basis[i] < n) x[t.basis[i]] = TE(&t, i, t.ncol);
    if (y)
      for (int i = 0; i < m; ++i) y[i] = TE(&t, m, n + i);
    if (obj) *obj = TE(&t, m, t.ncol);
  } else if (obj) {
    *obj = (status == OR_INFEASIBLE) ? -INFINITY : (status == OR_UNBOUNDED) ? INFINITY : NAN;
  }
  if (basis_out)
    for (int i = 0; i < m; ++i) basis_out[i] = (t.dropped[i] || t.basis[i] >= n + m) ? -1 : t.basis[i];
  if (iters_out) *iters_out = iters;

  free(t.T); free(t.basis); free(t.isbasic); free(t.dropped);
  return status;
}

int oracle_solve_one(int m, int n, const double *A, const double *b, const double *c,
                     int max_iter, double eps_p, double eps_d, double feas_tol,
                     double *x, double *y, double *obj, int *basis_out, int *iters_out,
                     double *cert) {
  const pivot_rule pr = {OR_RULE_LPC, 0, 0};
  return solve_one_rule(m, n, A, b, c, max_iter, eps_p, eps_d, feas_tol, x, y, obj, basis_out, iters_out,
                        cert, &pr);
}

/* oracle_solve_one under pivot rule `rule` (OR_RULE_LPC, OR_RULE_RPC with
 * generator seed `seed`, or OR_RULE_SE; `lp` is the LP's index in its batch). */
int oracle_solve_one_rule(int m, int n, const double *A, const double *b, const double *c,
                          int max_iter, double eps_p, double eps_d, double feas_tol,
                          double *x, double *y, double *obj, int *basis_out, int *iters_out,
                          double *cert, int rule, uint64_t seed, int64_t lp) {
  const pivot_rule pr = {rule, seed, (uint64_t)lp};
  return solve_one_rule(m, n, A, b, c, max_iter, eps_p, eps_d, feas_tol, x, y, obj, basis_out, iters_out,
                        cert, &pr);
}

/*
 * A packed batch, one LP per entry: A at a_off[k] (m[k] x n[k] row-major), b at
 * b_off[k], c at c_off[k].  Outputs x at x_off[k] (= c_off), y at y_off[k]
 * (= b_off), basis at y_off[k].  The LPs are independent and are spread over
 * `nthreads` OpenMP threads (0 = the runtime's default).
 */
void oracle_solve_batch_rule(int count, const int32_t *m, const int32_t *n,
                             const int64_t *a_off, const int64_t *b_off, const int64_t *c_off,
                             const double *A, const double *b, const double *c,
                             int max_iter, double eps_p, double eps_d, double feas_tol, int nthreads,
                             int32_t *status, double *x, double *y, double *obj,
                             int32_t *basis, int32_t *iters, int rule, uint64_t seed, int64_t first_lp) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int k = 0; k < count; ++k) {
    int it = 0;
    const pivot_rule pr = {rule, seed, (uint64_t)(first_lp + k)};
    status[k] = solve_one_rule(m[k], n[k], A + a_off[k], b + b_off[k], c + c_off[k],
                               max_iter, eps_p, eps_d, feas_tol,
                               x + c_off[k], y + b_off[k], obj + k, basis + b_off[k], &it, NULL, &pr);
    iters[k] = it;
  }
}

void oracle_solve_batch(int count, const int32_t *m, const int32_t *n,
                        const int64_t *a_off, const int64_t *b_off, const int64_t *c_off,
                        const double *A, const double *b, const double *c,
                        int max_iter, double eps_p, double eps_d, double feas_tol, int nthreads,
                        int32_t *status, double *x, double *y, double *obj,
                        int32_t *basis, int32_t *iters) {
  oracle_solve_batch_rule(count, m, n, a_off, b_off, c_off, A, b, c, max_iter, eps_p, eps_d, feas_tol,
                          nthreads, status, x, y, obj, basis, iters, OR_RULE_LPC, 0, 0);
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
