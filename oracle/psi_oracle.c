/*
 * psi_oracle.c -- plain FP64 CPU oracle for the psi-score and Power-psi.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may call this code.  It shares no code, header, table or helper with
 * the CUDA path; it is written from the paper (Arhachoui, Bautista, Danisch, Giovanidis,
 * "A Fast Algorithm for Ranking Users by their Influence in Online Social Platforms",
 * ASONAM 2022), section by section, and is deliberately slow and literal:
 *
 *   * the matrices A, B and the vectors c, d are built entry by entry from their
 *     definitions (Sec. II, the definitions that follow Eqs. 6-7): for j following i,
 *        a_ji = mu_i / sum_{l in L(j)} (lambda_l + mu_l),
 *        b_ji = lambda_i / sum_{l in L(j)} (lambda_l + mu_l),
 *        c_j  = mu_j / (lambda_j + mu_j),   d_j = lambda_j / (lambda_j + mu_j);
 *     they are stored explicitly, one value per edge (no factorisation);
 *   * Power-psi follows Algorithm 2 step by step: s <- c, B_norm <- ||B||, gap <- 1,
 *     while gap > eps { s_old <- s; s^T <- s_old^T A + c^T; gap <- B_norm ||s_old - s||_1 },
 *     psi^T <- (s^T B + d^T) / N   (Eqs. 12, 14-16);
 *   * Power-NF follows Algorithm 1 (Eq. 8) for every origin, then Eq. 7 and Eq. 1;
 *   * PageRank's power method is Eq. 22 with W = D_out^{-1} L (no dangling patch).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   * a user with no leaders has an empty newsfeed: its row of A and B is zero;
 *   * the leader set L(j) is a set: duplicate edges are merged;
 *   * the paper's model has no self-loops (Eq. 5): they are rejected, or dropped on
 *     request;
 *   * rates must be finite with lambda, mu >= 0 and lambda + mu > 0;
 *   * tolerance: gap = scale * ||s_t - s_{t-1}||_1 with scale = B_norm (1 unless the
 *     induced infinity norm max_j sum_i b_ji is asked for), divided by N in the
 *     psi-tolerance mode, which then bounds ||psi_t - psi_{t-1}||_1 by Eq. 19.
 *
 * OpenMP, when compiled in, only splits the loop over columns of one product; every
 * sum over a column and every norm is taken in a fixed sequential order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum {
  ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_ID = 2, ORC_ERR_SELF_LOOP = 3, ORC_ERR_RATE = 4,
  ORC_ERR_NOMEM = 5, ORC_NOT_CONVERGED = 7
};
enum { ORC_TOL_PSI = 0, ORC_TOL_S_ABS = 1 };
enum { ORC_BNORM_NONE = 0, ORC_BNORM_INF = 1 };

typedef struct {
  int64_t n, m;       /* users, unique follow edges */
  /* edges grouped by leader i ("column i" of A and B), followers j ascending */
  int64_t* colptr;    /* n+1 */
  int32_t* follower;  /* m: the j of each entry */
  double* a;          /* m: a_ji */
  double* b;          /* m: b_ji */
  /* edges grouped by follower j ("row j"), leaders ascending */
  int64_t* rowptr;    /* n+1 */
  int32_t* leader;    /* m */
  double* a_row;      /* m: a_ji in row order */
  double* b_row;      /* m */
  double* c;          /* n */
  double* d;          /* n */
  double* sigma;      /* n: sum over leaders of (lambda + mu); 0 if no leaders */
  double bnorm_inf;   /* max_j sum_i b_ji */
} orc_model;

typedef struct {
  int64_t iters;      /* iterations t performed */
  double gap_s;       /* ||s_t - s_{t-1}||_1 of the last iteration */
  double gap;         /* the scaled gap compared with eps */
  double bnorm;       /* the B_norm used */
  int32_t converged;
  int32_t threads;
} orc_info;

static int cmp_u64(const void* x, const void* y) {
  uint64_t a = *(const uint64_t*)x, b = *(const uint64_t*)y;
  return a < b ? -1 : (a > b ? 1 : 0);
}

int32_t orc_num_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int32_t t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/*
 * Canonical edge set: validate ids, handle self-loops, sort by (follower, leader) and
 * merge duplicates (L(j) is a set).  Writes at most m pairs; *m_out = unique count.
 */
int32_t orc_canonical_edges(int64_t n, int64_t m, const int32_t* f, const int32_t* l,
                            int32_t drop_self_loops, int32_t* f_out, int32_t* l_out,
                            int64_t* m_out) {
  if (n < 0 || m < 0) return ORC_ERR_ARG;
  uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
  if (!key) return ORC_ERR_NOMEM;
  int64_t k = 0;
  for (int64_t e = 0; e < m; ++e) {
    if (f[e] < 0 || f[e] >= n || l[e] < 0 || l[e] >= n) { free(key); return ORC_ERR_ID; }
    if (f[e] == l[e]) {
      if (!drop_self_loops) { free(key); return ORC_ERR_SELF_LOOP; }
      continue;
    }
    key[k++] = ((uint64_t)(uint32_t)f[e] << 32) | (uint32_t)l[e];
  }
  qsort(key, (size_t)k, sizeof(uint64_t), cmp_u64);
  int64_t u = 0;
  for (int64_t e = 0; e < k; ++e) {
    if (e > 0 && key[e] == key[e - 1]) continue;
    f_out[u] = (int32_t)(key[e] >> 32);
    l_out[u] = (int32_t)(key[e] & 0xFFFFFFFFULL);
    ++u;
  }
  free(key);
  *m_out = u;
  return ORC_OK;
}

void orc_model_destroy(orc_model* g) {
  if (!g) return;
  free(g->colptr); free(g->follower); free(g->a); free(g->b);
  free(g->rowptr); free(g->leader); free(g->a_row); free(g->b_row);
  free(g->c); free(g->d); free(g->sigma);
  free(g);
}

/*
 * Build A, B, c, d from the definitions.  (f, l) is any edge list (validated and made
 * canonical here); lambda and mu have n entries.
 */
orc_model* orc_model_create(int64_t n, int64_t m, const int32_t* f, const int32_t* l,
                            const double* lambda, const double* mu, int32_t drop_self_loops,
                            int32_t* status) {
  *status = ORC_OK;
  if (n <= 0 || m < 0) { *status = ORC_ERR_ARG; return NULL; }
  for (int64_t i = 0; i < n; ++i) {
    double x = lambda[i], y = mu[i];
    if (!isfinite(x) || !isfinite(y) || x < 0.0 || y < 0.0 || !(x + y > 0.0)) {
      *status = ORC_ERR_RATE;
      return NULL;
    }
  }
  orc_model* g = (orc_model*)calloc(1, sizeof(orc_model));
  int32_t* cf = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int32_t* cl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  if (!g || !cf || !cl) { free(g); free(cf); free(cl); *status = ORC_ERR_NOMEM; return NULL; }
  int64_t mu_n = 0;
  int32_t st = orc_canonical_edges(n, m, f, l, drop_self_loops, cf, cl, &mu_n);
  if (st != ORC_OK) { free(g); free(cf); free(cl); *status = st; return NULL; }
  g->n = n;
  g->m = mu_n;
  size_t mm = (size_t)(mu_n > 0 ? mu_n : 1);
  g->colptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  g->rowptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  g->follower = (int32_t*)malloc(sizeof(int32_t) * mm);
  g->leader = (int32_t*)malloc(sizeof(int32_t) * mm);
  g->a = (double*)malloc(sizeof(double) * mm);
  g->b = (double*)malloc(sizeof(double) * mm);
  g->a_row = (double*)malloc(sizeof(double) * mm);
  g->b_row = (double*)malloc(sizeof(double) * mm);
  g->c = (double*)malloc(sizeof(double) * (size_t)n);
  g->d = (double*)malloc(sizeof(double) * (size_t)n);
  g->sigma = (double*)calloc((size_t)n, sizeof(double));
  if (!g->colptr || !g->rowptr || !g->follower || !g->leader || !g->a || !g->b || !g->a_row ||
      !g->b_row || !g->c || !g->d || !g->sigma) {
    free(cf); free(cl); orc_model_destroy(g); *status = ORC_ERR_NOMEM; return NULL;
  }
  /* rows j: the canonical list is sorted by (follower, leader) already */
  for (int64_t e = 0; e < mu_n; ++e) g->rowptr[cf[e] + 1]++;
  for (int64_t j = 0; j < n; ++j) g->rowptr[j + 1] += g->rowptr[j];
  for (int64_t e = 0; e < mu_n; ++e) g->leader[e] = cl[e];
  /* sigma_j = sum_{l in L(j)} (lambda_l + mu_l)  (denominator of a_ji, b_ji) */
  for (int64_t j = 0; j < n; ++j) {
    double s = 0.0;
    for (int64_t e = g->rowptr[j]; e < g->rowptr[j + 1]; ++e) {
      int32_t ll = g->leader[e];
      s += lambda[ll] + mu[ll];
    }
    g->sigma[j] = s;
  }
  /* a_ji and b_ji for every edge j -> i, in row order */
  for (int64_t j = 0; j < n; ++j)
    for (int64_t e = g->rowptr[j]; e < g->rowptr[j + 1]; ++e) {
      int32_t i = g->leader[e];
      g->a_row[e] = mu[i] / g->sigma[j];
      g->b_row[e] = lambda[i] / g->sigma[j];
    }
  /* ||B||_inf = max_j sum_i b_ji */
  double bn = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double s = 0.0;
    for (int64_t e = g->rowptr[j]; e < g->rowptr[j + 1]; ++e) s += g->b_row[e];
    if (s > bn) bn = s;
  }
  g->bnorm_inf = bn;
  /* columns i: stable counting sort of the row-ordered entries by leader */
  for (int64_t e = 0; e < mu_n; ++e) g->colptr[cl[e] + 1]++;
  for (int64_t i = 0; i < n; ++i) g->colptr[i + 1] += g->colptr[i];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!fill) { free(cf); free(cl); orc_model_destroy(g); *status = ORC_ERR_NOMEM; return NULL; }
  for (int64_t i = 0; i < n; ++i) fill[i] = g->colptr[i];
  for (int64_t e = 0; e < mu_n; ++e) {
    int64_t p = fill[cl[e]]++;
    g->follower[p] = cf[e];
    g->a[p] = g->a_row[e];
    g->b[p] = g->b_row[e];
  }
  free(fill);
  /* c and d: diagonals of C and D */
  for (int64_t i = 0; i < n; ++i) {
    g->c[i] = mu[i] / (lambda[i] + mu[i]);
    g->d[i] = lambda[i] / (lambda[i] + mu[i]);
  }
  free(cf);
  free(cl);
  return g;
}

void orc_model_dims(const orc_model* g, int64_t* n, int64_t* m, double* bnorm_inf) {
  *n = g->n;
  *m = g->m;
  *bnorm_inf = g->bnorm_inf;
}

void orc_model_vectors(const orc_model* g, double* c, double* d, double* sigma) {
  memcpy(c, g->c, sizeof(double) * (size_t)g->n);
  memcpy(d, g->d, sizeof(double) * (size_t)g->n);
  memcpy(sigma, g->sigma, sizeof(double) * (size_t)g->n);
}

/* canonical edges back out (follower, leader), sorted by (follower, leader) */
void orc_model_edges(const orc_model* g, int32_t* f, int32_t* l) {
  for (int64_t j = 0; j < g->n; ++j)
    for (int64_t e = g->rowptr[j]; e < g->rowptr[j + 1]; ++e) {
      f[e] = (int32_t)j;
      l[e] = g->leader[e];
    }
}

/* out_i = sum_j s_j x_ji over the entries of column i: the row-vector product s^T X */
static void row_vec_times(const orc_model* g, const double* x, const double* s, double* out) {
  const int64_t n = g->n;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int64_t e = g->colptr[i]; e < g->colptr[i + 1]; ++e) acc += s[g->follower[e]] * x[e];
    out[i] = acc;
  }
}

/* sA = s^T A and sB = s^T B (either output may be NULL) */
void orc_apply_AB(const orc_model* g, const double* s, double* sA, double* sB) {
  if (sA) row_vec_times(g, g->a, s, sA);
  if (sB) row_vec_times(g, g->b, s, sB);
}

/* psi^T = (s^T B + d^T) / N  (Algorithm 2, final step; Eq. 12) */
void orc_psi_from_s(const orc_model* g, const double* s, double* psi) {
  row_vec_times(g, g->b, s, psi);
  for (int64_t i = 0; i < g->n; ++i) psi[i] = (psi[i] + g->d[i]) / (double)g->n;
}

/*
 * Power-psi, Algorithm 2.  s_init (nullable) replaces the start s_0 = c (a warm start
 * changes the iteration count only).  With to_floor != 0 the loop ignores eps and runs
 * until the FP64 gap is 0 or has not decreased for 8 iterations (the rounding floor),
 * or max_iter.  gap_hist (nullable, max_iter entries) receives the unscaled
 * ||s_t - s_{t-1}||_1 of every iteration.
 */
int32_t orc_power_psi(const orc_model* g, double eps, int32_t tol_mode, int32_t bnorm_mode,
                      int64_t max_iter, int32_t to_floor, const double* s_init, double* s_out,
                      double* psi_out, double* gap_hist, orc_info* info) {
  const int64_t n = g->n;
  double* s = (double*)malloc(sizeof(double) * (size_t)n);
  double* s_old = (double*)malloc(sizeof(double) * (size_t)n);
  if (!s || !s_old) { free(s); free(s_old); return ORC_ERR_NOMEM; }
  const double B_norm = (bnorm_mode == ORC_BNORM_INF) ? g->bnorm_inf : 1.0;
  const double scale = B_norm * (tol_mode == ORC_TOL_PSI ? 1.0 / (double)n : 1.0);
  for (int64_t i = 0; i < n; ++i) s[i] = s_init ? s_init[i] : g->c[i];
  int64_t t = 0;
  double gap = 1.0, gap_s = 0.0, best = INFINITY;
  int64_t stale = 0;
  while (t < max_iter && (to_floor || gap > eps)) {
    memcpy(s_old, s, sizeof(double) * (size_t)n);
    row_vec_times(g, g->a, s_old, s);         /* s^T <- s_old^T A ... */
    for (int64_t i = 0; i < n; ++i) s[i] += g->c[i]; /* ... + c^T  (Eq. 14) */
    double acc = 0.0;                         /* ||s_old - s||_1  (Eq. 15) */
    for (int64_t i = 0; i < n; ++i) acc += fabs(s_old[i] - s[i]);
    gap_s = acc;
    gap = scale * acc;
    if (gap_hist) gap_hist[t] = acc;
    ++t;
    if (to_floor) {
      if (acc == 0.0) break;
      if (acc < best) { best = acc; stale = 0; } else if (++stale >= 8) break;
    }
  }
  if (s_out) memcpy(s_out, s, sizeof(double) * (size_t)n);
  if (psi_out) orc_psi_from_s(g, s, psi_out);
  if (info) {
    info->iters = t;
    info->gap_s = gap_s;
    info->gap = gap;
    info->bnorm = B_norm;
    info->converged = (gap <= eps) ? 1 : 0;
    info->threads = orc_num_threads();
  }
  free(s);
  free(s_old);
  return (to_floor || gap <= eps) ? ORC_OK : ORC_NOT_CONVERGED;
}

/*
 * Power-NF, Algorithm 1, for one origin i: p_i <- b_i; while gap > eps
 * { p_old <- p_i; p_i <- A p_old + b_i; gap <- ||p_i - p_old||_1 }; then
 * q_i = C p_i + d_i (Eq. 7) and psi_i = (1/N) sum_n q_i^(n) (Eq. 1).  p, po, bi are
 * scratch vectors of n entries; adds the matrix-vector products to *mv and returns 1 if
 * the origin met its test.
 */
static int nf_origin(const orc_model* g, int64_t i, double eps, int64_t max_iter, double* p, double* po,
                     double* bi, double* psi_i, int64_t* mv) {
  const int64_t n = g->n;
  /* b_i: column i of B, entries b_ji for the followers j of i */
  for (int64_t j = 0; j < n; ++j) bi[j] = 0.0;
  for (int64_t e = g->colptr[i]; e < g->colptr[i + 1]; ++e) bi[g->follower[e]] = g->b[e];
  for (int64_t j = 0; j < n; ++j) p[j] = bi[j];
  double gap = 1.0;
  int64_t t = 0;
  while (gap > eps && t < max_iter) {
    memcpy(po, p, sizeof(double) * (size_t)n);
    for (int64_t j = 0; j < n; ++j) { /* (A p_old)_j = sum_{k in L(j)} a_jk p_old_k */
      double acc = 0.0;
      for (int64_t e = g->rowptr[j]; e < g->rowptr[j + 1]; ++e) acc += g->a_row[e] * po[g->leader[e]];
      p[j] = acc + bi[j];
    }
    double acc = 0.0;
    for (int64_t j = 0; j < n; ++j) acc += fabs(p[j] - po[j]);
    gap = acc;
    ++t;
    ++*mv;
  }
  /* q_i^(n) = c_n p_i^(n) + d_i 1{n = i};  psi_i = mean over n */
  double q = 0.0;
  for (int64_t j = 0; j < n; ++j) q += g->c[j] * p[j];
  q += g->d[i];
  *psi_i = q / (double)n;
  return gap <= eps;
}

/*
 * Power-NF (Algorithm 1) for the origins listed in origins[0..count) (input ids), or for
 * every origin in order when origins is NULL (count is then ignored): psi_out[q] is the
 * score of the q-th origin.  Each origin is an independent problem in Algorithm 1, so a
 * subset gives the same values as the full run.  Counts matrix-vector products in
 * *matvecs.  Meant for small N, or for a few origins of a larger graph.
 */
int32_t orc_power_nf_origins(const orc_model* g, double eps, int64_t max_iter, const int64_t* origins,
                             int64_t count, double* psi_out, int64_t* matvecs) {
  const int64_t n = g->n;
  if (!origins) count = n;
  double* p = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* po = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* bi = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!p || !po || !bi) { free(p); free(po); free(bi); return ORC_ERR_NOMEM; }
  int64_t mv = 0;
  int32_t st = ORC_OK;
  for (int64_t q = 0; q < count; ++q) {
    const int64_t i = origins ? origins[q] : q;
    if (i < 0 || i >= n) { st = ORC_ERR_ID; break; }
    if (!nf_origin(g, i, eps, max_iter, p, po, bi, &psi_out[q], &mv)) st = ORC_NOT_CONVERGED;
  }
  if (matvecs) *matvecs = mv;
  free(p);
  free(po);
  free(bi);
  return st;
}

/* Power-NF (Algorithm 1) for every origin: psi_out[i] for i = 0..n-1. */
int32_t orc_power_nf(const orc_model* g, double eps, int64_t max_iter, double* psi_out,
                     int64_t* matvecs) {
  return orc_power_nf_origins(g, eps, max_iter, NULL, 0, psi_out, matvecs);
}

/*
 * Newsfeed mass m = (I - A)^{-1} B 1 by the iteration m <- A m + B 1, run to the FP64
 * floor: m_j is the total share of posts on j's newsfeed (1 if j has a leader, 0 if not).
 * Used for the identity sum_i psi_i = (sum_n d_n + c^T m) / N.
 */
int64_t orc_newsfeed_mass(const orc_model* g, int64_t max_iter, double* m_out) {
  const int64_t n = g->n;
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* mo = (double*)malloc(sizeof(double) * (size_t)n);
  if (!r || !mo) { free(r); free(mo); return -1; }
  for (int64_t j = 0; j < n; ++j) {
    double acc = 0.0;
    for (int64_t e = g->rowptr[j]; e < g->rowptr[j + 1]; ++e) acc += g->b_row[e];
    r[j] = acc;
    m_out[j] = acc;
  }
  int64_t t = 0;
  double best = INFINITY;
  int64_t stale = 0;
  while (t < max_iter) {
    memcpy(mo, m_out, sizeof(double) * (size_t)n);
    double gap = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int64_t e = g->rowptr[j]; e < g->rowptr[j + 1]; ++e) acc += g->a_row[e] * mo[g->leader[e]];
      m_out[j] = acc + r[j];
      gap += fabs(m_out[j] - mo[j]);
    }
    ++t;
    if (gap == 0.0) break;
    if (gap < best) { best = gap; stale = 0; } else if (++stale >= 8) break;
  }
  free(r);
  free(mo);
  return t;
}

/*
 * PageRank power method, Eq. 22: pi_t^T = alpha pi_{t-1}^T W + (1-alpha)/N 1^T with
 * W = D_out^{-1} L, L_ji = 1 if j follows i, D_out the number of leaders; a user with
 * no leaders has a zero row (no dangling redistribution).  Start pi_0 = 1/N; runs to the
 * FP64 floor or max_iter.  Edges must be canonical (sorted, unique, no self-loops).
 */
int64_t orc_pagerank(int64_t n, int64_t m, const int32_t* f, const int32_t* l, double alpha,
                     int64_t max_iter, double* pi_out) {
  double* outdeg = (double*)calloc((size_t)n, sizeof(double));
  double* po = (double*)malloc(sizeof(double) * (size_t)n);
  if (!outdeg || !po) { free(outdeg); free(po); return -1; }
  for (int64_t e = 0; e < m; ++e) outdeg[f[e]] += 1.0;
  for (int64_t i = 0; i < n; ++i) pi_out[i] = 1.0 / (double)n;
  int64_t t = 0;
  double best = INFINITY;
  int64_t stale = 0;
  while (t < max_iter) {
    memcpy(po, pi_out, sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) pi_out[i] = 0.0;
    for (int64_t e = 0; e < m; ++e) pi_out[l[e]] += po[f[e]] / outdeg[f[e]];
    double gap = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      pi_out[i] = alpha * pi_out[i] + (1.0 - alpha) / (double)n;
      gap += fabs(pi_out[i] - po[i]);
    }
    ++t;
    if (gap == 0.0) break;
    if (gap < best) { best = gap; stale = 0; } else if (++stale >= 8) break;
  }
  free(outdeg);
  free(po);
  return t;
}

/* ranking: psi descending, ties by id ascending; first k */
static const double* g_sort_psi;
static int cmp_rank(const void* x, const void* y) {
  int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
  double pa = g_sort_psi[a], pb = g_sort_psi[b];
  if (pa > pb) return -1;
  if (pa < pb) return 1;
  return a < b ? -1 : (a > b ? 1 : 0);
}

int32_t orc_topk(int64_t n, const double* psi, int64_t k, int32_t* ids, double* vals) {
  int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!idx) return ORC_ERR_NOMEM;
  for (int64_t i = 0; i < n; ++i) idx[i] = (int32_t)i;
  g_sort_psi = psi;
  qsort(idx, (size_t)n, sizeof(int32_t), cmp_rank);
  if (k > n) k = n;
  for (int64_t i = 0; i < k; ++i) {
    ids[i] = idx[i];
    vals[i] = psi[idx[i]];
  }
  free(idx);
  return ORC_OK;
}
