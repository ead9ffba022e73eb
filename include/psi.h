/*
 * psi.h -- C ABI of the GB300 Power-psi solver (libpsi_gb300.so).
 *
 * Computes the psi-score of every user of a follower graph (Arhachoui, Bautista,
 * Danisch, Giovanidis, "A Fast Algorithm for Ranking Users by their Influence in Online
 * Social Platforms", ASONAM 2022):
 *
 *   psi^T = (1/N) [ (sum_{t>=0} c^T A^t) B + d^T ]                        (Eq. 12)
 *
 * with, for user j following user i (L(j) = leaders of j):
 *   a_ji = mu_i / sigma_j,  b_ji = lambda_i / sigma_j,  sigma_j = sum_{l in L(j)} (lambda_l + mu_l),
 *   c_j = mu_j / (lambda_j + mu_j),  d_j = lambda_j / (lambda_j + mu_j)   (Sec. II, Eqs. 6-7).
 *
 * The series is evaluated by Power-psi (Algorithm 2): s_0 = c, s_t^T = s_{t-1}^T A + c^T
 * (Eq. 14), gap eps_t = ||s_t - s_{t-1}||_1 (Eq. 15), stop when the scaled gap <= eps
 * (Eq. 16), then psi^T = (s_t^T B + d^T) / N.
 *
 * Conventions for every call:
 *   * Every function returns a psi_status; none aborts, traps or exits.  On failure a
 *     message is available from psi_last_error() (thread-local, valid until the next
 *     call on the same thread).
 *   * Array arguments may be host or device pointers (detected per call).  Inputs are
 *     copied and never retained; the caller keeps ownership of everything it passes.
 *   * Work is queued on the CUDA stream given in psi_options.stream (NULL = the legacy
 *     default stream).  psi_graph_create, psi_solve, psi_scores, psi_topk and
 *     psi_get_iterate return after their results are complete (they synchronise that
 *     stream once at the end, plus a few small status reads on the way).
 *   * User ids are 0-based int32; n < 2^31 and the edge count m < 2^31 - 1.
 *   * A graph handle may be used by one host thread at a time.
 */
#ifndef PSI_GB300_H
#define PSI_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct psi_graph psi_graph; /* opaque; owns all of its device memory */

typedef enum psi_status {
  PSI_OK = 0,
  PSI_ERR_INVALID_ARG = 1,     /* null pointer, negative size, unknown option, k out of range */
  PSI_ERR_OUT_OF_RANGE_ID = 2, /* an edge endpoint outside [0, n) */
  PSI_ERR_SELF_LOOP = 3,       /* a user follows itself and self_loops == PSI_REJECT */
  PSI_ERR_BAD_RATE = 4,        /* lambda or mu NaN, infinite or negative, or lambda + mu == 0 */
  PSI_ERR_OOM = 5,             /* the allocator returned NULL */
  PSI_ERR_CUDA = 6,            /* a CUDA runtime error (message in psi_last_error) */
  PSI_ERR_NOT_CONVERGED = 7,   /* max_iter reached; the last iterate and psi stay readable */
  PSI_ERR_TIMEOUT = 8,         /* a bounded device-side wait gave up */
  PSI_ERR_NOT_SOLVED = 9       /* scores asked for before a solve produced them */
} psi_status;

/* psi_options.precision */
enum {
  PSI_FP32 = 0,        /* Algorithm 2 literally, iterate stored and summed in FP32;
                          stalls near the FP32 rounding floor for tight eps */
  PSI_FP32_REFINE = 1, /* default: the series of Eq. 13 with FP32 terms summed into an
                          FP64 iterate, then confirming steps from that iterate near eps (see
                          psi_solve) */
  PSI_FP64 = 2         /* Algorithm 2 literally in FP64 */
};
/* psi_options.tol_mode: scale applied to eps_t before the test of Eq. 16 */
enum {
  PSI_TOL_PSI = 0,   /* default: B_norm * eps_t / N, a bound on ||psi_t - psi_{t-1}||_1 (Eq. 19) */
  PSI_TOL_S_ABS = 1  /* B_norm * eps_t, the paper's s-tolerance */
};
/* psi_options.bnorm_mode: the B_norm of Algorithm 2 */
enum {
  PSI_BNORM_NONE = 0, /* default: 1 (>= ||B||_inf, so the more conservative test) */
  PSI_BNORM_INF = 1   /* ||B||_inf = max_j sum_i b_ji */
};
/* psi_options.self_loops (the model has no self-loops, Eq. 5) */
enum { PSI_REJECT = 0, PSI_DROP = 1 };

/* Optional device allocator.  alloc returns device memory of `bytes` usable on
 * `stream` (or NULL on failure); free releases it.  Default: cudaMallocAsync /
 * cudaFreeAsync on the options' stream. */
typedef struct psi_allocator {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, size_t bytes, void* stream, void* ctx);
  void* ctx;
} psi_allocator;

typedef struct psi_options {
  int32_t precision;   /* PSI_FP32 | PSI_FP32_REFINE | PSI_FP64 */
  int32_t tol_mode;    /* PSI_TOL_PSI | PSI_TOL_S_ABS */
  int32_t bnorm_mode;  /* PSI_BNORM_NONE | PSI_BNORM_INF */
  int32_t self_loops;  /* PSI_REJECT | PSI_DROP */
  int32_t reorder;     /* 1 (default): number users internally by class and in-degree so
                          the gathered iterate is compact in L2; 0: keep the input order
                          within each class.  Results do not depend on it beyond rounding. */
  int32_t profile;     /* 1: time every sparse product with CUDA events (psi_solve_info) */
  int32_t spmv_tile;   /* nonzeros per tile of the sparse product (one warp per tile): 0
                          (default) picks 2048, 1024 or 512 from the edge count so that small
                          graphs still spread over every SM (psi_multi_create: 512); else
                          one of 512, 1024, 2048.  Results do not depend on it beyond
                          rounding. */
  void* stream;        /* cudaStream_t to queue all work on */
  const psi_allocator* allocator; /* NULL: cudaMallocAsync on stream */
  int32_t autotune;    /* 1 (default): the first psi_solve of a graph of at least 2^22 nonzeros
                          times the candidate configurations of the FP32 series product (tile of
                          512/1024/2048 nonzeros unless spmv_tile fixes it; 0, 24576, 28672 or
                          32768 most-gathered entries kept in shared memory) on the graph itself
                          and keeps the fastest, remembered for later graphs of the same sizes
                          in this process; 0: the fixed rule of spmv_tile, no shared-memory copy.
                          Results do not depend on it beyond rounding.  PSI_FP32_REFINE only. */
  int32_t spmv_hot;    /* -1 (default): chosen by the autotuner (0 without it); 0, 24576, 28672
                          or 32768: that many most-gathered entries of the FP32 series product
                          read from shared memory (at most the gathered users), which the
                          autotuner then keeps.  Results do not depend on it beyond rounding. */
} psi_options;

/* Fills the defaults listed above. */
void psi_options_default(psi_options* opt);

typedef struct psi_solve_info {
  int32_t iters;          /* power-iteration steps t performed (each yields s_t) */
  int32_t converged;      /* 1 if the scaled gap met eps */
  int32_t refinements;    /* confirming steps taken (PSI_FP32_REFINE) */
  int32_t spmv_launches;  /* sparse products run (iterations + final psi product) */
  double gap_s_l1;        /* eps_t = ||s_t - s_{t-1}||_1 of the last step */
  double gap_scaled;      /* the value compared with eps (tol_mode, bnorm_mode) */
  double gap_psi_bound;   /* eps_t * ||B||_inf / N, bounds ||psi_t - psi_{t-1}||_1 (Eq. 19) */
  double psi_sum;         /* sum_i psi_i (FP64); 1 when every user has a leader */
  double ms;              /* wall time of the solve on the stream (CUDA events) */
  double spmv_ms;         /* profile == 1: summed duration of the main-precision steps (FP32
                             series or FP32/FP64 Algorithm 2 steps): sparse product + fix-up */
  int32_t spmv_timed;     /* profile == 1: number of steps in spmv_ms */
  int32_t refine_timed;   /* profile == 1: number of confirming steps in refine_ms */
  double refine_ms;       /* profile == 1: summed duration of the confirming steps */
} psi_solve_info;

typedef struct psi_graph_stats {
  int64_t n;              /* users */
  int64_t m_input;        /* edges passed in */
  int64_t m_unique;       /* distinct follow edges after self-loop handling and merging */
  int64_t n_rows;         /* users with at least one follower (rows of the iteration) */
  int64_t n_gathered;     /* users with at least one leader (entries of the gathered iterate) */
  int64_t max_followers;  /* largest row */
  double bnorm_inf;       /* ||B||_inf */
  double rho_inf;         /* max_j sum_{l in L(j)} mu_l / sigma_j (< 1: contraction rate bound) */
  double build_ms;        /* wall time of psi_graph_create on the stream */
  int64_t device_bytes;   /* device memory held by the handle */
  int64_t spmv_tile;      /* nonzeros per tile of the sparse product (psi_options.spmv_tile) */
  int64_t spmv_hot;       /* entries of the FP32 series product's gathered vector read from
                             shared memory (0: none; psi_options.autotune) */
  double tune_ms;         /* time the autotuner spent timing candidates on this handle (0 when
                             the choice came from an earlier graph of the same sizes) */
} psi_graph_stats;

/*
 * Build the operator of Sec. II from an edge list.  Edge k: user follower[k] follows user
 * leader[k] (Sec. II).  Duplicate edges are merged (L(j) is a set); self-loops are
 * rejected or dropped per opt->self_loops.  lambda[i], mu[i]: posting and re-posting rates
 * of user i (n entries, FP64).  opt may be NULL (defaults).  m may be 0.
 * sigma_j and beta_j = sum_{l in L(j)} lambda_l are exact sums rounded once to FP64 when
 * the binary exponents of all nonzero rates lie within 40 of the smallest and none is
 * subnormal (they then do not depend on the order of the edges); otherwise they are
 * float-pair sums (about 48 bits; FP64 sums with PSI_FP64).
 * Errors: INVALID_ARG, OUT_OF_RANGE_ID, SELF_LOOP, BAD_RATE, OOM, CUDA; *out is NULL then.
 */
psi_status psi_graph_create(int64_t n, int64_t m, const int32_t* follower, const int32_t* leader,
                            const double* lambda, const double* mu, const psi_options* opt,
                            psi_graph** out);

/*
 * Power-psi (Algorithm 2) to tolerance eps with at most max_iter steps, then psi.
 * init_s (nullable, n FP64 values, host or device) replaces s_0 = c (warm start or
 * resume; the fixed point does not change).  Returns OK or NOT_CONVERGED (psi is then
 * computed from the last iterate).  info may be NULL.
 * PSI_FP32_REFINE: the terms c^T A^t of Eq. 13 are formed in FP32 and summed into an
 * FP64 s; when their gap meets eps, one confirming step s <- s A + c is taken from that s
 * and its gap is the one tested (repeating the FP32 series from its residual if needed), so
 * the returned gap is a gap of Algorithm 2 taken at the confirming step's precision.  The
 * confirming step and the final product sum the gathered values as float pairs (hi + lo
 * FP32, about 48 significant bits; each pair sum errs by at most ~2^-46 of the magnitudes
 * summed) and update s and psi in FP64, whenever the target gap eps/scale is at least
 * 2^-30 * n (true of the default psi tolerance for eps >= 1e-9); tighter targets, such as
 * an absolute s-tolerance of 1e-9 on millions of users, take FP64 products throughout.
 */
psi_status psi_solve(psi_graph* g, double eps, int32_t max_iter, const double* init_s,
                     psi_solve_info* info);

/* psi of every user (n FP64 values, host or device), in input user ids. */
psi_status psi_scores(const psi_graph* g, double* psi_out);

/*
 * The k highest psi (descending; equal psi by ascending user id): ids_out[k] int32 and
 * vals_out[k] FP64, host or device (vals_out may be NULL).  1 <= k <= min(n, 65536);
 * larger k is INVALID_ARG.
 */
psi_status psi_topk(const psi_graph* g, int32_t k, int32_t* ids_out, double* vals_out);

/* The last iterate s_t (n FP64 values, input user ids): resume or warm-start source. */
psi_status psi_get_iterate(const psi_graph* g, double* s_out);

/* Sizes and norms of the built operator. */
psi_status psi_graph_get_stats(const psi_graph* g, psi_graph_stats* stats);

/* Releases the handle and its device memory (NULL is ignored). */
void psi_graph_destroy(psi_graph* g);

const char* psi_status_string(psi_status s);
const char* psi_last_error(void);

/*
 * psi_pagerank -- the PageRank power method of Eq. 22 on the graph's follower structure:
 * pi_t = alpha * pi_{t-1} W + (1 - alpha)/N, with W the walk from a user to one of its
 * leaders chosen uniformly (a user without leaders has a zero row: no dangling
 * redistribution), pi_0 = 1/N, stopped when ||pi_t - pi_{t-1}||_1 <= eps (the paper's
 * pi-tolerance) or after max_iter steps.  It runs the Power-psi kernels with c = (1-alpha)/N,
 * mu = alpha, 1/sigma_j = 1/|L(j)| in the handle's precision mode; the graph's rates are not
 * used.  When every user has the same lambda and mu, psi_solve's psi equals this pi with
 * alpha = mu/(lambda+mu) (Sec. III).
 *   alpha: damping factor in [0, 1).  pi_out: n FP64 values in input order, host or device
 *   (may be NULL).  info: may be NULL; iters, converged, gap_s_l1 = the last pi gap,
 *   psi_sum = sum of pi.
 * The handle's psi scores are left as they were; its iterate (psi_get_iterate) is pi's.
 * Returns OK, NOT_CONVERGED (pi still written) or an error (INVALID_ARG for alpha).
 */
psi_status psi_pagerank(psi_graph* g, double alpha, double eps, int32_t max_iter, double* pi_out,
                        psi_solve_info* info);

/*
 * psi_power_nf -- Power-NF (Algorithm 1), the method Power-psi replaces: for every origin
 * user i, the newsfeed vector of Eq. 8, p_i <- A p_i + b_i from p_i = b_i, until
 * ||p_i^t - p_i^{t-1}||_1 <= eps (each origin on its own test; a gap of 1 before the first
 * step) or max_iter steps; then q_i = C p_i + d_i (Eq. 7) and psi_i = (1/N) sum_n q_i^(n)
 * (Eq. 1), in FP64.  Origins are stepped together in passes, as the columns of a matrix
 * with one row per user that has leaders (users without leaders have p = 0; origins without
 * followers have p_i = 0 and psi_i = d_i / N).  origins_per_pass: origins per pass, 0 to
 * take as many as a quarter of the free device memory holds (6 to 32 GiB of pass state,
 * two FP64 matrices); results do not depend on it.  The cost is that of about N Power-psi
 * solves.  psi_out: n FP64 values in input
 * order, host or device (may be NULL).  info (may be NULL): iters = the most steps any
 * origin took, spmv_launches = the matrix-vector products of Algorithm 1 (steps summed over
 * origins, saturating at INT32_MAX), gap_s_l1 = the largest last gap, converged, ms.  The
 * handle's psi scores are left as they were.
 * Returns OK, NOT_CONVERGED (psi still written) or an error (INVALID_ARG for more than 2^20
 * users with leaders, a negative origins_per_pass, NaN eps or a negative max_iter).
 */
psi_status psi_power_nf(psi_graph* g, double eps, int32_t max_iter, int32_t origins_per_pass, double* psi_out,
                        psi_solve_info* info);

/* ------------------------------------------------------------------------------------
 * Scenario batches: S sets of activity rates (lambda, mu) on one follower graph, solved
 * together.  Each scenario is an independent Power-psi problem (Algorithm 2 with its own
 * A, B, c, d from Sec. II, its own gap, stop test and step count); one sparse product per
 * step serves every scenario, so each column index fetched feeds S values.  Precision is
 * always PSI_FP32_REFINE (FP32 series, FP64 iterate, confirming step and final product in
 * float pairs or FP64 as for psi_solve, FP64 psi).
 */
typedef struct psi_batch psi_batch; /* opaque; owns all of its device memory */

/*
 * follower/leader/m as in psi_graph_create.  lambda and mu hold S * n FP64 values,
 * scenario-major (scenario q's rates at [q * n, (q+1) * n)), host or device.
 * 1 <= S <= 64.  Every scenario's rates are validated (PSI_ERR_BAD_RATE).
 */
psi_status psi_batch_create(int64_t n, int64_t m, const int32_t* follower, const int32_t* leader, int32_t S,
                            const double* lambda, const double* mu, const psi_options* opt, psi_batch** out);

/* Power-psi for every scenario to eps (scaled per opt->tol_mode / bnorm_mode, each scenario
 * with its own ||B||_inf), at most max_iter steps each.  info may be NULL or hold S entries.
 * Returns OK when every scenario converged, else NOT_CONVERGED (psi still computed). */
psi_status psi_batch_solve(psi_batch* b, double eps, int32_t max_iter, psi_solve_info* info);

/* psi of every scenario: S * n FP64 values, scenario-major, input user ids. */
psi_status psi_batch_scores(const psi_batch* b, double* psi_out);

/* The k highest psi of every scenario (as psi_topk): ids_out[S * k], vals_out[S * k]
 * (vals_out may be NULL), scenario-major. */
psi_status psi_batch_topk(const psi_batch* b, int32_t k, int32_t* ids_out, double* vals_out);

psi_status psi_batch_get_stats(const psi_batch* b, psi_graph_stats* stats);
void psi_batch_destroy(psi_batch* b);

/* ------------------------------------------------------------------------------------
 * Independent graphs: G follower graphs of their own (own users, N_g, edges, rates), each
 * solved as its own Power-psi problem (Algorithm 2 with its own N_g in psi = (.)/N_g and in
 * the psi tolerance, its own gap, stop test, step count and confirming step), all in
 * one object: the graphs are built together as one block-diagonal graph and stepped
 * together, graphs that have met their test skipping their part of each product, from a
 * CUDA graph of captured steps.  Precision is always PSI_FP32_REFINE.
 */
typedef struct psi_multi psi_multi; /* opaque; owns all of its device memory */

/*
 * 1 <= G <= 1024.  n_g[G], m_g[G]: host arrays, n_g >= 1, m_g >= 0, sums below 2^31 - 1.
 * follower/leader: sum(m_g) int32 ids, graph by graph (graph q's edges at
 * [m_0 + .. + m_{q-1}, +m_q)), each id LOCAL to its graph, in [0, n_g); host or device.
 * lambda/mu: sum(n_g) FP64 rates, graph by graph, host or device.  Errors as in
 * psi_graph_create (an id outside its own graph: PSI_ERR_OUT_OF_RANGE_ID).
 */
psi_status psi_multi_create(int32_t G, const int64_t* n_g, const int64_t* m_g, const int32_t* follower,
                            const int32_t* leader, const double* lambda, const double* mu, const psi_options* opt,
                            psi_multi** out);

/* Power-psi for every graph to eps (scaled per opt->tol_mode / bnorm_mode with the graph's
 * own N_g and ||B||_inf), at most max_iter steps each.  info may be NULL or hold G entries.
 * Returns OK when every graph converged, else NOT_CONVERGED (psi still computed). */
psi_status psi_multi_solve(psi_multi* mg, double eps, int32_t max_iter, psi_solve_info* info);

/* psi of every graph (psi = (.)/N_g with the graph's own N_g): sum(n_g) FP64 values, graph
 * by graph, local user order. */
psi_status psi_multi_scores(const psi_multi* mg, double* psi_out);

/* The k highest psi of every graph (psi descending, equal psi by ascending local id):
 * ids_out[G * k] local ids, vals_out[G * k] (may be NULL), graph-major.
 * 1 <= k <= min(1024, smallest n_g). */
psi_status psi_multi_topk(const psi_multi* mg, int32_t k, int32_t* ids_out, double* vals_out);

/* Statistics of the block-diagonal union (n = sum of n_g, ...). */
psi_status psi_multi_get_stats(const psi_multi* mg, psi_graph_stats* stats);
void psi_multi_destroy(psi_multi* mg);

/* ------------------------------------------------------------------------------------
 * Learned warm start.  The paper starts Algorithm 2 from s_0 = c (Eq. 14) and notes that
 * the fixed point does not depend on the start; here a small network predicts log s_i of
 * the converged iterate from per-user features and s_0 = exp(prediction) is used instead,
 * so only the number of steps can change.
 */

/* 8 features per user ([n][8] FP32, host or device, input user ids): log(1 + followers),
 * log(1 + leaders), log lambda, log mu, then the mean of each of these four over the user's
 * followers (0 for a user without followers).  Needs a built graph. */
psi_status psi_features(const psi_graph* g, float* feat_out);

typedef struct psi_mlp psi_mlp; /* 8 -> 64 -> 64 -> 1 network, GELU, 4801 parameters */

/* Parameters are kept in FP32 (Adam master copy) and BF16 (used by every forward/backward);
 * inputs are normalised with the model's (mean, std) per feature and rounded to BF16; all
 * sums are FP32.  Initial weights: uniform(+-sqrt(6/fan_in)) from a SplitMix64 seed. */
psi_status psi_mlp_create(uint64_t seed, void* stream, psi_mlp** out);
/* params: 4801 FP32 (W1[8][64], b1[64], W2[64][64], b2[64], W3[64], b3); norm: 18 FP32
 * (feature means[8], feature stds[8], target mean, target std); either may be NULL. */
psi_status psi_mlp_set_params(psi_mlp* m, const float* params, const float* norm);
psi_status psi_mlp_get_params(const psi_mlp* m, float* params, float* norm);
/* y[r] = predicted log s for x[r][0..8); device pointers. */
psi_status psi_mlp_forward(const psi_mlp* m, int64_t rows, const float* x, float* y);
/* Gradient of mean((yhat - t)^2) in normalised target units over the rows (device x, t);
 * kept for psi_mlp_adam_step, optionally copied to grad_out[4801]; loss_out (nullable). */
psi_status psi_mlp_grad(psi_mlp* m, int64_t rows, const float* x, const float* target, float* grad_out,
                        double* loss_out);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the last gradient. */
psi_status psi_mlp_adam_step(psi_mlp* m, float lr);
void psi_mlp_destroy(psi_mlp* m);

/* psi_solve from s_0 = exp(network prediction) (users without followers: s_0 = c). */
psi_status psi_solve_warm(psi_graph* g, const psi_mlp* m, double eps, int32_t max_iter, psi_solve_info* info);

/*
 * psi_topk_noalloc -- the ranking of psi_topk (psi descending, equal psi by ascending
 * user id) for a psi vector the caller holds in its own device memory, with no device
 * allocation: the paper has no counterpart; this entry point exists for callers that
 * cannot let a library call cudaMalloc, e.g. a serving process that reserves all of its
 * device memory up front in its own arena, or a host framework whose allocator owns every
 * device byte (a late cudaMalloc could fail, fragment that budget, or synchronise the
 * device mid-request).
 *   psi_in    device pointer: n FP64 values (for example written by psi_scores); user
 *             id = index.  Values are ranked in numeric order; -0.0 ranks as 0.0 and a
 *             NaN above +infinity (psi itself is never negative or NaN).
 *   n         1 <= n < 2^31 - 1
 *   k         1 <= k <= min(n, 4096); larger k is PSI_ERR_INVALID_ARG
 *   ids_out   device pointer, k int32 user ids; vals_out device pointer, k FP64 (or NULL):
 *             vals_out[i] = psi_in[ids_out[i]]
 *   stream    cudaStream_t to queue the work on (NULL = legacy default stream)
 * The work is queued and the call returns without waiting; results are complete when the
 * stream reaches that point.  Host pointers, and device memory of a GPU other than the
 * current one, are PSI_ERR_INVALID_ARG (managed memory is accepted).  A CUDA error left
 * pending by earlier work is reported as PSI_ERR_CUDA without being cleared, and nothing
 * is launched.
 * Working memory is one fixed 50,432-byte device array inside the library (held on every
 * device that loads it until the process exits).  All calls share it and it keeps the
 * last call's contents (each call clears what must start at zero), so calls whose work
 * overlaps on the GPU -- two streams or two host threads -- race and must be serialised by
 * the caller.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 */
psi_status psi_topk_noalloc(const double* psi_in, int64_t n, int32_t k, int32_t* ids_out, double* vals_out,
                            void* stream);

/* Without a caller allocator (psi_options.allocator NULL), device memory comes from a
 * stream-ordered pool private to the library on each device, which keeps freed memory for
 * the next call.  psi_trim_memory waits for the current device and returns that pool's
 * unused memory to the device. */
psi_status psi_trim_memory(void);

/* Number of CUDA kernels this library has launched in this process (instrumentation). */
int64_t psi_kernel_launches(void);

/* Library version (major*10000 + minor*100 + patch). */
int32_t psi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PSI_GB300_H */
