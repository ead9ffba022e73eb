/*
 * psigen.c -- seeded synthetic inputs for the psi-score solver and its oracle.
 *
 * This module holds NO arithmetic of the psi-score method: it only draws follower
 * graphs and activity rates.  Both the CUDA path's tests/benchmark and the CPU oracle
 * read the arrays it writes, so they always see identical inputs.
 *
 * Random numbers come from one counter-based generator: the i-th output of a
 * SplitMix64 sequence (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014; output function as in Vigna's public-domain
 * splitmix64.c).  Output i of the sequence with initial state S is
 *     mix64(S + (i+1) * 0x9E3779B97F4A7C15).
 * Every draw is addressed by (seed, stream, counter), so results do not depend on the
 * number of OpenMP threads.
 *
 * Edge convention (paper Sec. II): edge k means "follower[k] follows leader[k]".
 * Self-loops are never emitted (the paper's model has none, Eq. 5): a draw that would
 * give one is redrawn with the next attempt counter.  Duplicate edges are kept; the
 * consumers merge them (the leader set of a user is a set).
 *
 * Compile with -ffp-contract=off so that host results are the same on x86-64 and
 * aarch64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN 0x9E3779B97F4A7C15ULL

/* stream ids: one independent sequence per purpose */
enum {
  S_POISSON = 1, S_LEADERS = 2, S_RMAT = 3, S_PERM = 4, S_CL_DRAW = 5,
  S_CL_PERM_OUT = 6, S_CL_PERM_IN = 7
};

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* initial state of the sequence (seed, stream) */
static inline uint64_t stream_state(uint64_t seed, uint64_t stream) {
  return mix64(mix64(seed + GOLDEN) ^ (stream * 0xD1B54A32D192ED03ULL));
}

static inline uint64_t draw(uint64_t state, uint64_t i) { return mix64(state + GOLDEN * (i + 1)); }

/* uniform in [0,1) with 53 random bits */
static inline double u01(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }
/* uniform in (0,1) */
static inline double uopen(uint64_t x) { return ((double)(x >> 11) + 0.5) * 0x1.0p-53; }
/* uniform integer in [0, k) (k < 2^32), by the high half of a 64x32 product */
static inline uint32_t below(uint64_t x, uint32_t k) { return (uint32_t)(((x >> 32) * (uint64_t)k) >> 32); }

/* ------------------------------------------------------------------ raw stream */

uint64_t psigen_splitmix64_at(uint64_t state, uint64_t i) { return draw(state, i); }

uint64_t psigen_stream_state(uint64_t seed, uint64_t stream) { return stream_state(seed, stream); }

void psigen_uniform(uint64_t seed, uint64_t stream, int64_t n, double* out) {
  const uint64_t st = stream_state(seed, stream);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = u01(draw(st, (uint64_t)i));
}

/* ------------------------------------------------------------------ rates */

/* lambda or mu ~ Uniform(lo, hi), i.i.d. */
void psigen_rates_uniform(int64_t n, double lo, double hi, uint64_t seed, uint64_t stream,
                          double* out) {
  const uint64_t st = stream_state(seed, stream);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = lo + (hi - lo) * u01(draw(st, (uint64_t)i));
}

/* exp(m + s Z), Z ~ N(0,1) by Box-Muller, clipped to [lo, hi] */
void psigen_rates_lognormal(int64_t n, double m, double s, double lo, double hi, uint64_t seed,
                            uint64_t stream, double* out) {
  const uint64_t st = stream_state(seed, stream);
  const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double a = uopen(draw(st, 2 * (uint64_t)i));
    double b = u01(draw(st, 2 * (uint64_t)i + 1));
    double z = sqrt(-2.0 * log(a)) * cos(two_pi * b);
    double x = exp(m + s * z);
    out[i] = x < lo ? lo : (x > hi ? hi : x);
  }
}

/* ------------------------------------------------------------------ permutation */

/* Fisher-Yates shuffle of the identity (Durstenfeld form), counter i drives step i */
static void random_permutation(int64_t n, uint64_t seed, uint64_t stream, int32_t* perm) {
  const uint64_t st = stream_state(seed, stream);
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  for (int64_t i = n - 1; i > 0; --i) {
    uint32_t j = below(draw(st, (uint64_t)i), (uint32_t)(i + 1));
    int32_t t = perm[i];
    perm[i] = perm[j];
    perm[j] = t;
  }
}

void psigen_permutation(int64_t n, uint64_t seed, uint64_t stream, int32_t* perm) {
  random_permutation(n, seed, stream, perm);
}

/* ------------------------------------------------------------------ Poisson-uniform */

/*
 * Each user i follows k_i ~ Poisson(mean) leaders (capped at n-1), drawn uniformly
 * without replacement among the other n-1 users.  Pass follower == NULL to get the
 * edge count only.  Edges are written user by user, leaders in draw order.
 */
int64_t psigen_poisson_uniform(int64_t n, double mean, uint64_t seed, int32_t* follower,
                               int32_t* leader) {
  if (n < 2) return 0;
  const uint64_t sk = stream_state(seed, S_POISSON);
  const uint64_t sl = stream_state(seed, S_LEADERS);
  const double p0 = exp(-mean);
  int64_t e = 0;
  int32_t* chosen = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!chosen) return -1;
  for (int64_t i = 0; i < n; ++i) {
    /* inversion: smallest k with F(k) >= u */
    double u = u01(draw(sk, (uint64_t)i)), p = p0, F = p0;
    int64_t k = 0;
    while (u > F && k < n - 1) {
      ++k;
      p *= mean / (double)k;
      F += p;
    }
    int64_t got = 0;
    for (uint64_t r = 0; got < k; ++r) {
      uint32_t c = below(draw(sl, ((uint64_t)i << 24) + r), (uint32_t)(n - 1));
      if ((int64_t)c >= i) ++c; /* skip the user itself */
      int dup = 0;
      for (int64_t q = 0; q < got; ++q)
        if (chosen[q] == (int32_t)c) { dup = 1; break; }
      if (dup) continue;
      chosen[got++] = (int32_t)c;
    }
    if (follower)
      for (int64_t q = 0; q < got; ++q) {
        follower[e + q] = (int32_t)i;
        leader[e + q] = chosen[q];
      }
    e += got;
  }
  free(chosen);
  return e;
}

/* ------------------------------------------------------------------ R-MAT */

/*
 * R-MAT (Chakrabarti, Zhan, Faloutsos 2004): m = edge_factor * 2^scale draws; each picks
 * one quadrant per level with probabilities (a, b, c, 1-a-b-c), most significant bit
 * first.  Quadrant b sets the destination bit, c the source bit.  Source = follower,
 * destination = leader.  A self-loop is redrawn (next attempt counter).  With relabel,
 * ids are mapped through one seeded random permutation, so R-MAT id locality is gone.
 */
int64_t psigen_rmat(int32_t scale, int64_t edge_factor, double a, double b, double c,
                    uint64_t seed, int32_t relabel, int32_t* follower, int32_t* leader) {
  if (scale < 1 || scale > 30) return -1;
  const int64_t n = (int64_t)1 << scale;
  const int64_t m = edge_factor * n;
  const uint64_t st = stream_state(seed, S_RMAT);
  const uint64_t ta = (uint64_t)(a * 4294967296.0);
  const uint64_t tab = (uint64_t)((a + b) * 4294967296.0);
  const uint64_t tabc = (uint64_t)((a + b + c) * 4294967296.0);
  int32_t* perm = NULL;
  if (relabel) {
    perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!perm) return -1;
    random_permutation(n, seed, S_PERM, perm);
  }
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    uint32_t src = 0, dst = 0;
    for (uint64_t att = 0; att < 64; ++att) {
      src = 0;
      dst = 0;
      uint64_t base = (((uint64_t)e << 6) + att) << 4;
      uint64_t x = 0;
      for (int lv = 0; lv < scale; ++lv) {
        uint64_t u;
        if ((lv & 1) == 0) {
          x = draw(st, base + (uint64_t)(lv >> 1));
          u = x & 0xFFFFFFFFULL;
        } else {
          u = x >> 32;
        }
        uint32_t sb, db;
        if (u < ta) { sb = 0; db = 0; }
        else if (u < tab) { sb = 0; db = 1; }
        else if (u < tabc) { sb = 1; db = 0; }
        else { sb = 1; db = 1; }
        src = (src << 1) | sb;
        dst = (dst << 1) | db;
      }
      if (src != dst) break;
    }
    follower[e] = relabel ? perm[src] : (int32_t)src;
    leader[e] = relabel ? perm[dst] : (int32_t)dst;
  }
  free(perm);
  return m;
}

/* ------------------------------------------------------------------ Chung-Lu */

static int64_t upper_index(const double* cdf, int64_t n, double x) {
  /* smallest i in [0,n) with cdf[i+1] > x; cdf[0] = 0, cdf[n] = total */
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (cdf[mid + 1] > x) hi = mid; else lo = mid + 1;
  }
  return lo;
}

/*
 * Chung-Lu by ball dropping: expected-degree weights w_r = (r+1)^(-1/(gamma-1)) for
 * rank r, the same law for out- and in-degree; ranks map to user ids through two
 * independent random permutations.  Each of `draws` edges picks its follower with
 * probability proportional to the out-weight and its leader proportional to the
 * in-weight; a self-loop is redrawn.
 */
int64_t psigen_chung_lu(int64_t n, double gamma, int64_t draws, uint64_t seed, int32_t* follower,
                        int32_t* leader) {
  if (n < 2 || gamma <= 1.0) return -1;
  double* cdf = (double*)malloc(sizeof(double) * (size_t)(n + 1));
  int32_t* pout = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* pin = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!cdf || !pout || !pin) { free(cdf); free(pout); free(pin); return -1; }
  const double ex = -1.0 / (gamma - 1.0);
  cdf[0] = 0.0;
  for (int64_t r = 0; r < n; ++r) cdf[r + 1] = cdf[r] + pow((double)(r + 1), ex);
  const double total = cdf[n];
  random_permutation(n, seed, S_CL_PERM_OUT, pout);
  random_permutation(n, seed, S_CL_PERM_IN, pin);
  const uint64_t st = stream_state(seed, S_CL_DRAW);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < draws; ++e) {
    int32_t f = 0, l = 0;
    for (uint64_t att = 0; att < 64; ++att) {
      uint64_t base = (((uint64_t)e << 6) + att) << 1;
      f = pout[upper_index(cdf, n, u01(draw(st, base)) * total)];
      l = pin[upper_index(cdf, n, u01(draw(st, base + 1)) * total)];
      if (f != l) break;
    }
    follower[e] = f;
    leader[e] = l;
  }
  free(cdf);
  free(pout);
  free(pin);
  return draws;
}

int32_t psigen_num_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}
