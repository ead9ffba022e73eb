// leader_sums.cuh -- sigma_j = sum_{l in L(j)} (lambda_l + mu_l) and beta_j = sum_{l in L(j)}
// lambda_l (Sec. II: the denominators of a_ji and b_ji) as exact sums, for the builds of single
// graphs and of multi-graph objects.
//
// Every nonzero rate is m * 2^(e - 1075) with a 53-bit integer m and biased exponent e.  When
// all rates of the graph have exponents in [ebase, ebase + kFixedSpan], a rate divided by
// 2^(ebase - 1075) is the integer m << (e - ebase) < 2^94, and the sum over up to 2^31
// leaders fits 128 bits.  Integer addition is exact and associative, so the sums can be
// formed in any order (atomics included) and are rounded to FP64 once, at the end: the
// result does not depend on the order of the edges, the schedule or the grouping.
//
// The sums are formed from the edge keys (leader row << bf | follower's gathered index)
// while they are grouped by follower, half-way through the edge sort (all edges, duplicates
// included), and the duplicates found after the sort are subtracted (again exact).
#pragma once

#include "common.cuh"

namespace psi {

constexpr int kFixedSpan = 40;  // largest exponent range of the rates the exact sums accept

// lambda_l + mu_l (s) and lambda_l (b) of one leader row, each as a 128-bit integer
struct __align__(32) FixedRow {
  unsigned long long s_lo, s_hi, b_lo, b_hi;
};

// Group sums are kept as four counters of 32-bit limbs (value = sum_k c_k 2^(32k)), so every
// update is a plain atomic add without a returned value.  The graph has fewer than 2^31 edges,
// so a counter (at most one limb below 2^32 added or subtracted per edge) stays within +-2^63
// and is read back as a signed integer (leader_sums.cu).
__device__ __forceinline__ void red_add_u64(unsigned long long* p, unsigned long long v) {
  if (v) atomicAdd(p, v);
}
__device__ __forceinline__ void red_limbs(unsigned long long* c, unsigned long long lo, unsigned long long hi) {
  red_add_u64(c, lo & 0xFFFFFFFFull);
  red_add_u64(c + 1, lo >> 32);
  red_add_u64(c + 2, hi & 0xFFFFFFFFull);
  red_add_u64(c + 3, hi >> 32);
}
// minus a 128-bit value: each limb counter takes 2^64 - limb
__device__ __forceinline__ void red_sub_limbs(unsigned long long* c, unsigned long long lo, unsigned long long hi) {
  red_add_u64(c, 0ull - (lo & 0xFFFFFFFFull));
  red_add_u64(c + 1, 0ull - (lo >> 32));
  red_add_u64(c + 2, 0ull - (hi & 0xFFFFFFFFull));
  red_add_u64(c + 3, 0ull - (hi >> 32));
}

// take t copies of one leader row's (s, b) and t counts back out of follower group g (a row
// value is below 2^94 and t below 2^32, so the products fit 128 bits)
__device__ __forceinline__ void fixed_sub_rows(const FixedRow& v, uint32_t t, unsigned long long* acc_s,
                                               unsigned long long* acc_b, uint32_t* acc_c, uint32_t g) {
  red_sub_limbs(acc_s + 4 * (size_t)g, v.s_lo * t, v.s_hi * t + __umul64hi(v.s_lo, t));
  red_sub_limbs(acc_b + 4 * (size_t)g, v.b_lo * t, v.b_hi * t + __umul64hi(v.b_lo, t));
  atomicSub(acc_c + g, t);
}

__device__ __forceinline__ FixedRow ld_fixed_row(const FixedRow* p) {
  FixedRow v;
  asm volatile("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];"
               : "=l"(v.s_lo), "=l"(v.s_hi), "=l"(v.b_lo), "=l"(v.b_hi)
               : "l"(p));
  return v;
}

// The exact-sum state of one build.
struct ExactLeaderSums {
  DBuf<FixedRow> rows;           // [n_rows]
  DBuf<unsigned long long> s, b;  // [4 * nu]: limb counters per follower group
  DBuf<uint32_t> cnt;             // [nu]: distinct leaders
  int ebase = 0;
};

// Whether the rates' biased exponents (over the nonzero rates; 0 when one is subnormal)
// allow exact sums.
bool exact_sums_apply(uint32_t emin_biased, uint32_t emax_biased);

// Fixed-point rows of the leaders (internal order), zeroed group sums.
void exact_sums_prepare(ExactLeaderSums& x, const double* lam_i, const double* mu_i, int32_t n_rows, int32_t nu,
                        uint32_t emin_biased, Allocator& al, cudaStream_t s);
// Group sums over all m edge keys, which are sorted by their low bf bits (the follower); also
// the per-tile counts of the next sort digit ((key >> bf) & next_mask) into next_counts, in
// the layout radix_sort_bits takes as first_counts.
void exact_sums_groups(ExactLeaderSums& x, const uint64_t* keys, int64_t m, int bf, int32_t nu, uint32_t next_mask,
                       uint32_t* next_counts, cudaStream_t s);
// sigma, beta (FP64, rounded once) and the number of distinct leaders of every gathered user,
// stored at its internal id (gathered index g < nX: g; otherwise g + nR).
void exact_sums_finish(ExactLeaderSums& x, int32_t nu, int32_t nX, int32_t nR, double* sigma, double* beta,
                       int32_t* n_leaders, cudaStream_t s);

}  // namespace psi
