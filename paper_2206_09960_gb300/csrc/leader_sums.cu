// leader_sums.cu -- exact sigma and beta sums of the graph build (leader_sums.cuh).
#include "leader_sums.cuh"
#include "primitives.cuh"

namespace psi {

namespace {

constexpr int kGsThreads = 256;
constexpr int kGsWarpKeys = kRadixTileKeys / (kGsThreads / 32);  // consecutive keys per warp
constexpr int kGsItems = kGsWarpKeys / 32;                        // consecutive keys per lane
constexpr int kGsBatch = 6;                                        // row gathers in flight per lane
static_assert(kGsWarpKeys * (kGsThreads / 32) == kRadixTileKeys && kGsItems * 32 == kGsWarpKeys, "whole tiles");
static_assert(kGsItems % 4 == 0 && kGsItems % kGsBatch == 0 && kGsThreads == 256, "loads, batches, one count per thread");
constexpr uint32_t kNoGroup = 0xFFFFFFFFu;  // sentinel keys and keys past the end

struct U128 {
  unsigned long long lo, hi;
};

__device__ __forceinline__ void add128(U128& a, unsigned long long lo, unsigned long long hi) {
  a.lo += lo;
  a.hi += hi + (a.lo < lo ? 1ull : 0ull);
}

// a rate as the integer rate / 2^(ebase - 1075): zero, or its 53-bit significand shifted
// left by its exponent's distance from ebase (0 .. kFixedSpan)
__device__ __forceinline__ U128 to_fixed(double x, int ebase) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
  if (b == 0) return U128{0ull, 0ull};
  const int sh = (int)(b >> 52) - ebase;
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  return U128{m << sh, sh ? m >> (64 - sh) : 0ull};
}

// a (units of 2^(ebase - 1075)) rounded to the nearest FP64 value, ties to even.  A nonzero
// sum is at least one rate, m >= 2^52 units, so its leading bit p is >= 52 and the result's
// biased exponent is ebase + p - 52 (normal: ebase >= 1, and the caller keeps it below 2047).
__device__ __forceinline__ double fixed_to_double(U128 a, int ebase) {
  if ((a.lo | a.hi) == 0) return 0.0;
  const int p = a.hi ? 127 - __clzll((long long)a.hi) : 63 - __clzll((long long)a.lo);
  const int s = p - 52;  // bits below the 53 kept
  unsigned long long mant;
  int e = ebase + s;
  if (s <= 0) {
    mant = a.lo << (-s);
  } else {
    mant = s >= 64 ? a.hi >> (s - 64) : (a.lo >> s) | (a.hi << (64 - s));
    const int k = s - 1;  // the rounding bit
    const bool half = k >= 64 ? (a.hi >> (k - 64)) & 1ull : (a.lo >> k) & 1ull;
    bool sticky;  // any bit below the rounding bit
    if (k == 0) sticky = false;
    else if (k < 64) sticky = (a.lo & ((1ull << k) - 1ull)) != 0;
    else if (k == 64) sticky = a.lo != 0;
    else sticky = a.lo != 0 || (a.hi & ((1ull << (k - 64)) - 1ull)) != 0;
    if (half && (sticky || (mant & 1ull))) {
      ++mant;
      if (mant >> 53) {  // rounded up to the next power of two
        mant >>= 1;
        ++e;
      }
    }
  }
  const unsigned long long bits = ((unsigned long long)e << 52) | (mant & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

__global__ void k_fixed_rows(const double* __restrict__ lam_i, const double* __restrict__ mu_i, int32_t n_rows,
                             int ebase, FixedRow* __restrict__ rows) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_rows; r += (int64_t)gridDim.x * blockDim.x) {
    const U128 l = to_fixed(lam_i[r], ebase), m = to_fixed(mu_i[r], ebase);
    U128 s = l;
    add128(s, m.lo, m.hi);
    rows[r] = FixedRow{s.lo, s.hi, l.lo, l.hi};
  }
}

struct Part {  // one run's partial sums
  U128 s, b;
  uint32_t c;
};

__device__ __forceinline__ void part_add(Part& a, const Part& x) {
  add128(a.s, x.s.lo, x.s.hi);
  add128(a.b, x.b.lo, x.b.hi);
  a.c += x.c;
}

__device__ __forceinline__ Part shfl_up_part(const Part& x, int o) {
  Part y;
  y.s.lo = __shfl_up_sync(0xffffffffu, x.s.lo, o);
  y.s.hi = __shfl_up_sync(0xffffffffu, x.s.hi, o);
  y.b.lo = __shfl_up_sync(0xffffffffu, x.b.lo, o);
  y.b.hi = __shfl_up_sync(0xffffffffu, x.b.hi, o);
  y.c = __shfl_up_sync(0xffffffffu, x.c, o);
  return y;
}

__device__ __forceinline__ void st_limbs(unsigned long long* c, const U128& x) {
  asm volatile("st.global.v4.u64 [%0], {%1,%2,%3,%4};" ::"l"(c), "l"(x.lo & 0xFFFFFFFFull), "l"(x.lo >> 32),
               "l"(x.hi & 0xFFFFFFFFull), "l"(x.hi >> 32)
               : "memory");
}

// The limb counters c_0..c_3 of a group as one 128-bit value.  A counter holds limbs of run
// sums minus limbs of repeated rows, so on its own it can end below zero (carries between limbs
// differ); with fewer than 2^31 edges per group it stays within +-2^63, so each counter is
// read as a signed integer and sign-extended: the sum modulo 2^128 is the exact sum.
__device__ __forceinline__ U128 from_limbs(const unsigned long long* c) {
  U128 a{0ull, 0ull};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const unsigned long long lo = c[k], hi = (long long)c[k] < 0 ? ~0ull : 0ull;  // c_k as 128 bits
    if (k == 0) add128(a, lo, hi);
    else if (k == 1) add128(a, lo << 32, (hi << 32) | (lo >> 32));
    else if (k == 2) add128(a, 0ull, lo);
    else add128(a, 0ull, lo << 32);
  }
  return a;
}

// the run of group g closed with sums x: groups that may continue in another tile (the
// tile's first and last groups) are added atomically, every other group lies in this tile
// alone and is stored
__device__ __forceinline__ void emit(uint32_t g, const Part& x, bool shared_group, unsigned long long* acc_s,
                                     unsigned long long* acc_b, uint32_t* acc_c) {
  if (g == kNoGroup) return;
  if (shared_group) {
    red_limbs(acc_s + 4 * (size_t)g, x.s.lo, x.s.hi);
    red_limbs(acc_b + 4 * (size_t)g, x.b.lo, x.b.hi);
    atomicAdd(acc_c + g, x.c);
  } else {
    st_limbs(acc_s + 4 * (size_t)g, x.s);
    st_limbs(acc_b + 4 * (size_t)g, x.b);
    acc_c[g] = x.c;
  }
}

// Per-follower sums over keys sorted by follower (duplicates included).  One block per tile
// of kRadixTileKeys keys; a warp takes 384 consecutive keys, 12 per lane.  A lane sums its
// runs of equal follower in order (a run strictly inside the lane is a whole group: stored),
// and the runs that cross lanes are joined by a segmented scan of the lanes' last runs.  The
// block also counts the tile's values of the next sort pass's digit ((key >> bf) & mask) for
// the second half of the edge sort.
__global__ void __launch_bounds__(kGsThreads) k_group_sums(const unsigned long long* __restrict__ keys, int64_t m,
                                                          int bf, uint32_t nu, const FixedRow* __restrict__ rows,
                                                          unsigned long long* __restrict__ acc_s,
                                                          unsigned long long* __restrict__ acc_b,
                                                          uint32_t* __restrict__ acc_c, uint32_t mask,
                                                          uint32_t* __restrict__ counts) {
  __shared__ uint32_t hist[kGsThreads / 32][256];
  for (int i = threadIdx.x; i < (kGsThreads / 32) * 256; i += kGsThreads) (&hist[0][0])[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long fmask = (1ull << bf) - 1ull;
  const uint64_t pol = policy_evict_first();  // the keys are read once
  const int64_t base = (int64_t)blockIdx.x * kRadixTileKeys + (int64_t)warp * kGsWarpKeys + (int64_t)lane * kGsItems;
  unsigned long long k[kGsItems];
  if (base + kGsItems <= m) {  // the lane's 96 bytes in three 32-byte loads
#pragma unroll
    for (int h = 0; h < kGsItems / 4; ++h) {
      int w[8];
      ld_stream_v8(reinterpret_cast<const int*>(keys + base + 4 * h), pol, w);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        k[4 * h + q] = (unsigned long long)(uint32_t)w[2 * q] | ((unsigned long long)(uint32_t)w[2 * q + 1] << 32);
    }
  } else {
#pragma unroll
    for (int j = 0; j < kGsItems; ++j) k[j] = base + j < m ? keys[base + j] : ~0ull;
  }
#pragma unroll
  for (int j = 0; j < kGsItems; ++j)
    if (base + j < m) atomicAdd(&hist[warp][(uint32_t)(k[j] >> bf) & mask], 1u);
  auto group = [&](int j) -> uint32_t {  // sorted by group: the no-group keys come last
    const uint32_t gg = (uint32_t)(k[j] & fmask);
    return base + j < m && gg < nu ? gg : kNoGroup;
  };
  // runs inside the lane, the rows gathered kGsBatch at a time
  Part cur{}, head{};
  uint32_t cur_g = group(0);
  const uint32_t head_g = cur_g;
  bool single = true;
#pragma unroll
  for (int j0 = 0; j0 < kGsItems; j0 += kGsBatch) {
    FixedRow v[kGsBatch];
#pragma unroll
    for (int q = 0; q < kGsBatch; ++q)
      v[q] = group(j0 + q) != kNoGroup ? ld_fixed_row(rows + (k[j0 + q] >> bf)) : FixedRow{0, 0, 0, 0};
#pragma unroll
    for (int q = 0; q < kGsBatch; ++q) {
      const int j = j0 + q;
      const uint32_t gj = group(j);
      const uint32_t one = gj != kNoGroup ? 1u : 0u;
      if (j > 0 && gj != cur_g) {
        if (single) head = cur;
        else emit(cur_g, cur, false, acc_s, acc_b, acc_c);  // both ends inside the lane
        single = false;
        cur_g = gj;
        cur = Part{{v[q].s_lo, v[q].s_hi}, {v[q].b_lo, v[q].b_hi}, one};
      } else if (j == 0) {
        cur = Part{{v[q].s_lo, v[q].s_hi}, {v[q].b_lo, v[q].b_hi}, one};
      } else {
        add128(cur.s, v[q].s_lo, v[q].s_hi);
        add128(cur.b, v[q].b_lo, v[q].b_hi);
        cur.c += one;
      }
    }
  }
  if (single) head = cur;
  const uint32_t last_g = cur_g;
  // across lanes
  const uint32_t prev_last = __shfl_up_sync(0xffffffffu, last_g, 1);
  const uint32_t next_first = __shfl_down_sync(0xffffffffu, head_g, 1);
  const bool cont = lane > 0 && head_g == prev_last;          // my first run goes on from the lane before
  const bool tail_open = lane < 31 && next_first == last_g;    // my last run goes on in the lane after
  const uint32_t tile_first = __shfl_sync(0xffffffffu, head_g, 0);
  const uint32_t tile_last = __shfl_sync(0xffffffffu, last_g, 31);
  // segmented inclusive scan of the last runs; a lane that is one run continuing the lane
  // before extends its segment
  const uint32_t starts = __ballot_sync(0xffffffffu, !(single && cont));
  const int seg0 = 31 - __clz((int)(starts & (0xFFFFFFFFu >> (31 - lane))));
  Part sc = cur;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const Part y = shfl_up_part(sc, o);
    if (lane - o >= seg0) part_add(sc, y);
  }
  const Part in = shfl_up_part(sc, 1);  // the chain ending in the lane before
  if (!single) {  // my first run ends inside the lane
    Part h = head;
    if (cont) part_add(h, in);
    emit(head_g, h, head_g == tile_first || head_g == tile_last, acc_s, acc_b, acc_c);
  }
  if (!tail_open) emit(last_g, sc, last_g == tile_first || last_g == tile_last, acc_s, acc_b, acc_c);
  __syncthreads();
  const int64_t tiles = ceil_div(m, kRadixTileKeys);
  uint32_t t = 0;
#pragma unroll
  for (int w = 0; w < kGsThreads / 32; ++w) t += hist[w][threadIdx.x];
  counts[(int64_t)threadIdx.x * tiles + blockIdx.x] = t;
}

__global__ void k_group_finish(const unsigned long long* __restrict__ acc_s, const unsigned long long* __restrict__ acc_b,
                               const uint32_t* __restrict__ acc_c, int32_t nu, int32_t nX, int32_t nR, int ebase,
                               double* __restrict__ sigma, double* __restrict__ beta, int32_t* __restrict__ n_leaders) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nu; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t user = g < nX ? g : g + nR;
    sigma[user] = fixed_to_double(from_limbs(acc_s + 4 * g), ebase);
    beta[user] = fixed_to_double(from_limbs(acc_b + 4 * g), ebase);
    n_leaders[user] = (int32_t)acc_c[g];
  }
}

int flat_grid(int64_t n) {
  const int64_t g = ceil_div(n > 0 ? n : 1, 256), cap = num_sms() * 16;
  return (int)(g < cap ? g : cap);
}

}  // namespace

bool exact_sums_apply(uint32_t emin_biased, uint32_t emax_biased) {
  // no subnormal rate, the range within kFixedSpan, and sums of up to 2^31 rows (< 2^(e+33))
  // below the FP64 overflow
  return emin_biased >= 1 && emin_biased <= emax_biased && emax_biased - emin_biased <= (uint32_t)kFixedSpan &&
         emax_biased <= 2000;
}

void exact_sums_prepare(ExactLeaderSums& x, const double* lam_i, const double* mu_i, int32_t n_rows, int32_t nu,
                        uint32_t emin_biased, Allocator& al, cudaStream_t s) {
  x.ebase = (int)emin_biased;
  x.rows.reset(al, (size_t)(n_rows > 0 ? n_rows : 1));
  x.s.reset(al, 4 * (size_t)nu);
  x.b.reset(al, 4 * (size_t)nu);
  x.cnt.reset(al, (size_t)nu);
  if (n_rows > 0) {
    k_fixed_rows<<<flat_grid(n_rows), 256, 0, s>>>(lam_i, mu_i, n_rows, x.ebase, x.rows.get());
    PSI_LAUNCHED();
  }
  // groups touched by atomics start from zero; every other group is stored whole
  PSI_CUDA(cudaMemsetAsync(x.s.get(), 0, x.s.bytes(), s));
  PSI_CUDA(cudaMemsetAsync(x.b.get(), 0, x.b.bytes(), s));
  PSI_CUDA(cudaMemsetAsync(x.cnt.get(), 0, x.cnt.bytes(), s));
}

void exact_sums_groups(ExactLeaderSums& x, const uint64_t* keys, int64_t m, int bf, int32_t nu, uint32_t next_mask,
                       uint32_t* next_counts, cudaStream_t s) {
  if (m <= 0 || nu <= 0) return;
  k_group_sums<<<(unsigned)ceil_div(m, kRadixTileKeys), kGsThreads, 0, s>>>(
      reinterpret_cast<const unsigned long long*>(keys), m, bf, (uint32_t)nu, x.rows.get(), x.s.get(), x.b.get(),
      x.cnt.get(), next_mask, next_counts);
  PSI_LAUNCHED();
}

void exact_sums_finish(ExactLeaderSums& x, int32_t nu, int32_t nX, int32_t nR, double* sigma, double* beta,
                       int32_t* n_leaders, cudaStream_t s) {
  if (nu <= 0) return;
  k_group_finish<<<flat_grid(nu), 256, 0, s>>>(x.s.get(), x.b.get(), x.cnt.get(), nu, nX, nR, x.ebase, sigma, beta,
                                               n_leaders);
  PSI_LAUNCHED();
}

}  // namespace psi
