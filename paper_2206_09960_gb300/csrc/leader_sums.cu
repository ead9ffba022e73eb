// leader_sums.cu -- exact sigma and beta sums of the single-graph build (leader_sums.cuh).
#include "leader_sums.cuh"

namespace psi {

namespace {

constexpr int kGsThreads = 256;
constexpr int kGsItems = 8;               // consecutive edge keys per lane
constexpr int kGsTile = 32 * kGsItems;    // keys per warp tile
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

// the run of group g closed with sums x: groups that may continue in another tile (the
// tile's first and last groups) are added atomically, every other group lies in this tile
// alone and is stored
__device__ __forceinline__ void emit(uint32_t g, const Part& x, bool shared_group, unsigned long long* acc_s,
                                     unsigned long long* acc_b, uint32_t* acc_c) {
  if (g == kNoGroup) return;
  if (shared_group) {
    atomic_add128(acc_s + 2 * (size_t)g, x.s.lo, x.s.hi);
    atomic_add128(acc_b + 2 * (size_t)g, x.b.lo, x.b.hi);
    atomicAdd(acc_c + g, x.c);
  } else {
    acc_s[2 * (size_t)g] = x.s.lo;
    acc_s[2 * (size_t)g + 1] = x.s.hi;
    acc_b[2 * (size_t)g] = x.b.lo;
    acc_b[2 * (size_t)g + 1] = x.b.hi;
    acc_c[g] = x.c;
  }
}

// Per-follower sums over keys sorted by follower (duplicates included).  A warp takes tiles
// of 256 consecutive keys, 8 per lane; a lane sums its runs of equal follower in order (a
// run strictly inside the lane is a whole group: stored), and the runs that cross lanes are
// joined by a segmented scan of the lanes' last runs.
__global__ void __launch_bounds__(kGsThreads) k_group_sums(const unsigned long long* __restrict__ keys, int64_t m,
                                                          int bf, uint32_t nu, const FixedRow* __restrict__ rows,
                                                          unsigned long long* __restrict__ acc_s,
                                                          unsigned long long* __restrict__ acc_b,
                                                          uint32_t* __restrict__ acc_c) {
  const int lane = threadIdx.x & 31;
  const unsigned long long fmask = (1ull << bf) - 1ull;
  const int64_t tiles = ceil_div(m, kGsTile);
  const int64_t nwarps = (int64_t)gridDim.x * (kGsThreads / 32);
  for (int64_t t = (int64_t)blockIdx.x * (kGsThreads / 32) + (threadIdx.x >> 5); t < tiles; t += nwarps) {
    const int64_t base = t * kGsTile + (int64_t)lane * kGsItems;
    uint32_t g[kGsItems], r[kGsItems];
#pragma unroll
    for (int j = 0; j < kGsItems; ++j) {
      const int64_t e = base + j;
      const unsigned long long k = e < m ? keys[e] : ~0ull;
      const uint32_t gg = (uint32_t)(k & fmask);
      g[j] = e < m && gg < nu ? gg : kNoGroup;  // sorted by g: the no-group keys come last
      r[j] = (uint32_t)(k >> bf);
    }
    FixedRow v[kGsItems];
#pragma unroll
    for (int j = 0; j < kGsItems; ++j) v[j] = g[j] != kNoGroup ? ld_fixed_row(rows + r[j]) : FixedRow{0, 0, 0, 0};
    // runs inside the lane
    Part cur{{v[0].s_lo, v[0].s_hi}, {v[0].b_lo, v[0].b_hi}, g[0] != kNoGroup ? 1u : 0u};
    Part head = cur;
    uint32_t cur_g = g[0];
    const uint32_t head_g = g[0];
    bool single = true;
#pragma unroll
    for (int j = 1; j < kGsItems; ++j) {
      if (g[j] != cur_g) {
        if (single) head = cur;
        else emit(cur_g, cur, false, acc_s, acc_b, acc_c);  // both ends inside the lane
        single = false;
        cur_g = g[j];
        cur = Part{{v[j].s_lo, v[j].s_hi}, {v[j].b_lo, v[j].b_hi}, g[j] != kNoGroup ? 1u : 0u};
      } else {
        add128(cur.s, v[j].s_lo, v[j].s_hi);
        add128(cur.b, v[j].b_lo, v[j].b_hi);
        cur.c += 1u;
      }
    }
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
  }
}

__global__ void k_group_finish(const unsigned long long* __restrict__ acc_s, const unsigned long long* __restrict__ acc_b,
                               const uint32_t* __restrict__ acc_c, int32_t nu, int32_t nX, int32_t nR, int ebase,
                               double* __restrict__ sigma, double* __restrict__ beta, int32_t* __restrict__ n_leaders) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nu; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t user = g < nX ? g : g + nR;
    sigma[user] = fixed_to_double(U128{acc_s[2 * g], acc_s[2 * g + 1]}, ebase);
    beta[user] = fixed_to_double(U128{acc_b[2 * g], acc_b[2 * g + 1]}, ebase);
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
  x.s.reset(al, 2 * (size_t)nu);
  x.b.reset(al, 2 * (size_t)nu);
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

void exact_sums_groups(ExactLeaderSums& x, const uint64_t* keys, int64_t m, int bf, int32_t nu, cudaStream_t s) {
  if (m <= 0 || nu <= 0) return;
  const int64_t warps = ceil_div(m, kGsTile);
  const int64_t blocks = std::min<int64_t>(ceil_div(warps, kGsThreads / 32), num_sms() * 8);
  k_group_sums<<<(unsigned)blocks, kGsThreads, 0, s>>>(reinterpret_cast<const unsigned long long*>(keys), m, bf,
                                                      (uint32_t)nu, x.rows.get(), x.s.get(), x.b.get(), x.cnt.get());
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
