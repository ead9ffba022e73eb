// build.cu -- the operator of Sec. II built on the device from an edge list.
//
//  1. validate ids, self-loops and rates; mark users with followers / with leaders (exact,
//     two bitmaps) and count degrees (on a fixed 1-in-2^k subset of the edges for large
//     graphs);
//  2. renumber users by class (X: followers and leaders, R: followers only, U: leaders
//     only, Z: isolated) and, within a class, by decreasing degree, so rows form one range
//     [0, nX+nR) and the gathered users one compact L2-friendly range;
//  3. sort the renumbered (leader, follower) pairs (stable LSD radix), merge duplicates
//     (L(j) is a set) and cut the transposed CSR (row i = followers of leader i) in one
//     stream compaction;
//  4. regroup the unique edges by follower (stable radix on the follower id) and form,
//     for every follower j, sigma_j = sum_{l in L(j)} (lambda_l + mu_l) and
//     beta_j = sum_{l in L(j)} lambda_l (the denominators of a_ji, b_ji; float-pair sums,
//     FP64 in the FP64 mode) in one load-balanced product over that follower-grouped CSR;
//  5. per-user constants c, d, 1/sigma in FP64 and FP32; ||B||_inf = max_j beta_j/sigma_j;
//  6. the tile schedule of the sparse product (tiles of nonzeros, one warp each).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "primitives.cuh"
#include "trace.cuh"
#include "solve.cuh"
#include "spmv.cuh"
#include "build.cuh"
#include "leader_sums.cuh"

namespace psi {

namespace {

enum : uint32_t { kErrId = 1u, kErrSelf = 2u, kErrRate = 4u };

int grid_for(int64_t n, int threads = 256) {
  int64_t g = ceil_div(n > 0 ? n : 1, threads);
  int64_t cap = num_sms() * 16;
  return (int)(g < cap ? g : cap);
}

// Per-device streams and events for staging host inputs (see build_graph).
struct CopyLane {
  std::mutex mu;
  cudaStream_t cs[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> ev;
};
CopyLane& copy_lane() {
  static CopyLane lanes[64];
  int dev = 0;
  PSI_CUDA(cudaGetDevice(&dev));
  PSI_REQUIRE(dev >= 0 && dev < 64, PSI_ERR_CUDA, "device ordinal out of range");
  return lanes[dev];
}

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// f(i) for every i in [0, n), four independent indices per thread per round: the grids are
// capped at 16 blocks per SM, so a plain grid-stride loop keeps one load per thread in
// flight and streaming kernels end up latency-bound.
template <typename F>
__device__ __forceinline__ void grid_stride4(int64_t n, F&& f) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {
    f(i);
    f(i + stride);
    f(i + 2 * stride);
    f(i + 3 * stride);
  }
  for (; i < n; i += stride) f(i);
}

// block-wide reductions (blockDim.x a multiple of 32, at most 1024); every thread gets the result
__device__ __forceinline__ double block_max(double v) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();  // sh may still be read by a previous call
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, sh[w]);
  return r;
}
__device__ __forceinline__ uint32_t block_sum(uint32_t v) {
  __shared__ uint32_t sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  uint32_t r = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
  return r;
}

// lambda, mu finite, >= 0 and lambda + mu > 0 (the model needs c, d defined).  Tested on
// the bit patterns with integer operations (this part's FP64 pipe is narrow): a rate is
// valid when its exponent field is not all ones (finite) and it is either non-negative or
// a zero (-0.0 >= 0 holds); the pair when not both are zeros.
__device__ __forceinline__ bool rate_ok(uint64_t b) {
  const uint64_t mag = b & 0x7FFFFFFFFFFFFFFFull;
  return (mag >> 52) != 0x7FFull && ((b >> 63) == 0 || mag == 0);
}
// Also the range of the biased exponents of the nonzero rates (a subnormal rate counts as
// exponent 0): exp_range[0] = min (start at ~0), exp_range[1] = max (start at 0).
__global__ void k_check_rates(const double* __restrict__ lam, const double* __restrict__ mu, int64_t n,
                              uint32_t* err, uint32_t* exp_range) {
  uint32_t bad = 0, emin = 0xFFFFFFFFu, emax = 0;
  const unsigned long long* lb = reinterpret_cast<const unsigned long long*>(lam);
  const unsigned long long* mb = reinterpret_cast<const unsigned long long*>(mu);
  grid_stride4(n, [&](int64_t i) {
    const uint64_t x = lb[i], y = mb[i];
    const bool both_zero = ((x | y) & 0x7FFFFFFFFFFFFFFFull) == 0;
    if (!(rate_ok(x) && rate_ok(y)) || both_zero) bad = kErrRate;
    const uint64_t xm = x & 0x7FFFFFFFFFFFFFFFull, ym = y & 0x7FFFFFFFFFFFFFFFull;
    if (xm) {
      emin = min(emin, (uint32_t)(xm >> 52));
      emax = max(emax, (uint32_t)(xm >> 52));
    }
    if (ym) {
      emin = min(emin, (uint32_t)(ym >> 52));
      emax = max(emax, (uint32_t)(ym >> 52));
    }
  });
  if (bad) atomicOr(err, bad);
  emin = __reduce_min_sync(0xffffffffu, emin);
  emax = __reduce_max_sync(0xffffffffu, emax);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(exp_range, emin);
    atomicMax(exp_range + 1, emax);
  }
}

// Validates every edge and marks, exactly, who has followers (fol_bits) and who has leaders
// (lead_bits), one bit per user: a bit is set with an atomic OR only after a plain load
// found it clear (hub users are hit by many edges, and the 4 MB bitmaps mostly stay in L1
// and L2, so most edges cost two cached loads and no store).  Degrees are only an ordering key for locality: they
// are counted on the edges whose global index is a multiple of sample_mask + 1 (a power of
// two; all edges when sample_mask == 0).
// Runs on edges [e_base, e_base + m) (f and l point at edge e_base), so that the edges can
// be validated chunk by chunk as they arrive.  Four edges per thread per round, their eight
// bitmap loads issued before any update, so that the random reads overlap (updates only
// ever set bits, so reading the bits of later edges first changes nothing).
__global__ void k_edges(const int32_t* __restrict__ f, const int32_t* __restrict__ l, int64_t m, int64_t e_base,
                        int64_t n, int drop_self, int64_t sample_mask, uint32_t* fol_bits, uint32_t* lead_bits,
                        uint32_t* in_deg, uint32_t* out_deg, uint32_t* err) {
  constexpr int kQ = 4;
  uint32_t bits = 0;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e0 < m; e0 += kQ * gs) {
    int32_t a[kQ], b[kQ];
    bool ok[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const int64_t e = e0 + q * gs;
      ok[q] = e < m;
      a[q] = ok[q] ? f[e] : 0;
      b[q] = ok[q] ? l[e] : 0;
    }
    uint32_t hl[kQ], hf[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      if (ok[q]) {
        if (a[q] < 0 || a[q] >= n || b[q] < 0 || b[q] >= n) {
          bits |= kErrId;
          ok[q] = false;
        } else if (a[q] == b[q]) {
          if (!drop_self) bits |= kErrSelf;
          ok[q] = false;
        }
      }
      hl[q] = ok[q] ? ~lead_bits[a[q] >> 5] & (1u << (a[q] & 31)) : 0u;  // bit still to set
      hf[q] = ok[q] ? ~fol_bits[b[q] >> 5] & (1u << (b[q] & 31)) : 0u;
    }
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      if (hl[q]) atomicOr(&lead_bits[a[q] >> 5], hl[q]);
      if (hf[q]) atomicOr(&fol_bits[b[q] >> 5], hf[q]);
      if (ok[q] && ((e_base + e0 + q * gs) & sample_mask) == 0) {
        atomicAdd(&out_deg[a[q]], 1u);
        atomicAdd(&in_deg[b[q]], 1u);
      }
    }
  }
  if (bits) atomicOr(err, bits);
}

// key = class (2 bits) | rank (23 bits); value = user id.  A stable sort gives ties by id.
// With groups (independent graphs solved together), the key is class | group (10 bits) |
// rank (13 bits), so each group's users stay contiguous inside every class.
__global__ void k_node_keys(const uint32_t* __restrict__ fol_bits, const uint32_t* __restrict__ lead_bits,
                            const uint32_t* __restrict__ in_deg, const uint32_t* __restrict__ out_deg, int64_t n,
                            int reorder, const int32_t* __restrict__ group, uint32_t* key, uint32_t* val,
                            uint32_t* class_count) {
  __shared__ uint32_t cc[4];
  if (threadIdx.x < 4) cc[threadIdx.x] = 0;
  __syncthreads();
  GRID_STRIDE(i, n) {
    uint32_t di = in_deg[i], dout = out_deg[i];
    const bool has_fol = (fol_bits[i >> 5] >> (i & 31)) & 1u, has_lead = (lead_bits[i >> 5] >> (i & 31)) & 1u;
    uint32_t cls = has_fol ? (has_lead ? 0u : 1u) : (has_lead ? 2u : 3u);
    // rows (X, R) by row length (in-degree, which in these graphs also tracks how often a
    // user is gathered); U by how often it is gathered (out-degree)
    uint32_t deg = cls <= 1 ? di : (cls == 2 ? dout : 0u);
    if (group) {
      const uint32_t r13 = reorder ? (deg >= 0x1FFFu ? 0u : 0x1FFFu - deg) : 0u;
      key[i] = (cls << 23) | ((uint32_t)group[i] << 13) | r13;
    } else {
      const uint32_t rank = reorder ? (deg >= 0x7FFFFFu ? 0u : 0x7FFFFFu - deg) : 0u;
      key[i] = (cls << 23) | rank;
    }
    val[i] = (uint32_t)i;
    atomicAdd(&cc[cls], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 4 && cc[threadIdx.x]) atomicAdd(&class_count[threadIdx.x], cc[threadIdx.x]);
}

__global__ void k_invert(const uint32_t* __restrict__ perm, int64_t n, int32_t* __restrict__ inv) {
  grid_stride4(n, [&](int64_t k) { inv[perm[k]] = (int32_t)k; });
}

// key = (leader row << bf) | follower's gathered index (X: its id, U: id - nR); a dropped
// self-loop becomes the sentinel
__global__ void k_edge_keys(const int32_t* __restrict__ f, const int32_t* __restrict__ l, int64_t m,
                            const int32_t* __restrict__ inv, int32_t nX, int32_t nR, int bf, uint64_t sentinel,
                            uint64_t* __restrict__ key) {
  grid_stride4(m, [&](int64_t e) {
    const int32_t a = f[e], c = l[e];
    if (a == c) {
      key[e] = sentinel;
    } else {
      const uint32_t fi = (uint32_t)inv[a];
      const uint32_t gi = fi < (uint32_t)nX ? fi : fi - (uint32_t)nR;
      key[e] = ((uint64_t)(uint32_t)inv[c] << bf) | (uint64_t)gi;
    }
  });
}

// Duplicate merge and CSR of the sorted edge keys as one stream compaction over tiles of
// kUqTile keys: k_unique_count counts the unique keys of every tile, an exclusive scan of
// those counts gives each tile its output offset, and k_unique_write writes the unique keys
// in order (li: leader row, col: follower gathered index) with row_ptr[r] at the first
// unique key of row r, counting the rows seen.
constexpr int kUqThreads = 256;
constexpr int kUqItems = 16;
constexpr int kUqTile = kUqThreads * kUqItems;

// With exact leader sums (DUPS): every repeat of a key takes its leader's rates and one count
// back out of its follower's sums, which counted all edges.  Repeats of one key are adjacent:
// the lanes of a warp holding the same repeated key subtract once, times their number (a pair
// repeated hundreds of times would otherwise queue hundreds of atomics on one address).
template <bool DUPS>
__global__ void __launch_bounds__(kUqThreads) k_unique_count(const uint64_t* __restrict__ key, int64_t m,
                                                             uint64_t sentinel, uint32_t* __restrict__ count, int bf,
                                                             const FixedRow* __restrict__ rows,
                                                             unsigned long long* acc_s, unsigned long long* acc_b,
                                                             uint32_t* acc_c) {
  const int64_t base = (int64_t)blockIdx.x * kUqTile;
  const int lane = threadIdx.x & 31;
  uint32_t c = 0;
#pragma unroll 4
  for (int j = 0; j < kUqItems; ++j) {
    const int64_t e = base + (int64_t)j * kUqThreads + threadIdx.x;
    bool dup = false;
    uint64_t k = sentinel;
    if (e < m) {
      k = key[e];
      if (k != sentinel) {
        if (e == 0 || key[e - 1] != k) ++c;
        else dup = DUPS;
      }
    }
    if (DUPS && __any_sync(0xffffffffu, dup)) {
      const uint32_t peers = __match_any_sync(0xffffffffu, dup ? k : ~(uint64_t)lane);  // repeats of my key
      if (dup && __ffs(peers) - 1 == lane)
        fixed_sub_rows(ld_fixed_row(rows + (k >> bf)), (uint32_t)__popc(peers), acc_s, acc_b, acc_c,
                       (uint32_t)(k & ((1ull << bf) - 1)));
    }
  }
  c = block_sum(c);
  if (threadIdx.x == 0) count[blockIdx.x] = c;
}

__global__ void __launch_bounds__(kUqThreads) k_unique_write(const uint64_t* __restrict__ key, int64_t m,
                                                             uint64_t sentinel, const uint32_t* __restrict__ off,
                                                             int b, int32_t* __restrict__ li,
                                                             int32_t* __restrict__ col, int32_t* __restrict__ row_ptr,
                                                             uint32_t* rows_seen) {
  __shared__ uint32_t wcount[2][kUqThreads / 32];  // double-buffered: one barrier per round
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint64_t low = ((uint64_t)1 << b) - 1;
  const int64_t base = (int64_t)blockIdx.x * kUqTile;
  uint32_t run = off[blockIdx.x];  // output position of the tile's next unique key
  uint32_t rows = 0;
  for (int j = 0; j < kUqItems; ++j) {
    const int64_t e = base + (int64_t)j * kUqThreads + threadIdx.x;
    uint64_t k = sentinel;
    bool uniq = false, first_in_row = false;
    if (e < m) {
      k = key[e];
      if (k != sentinel) {
        const uint64_t prev = e > 0 ? key[e - 1] : 0;
        uniq = e == 0 || prev != k;
        first_in_row = e == 0 || (prev >> b) != (k >> b);
      }
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, uniq);
    if (lane == 0) wcount[j & 1][warp] = __popc(bal);
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kUqThreads / 32; ++w) {
      const uint32_t t = wcount[j & 1][w];
      before += w < warp ? t : 0u;
      total += t;
    }
    if (uniq) {
      const uint32_t o = run + before + __popc(bal & lt_mask);
      const int32_t r = (int32_t)(k >> b);
      if (li) li[o] = r;
      col[o] = (int32_t)(k & low);
      if (first_in_row) {
        row_ptr[r] = (int32_t)o;
        ++rows;
      }
    }
    run += total;
  }
  rows = block_sum(rows);  // one atomic per block
  if (threadIdx.x == 0 && rows) atomicAdd(rows_seen, rows);
}

// row_ptr[r] = first unique edge of leader r; counts the rows seen
__global__ void k_row_bounds(const int32_t* __restrict__ li, int64_t mu, int32_t* __restrict__ row_ptr,
                             uint32_t* rows_seen) {
  uint32_t c = 0;
  grid_stride4(mu, [&](int64_t e) {
    const int32_t r = li[e];
    if (e == 0 || li[e - 1] != r) {
      row_ptr[r] = (int32_t)e;
      ++c;
    }
  });
  c = block_sum(c);  // one atomic per block, not per thread
  if (threadIdx.x == 0 && c) atomicAdd(rows_seen, c);
}

__global__ void k_set_i32(int32_t* p, int32_t v) { *p = v; }

__global__ void k_row_max(const int32_t* __restrict__ row_ptr, int32_t n_rows, int32_t* mx) {
  int32_t best = 0;
  GRID_STRIDE(r, n_rows) {
    int32_t len = row_ptr[r + 1] - row_ptr[r];
    best = len > best ? len : best;
  }
  atomicMax(mx, best);
}

__global__ void k_permute_rates(const double* __restrict__ lam, const double* __restrict__ mu,
                                const uint32_t* __restrict__ perm, int64_t n, double* __restrict__ lam_i,
                                double* __restrict__ mu_i) {
  grid_stride4(n, [&](int64_t k) {
    const uint32_t o = perm[k];
    lam_i[k] = lam[o];
    mu_i[k] = mu[o];
  });
}

// leaders of every user from the follower-grouped CSR (rows: X then U, compact)
__global__ void k_leader_counts(const int32_t* __restrict__ rp_f, int32_t n_f, int32_t nX, int32_t nR, int32_t* cnt) {
  GRID_STRIDE(r, n_f) {
    const int64_t user = r < nX ? r : r + nR;
    cnt[user] = rp_f[r + 1] - rp_f[r];
  }
}

// w[k] = (lambda_k + mu_k, lambda_k), with the pad entry w[n] = (0, 0)
__global__ void k_leader_weights(const double* __restrict__ lam_i, const double* __restrict__ mu_i, int64_t n,
                                 D2* w) {
  GRID_STRIDE(k, n + 1) w[k] = k < n ? D2(lam_i[k] + mu_i[k], lam_i[k]) : D2(0.0, 0.0);
}
// the same weights as float pairs
__global__ void k_leader_weights_df(const double* __restrict__ lam_i, const double* __restrict__ mu_i, int64_t n,
                                    DF2* w) {
  GRID_STRIDE(k, n + 1) w[k] = k < n ? DF2(df_from(lam_i[k] + mu_i[k]), df_from(lam_i[k])) : DF2(0);
}

// 1/v for a positive finite v: an FP32 reciprocal as the seed (relative error <= 2^-24), then
// two steps of Newton's iteration for the reciprocal, r <- r + r (1 - v r), each of which
// squares the relative error (2^-48, then below FP64 rounding): the result is within about
// an ulp of 1/v.  Outside the FP32 normal range the FP64 division is used.
__device__ __forceinline__ double recip64(double v) {
  if (v > 1e-37 && v < 1e37) {
    double r = (double)(1.0f / (float)v);
    double e = fma(-v, r, 1.0);
    r = fma(r, e, r);
    e = fma(-v, r, 1.0);
    return fma(r, e, r);
  }
  return 1.0 / v;
}

// c_j = mu_j/(lambda_j+mu_j), d_j = lambda_j/(lambda_j+mu_j), 1/sigma_j (0 without leaders)
__global__ void k_user_vectors(const double* __restrict__ lam_i, const double* __restrict__ mu_i,
                               const double* __restrict__ sigma, const double* __restrict__ beta, int64_t n,
                               double* __restrict__ c64, double* __restrict__ d64, double* __restrict__ isig64,
                               float* __restrict__ c32, float* __restrict__ mu32, float* __restrict__ isig32,
                               unsigned long long* bnorm_bits, unsigned long long* rho_bits) {
  double bn = 0.0, rho = 0.0;
  grid_stride4(n, [&](int64_t k) {
    // two FP64 reciprocals per user (FP64 throughput is low on this part, and division is
    // a long FP64 sequence); c and d within about an ulp of mu/(lambda+mu), lambda/(lambda+mu)
    const double x = lam_i[k], y = mu_i[k], sg = sigma[k];
    const double inv = recip64(x + y);
    const double c = y * inv, d = x * inv;
    const double is = sg > 0.0 ? recip64(sg) : 0.0;
    c64[k] = c;
    d64[k] = d;
    isig64[k] = is;
    c32[k] = (float)c;
    mu32[k] = (float)y;
    isig32[k] = (float)is;
    if (sg > 0.0) {
      const double b = beta[k] * is, r = 1.0 - b;
      bn = b > bn ? b : bn;
      rho = r > rho ? r : rho;
    }
  });
  // one atomic per block (per-thread atomics on one address serialise); non-negative
  // doubles order like their bit patterns
  bn = block_max(bn);
  rho = block_max(rho);
  if (threadIdx.x == 0) {
    atomicMax(bnorm_bits, (unsigned long long)__double_as_longlong(bn));
    atomicMax(rho_bits, (unsigned long long)__double_as_longlong(rho));
  }
}

// tile_row[k] = row holding nonzero k*T (largest r with row_ptr[r] <= k*T); last = n_rows-1
__global__ void k_tile_rows(const int32_t* __restrict__ row_ptr, int32_t n_rows, int32_t num_tiles, int32_t tile,
                            int32_t* tile_row) {
  GRID_STRIDE(k, (int64_t)num_tiles + 1) {
    if (k == num_tiles) {
      tile_row[k] = n_rows - 1;
    } else {
      const int64_t pos = k * (int64_t)tile;
      int32_t lo = 0, hi = n_rows;  // search r in [0, n_rows)
      while (lo < hi) {
        int32_t mid = (lo + hi + 1) >> 1;
        if ((int64_t)row_ptr[mid] <= pos) lo = mid; else hi = mid - 1;
      }
      tile_row[k] = lo;
    }
  }
}

// tiles whose first row began in an earlier tile and ends inside this one
__global__ void k_fix_flags(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ tile_row,
                            int32_t num_tiles, int32_t tile, int64_t mu, uint32_t* flag) {
  GRID_STRIDE(k, num_tiles) {
    const int64_t nnz0 = k * (int64_t)tile;
    const int64_t nnz1 = nnz0 + tile < mu ? nnz0 + tile : mu;
    const int32_t r0 = tile_row[k];
    flag[k] = (k > 0 && (int64_t)row_ptr[r0] < nnz0 && (int64_t)row_ptr[r0 + 1] <= nnz1) ? 1u : 0u;
  }
}

__global__ void k_fix_compact(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ tile_row,
                              int32_t num_tiles, int32_t tile, int64_t mu, const uint32_t* __restrict__ pos,
                              int32_t* fix) {
  GRID_STRIDE(k, num_tiles) {
    const int64_t nnz0 = k * (int64_t)tile;
    const int64_t nnz1 = nnz0 + tile < mu ? nnz0 + tile : mu;
    const int32_t r0 = tile_row[k];
    if (k > 0 && (int64_t)row_ptr[r0] < nnz0 && (int64_t)row_ptr[r0 + 1] <= nnz1) fix[pos[k]] = (int32_t)k;
  }
}

__global__ void k_fill_i32(int32_t* x, int64_t lo, int64_t hi, int32_t v) {
  GRID_STRIDE(i, hi - lo) x[lo + i] = v;
}



template <typename T>
T read1(const T* d, cudaStream_t s) {
  T h{};
  PSI_CUDA(cudaMemcpyAsync(&h, d, sizeof(T), cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaStreamSynchronize(s));
  return h;
}

}  // namespace

// Merge-path schedule of a CSR with n_rows non-empty rows and m nonzeros.
Schedule make_schedule(const int32_t* row_ptr, int32_t n_rows, int64_t m, Allocator& al, cudaStream_t s,
                       int32_t tile) {
  Schedule sc;
  sc.tile = tile;
  sc.tiles = (int32_t)ceil_div(m, tile);
  sc.tile_row.reset(al, (size_t)sc.tiles + 1);
  if (sc.tiles == 0) {
    k_set_i32<<<1, 1, 0, s>>>(sc.tile_row.get(), n_rows - 1);
    PSI_LAUNCHED();
    sc.fix_tile.reset(al, 1);
    return sc;
  }
  k_tile_rows<<<grid_for(sc.tiles + 1), 256, 0, s>>>(row_ptr, n_rows, sc.tiles, tile, sc.tile_row.get());
  PSI_LAUNCHED();
  DBuf<uint32_t> fpos(al, (size_t)sc.tiles);
  DBuf<uint32_t> ftot(al, 1);
  k_fix_flags<<<grid_for(sc.tiles), 256, 0, s>>>(row_ptr, sc.tile_row.get(), sc.tiles, tile, m, fpos.get());
  PSI_LAUNCHED();
  exclusive_scan_u32(fpos.get(), fpos.get(), sc.tiles, al, s, ftot.get());
  sc.num_fix = (int32_t)read1(ftot.get(), s);
  sc.fix_tile.reset(al, (size_t)(sc.num_fix > 0 ? sc.num_fix : 1));
  if (sc.num_fix > 0) {
    k_fix_compact<<<grid_for(sc.tiles), 256, 0, s>>>(row_ptr, sc.tile_row.get(), sc.tiles, tile, m, fpos.get(),
                                                     sc.fix_tile.get());
    PSI_LAUNCHED();
  }
  return sc;
}

// y = (CSR) w for every row, both sums of the pair at once (one product + fix-up, FP64)
template <typename W>
void run_store_product(const int32_t* row_ptr, const int32_t* col, const Schedule& sc, int32_t n_rows, int64_t m,
                       const W* w, const EpiStore2& epi, Allocator& al, cudaStream_t s) {
  if (sc.tiles == 0) return;
  DBuf<DevState> st(al, 1);
  PSI_CUDA(cudaMemsetAsync(st.get(), 0, sizeof(DevState), s));
  int per_sm = 0;
  PSI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmv<W, EpiStore2>, kSpmvThreads, 0));
  const int grid = spmv_blocks(per_sm, sc.tiles);
  DBuf<double> gap_part(al, (size_t)grid);
  DBuf<W> carry_head(al, (size_t)sc.tiles), carry_tail(al, (size_t)sc.tiles);
  SpmvArgs a{};
  a.row_ptr = row_ptr;
  a.col = col;
  a.tile_row = sc.tile_row.get();
  a.tile = sc.tile;
  a.num_tiles = sc.tiles;
  a.n_rows = n_rows;
  a.m = m;
  a.state = st.get();
  a.gap_part = gap_part.get();
  a.carry_head = carry_head.get();
  a.carry_tail = carry_tail.get();
  k_spmv<W, EpiStore2><<<grid, kSpmvThreads, 0, s>>>(a, w, epi);
  PSI_LAUNCHED();
  if (sc.num_fix > 0) {
    int fgrid = fix_blocks(sc.num_fix);
    DBuf<double> gap_fix(al, (size_t)fgrid);
    FixArgs f{};
    f.row_ptr = row_ptr;
    f.tile_row = sc.tile_row.get();
    f.tile = sc.tile;
    f.fix_tile = sc.fix_tile.get();
    f.num_fix = sc.num_fix;
    f.state = st.get();
    f.gap_fix = gap_fix.get();
    f.carry_head = carry_head.get();
    f.carry_tail = carry_tail.get();
    k_fixup<W, EpiStore2><<<fgrid, kFixThreads, 0, s>>>(f, epi);
    PSI_LAUNCHED();
  }
}
template void run_store_product<D2>(const int32_t*, const int32_t*, const Schedule&, int32_t, int64_t, const D2*,
                                    const EpiStore2&, Allocator&, cudaStream_t);
template void run_store_product<DF2>(const int32_t*, const int32_t*, const Schedule&, int32_t, int64_t, const DF2*,
                                     const EpiStore2&, Allocator&, cudaStream_t);


bool is_device_pointer(const void* p);

void build_graph(Graph& g, int64_t n, int64_t m, const int32_t* follower, const int32_t* leader,
                 const double* lambda, const double* mu, BuildHook* hook) {
  cudaStream_t s = g.stream;
  Allocator& al = g.al;
  g.n = n;
  g.m_input = m;
  cudaEvent_t t0, t1;
  PSI_CUDA(cudaEventCreate(&t0));
  PSI_CUDA(cudaEventCreate(&t1));
  PSI_CUDA(cudaEventRecord(t0, s));

  NvtxPhases phases;
  phases.next("psi build 0: staging");
  // ---- stage inputs (host pointers are copied; device pointers are read in place).  Host
  //      copies run on two private streams (followers and lambda on one, leaders and mu on
  //      the other), the rates first, then the edges in chunks; the validation pass (step 1)
  //      takes each chunk as soon as both halves have arrived, so it overlaps the transfer.
  DBuf<int32_t> fbuf, lbuf;
  DBuf<double> lam_buf, mu_buf;
  const int32_t* df = follower;
  const int32_t* dl = leader;
  const double* dlam = lambda;
  const double* dmu = mu;
  const bool f_host = m > 0 && !is_device_pointer(follower);
  const bool l_host = m > 0 && !is_device_pointer(leader);
  const bool lam_host = !is_device_pointer(lambda);
  const bool mu_host = !is_device_pointer(mu);
  if (f_host) {
    fbuf.reset(al, (size_t)m);
    df = fbuf.get();
  }
  if (l_host) {
    lbuf.reset(al, (size_t)m);
    dl = lbuf.get();
  }
  if (lam_host) {
    lam_buf.reset(al, (size_t)n);
    dlam = lam_buf.get();
  }
  if (mu_host) {
    mu_buf.reset(al, (size_t)n);
    dmu = mu_buf.get();
  }
  const bool any_host = f_host || l_host || lam_host || mu_host;
  // two copy streams, so that two copy engines move the follower and the leader arrays at
  // once; they and their events belong to the device's copy lane (created once, kept for the
  // process: creating and destroying them on every build measured up to ~250 ms per build on
  // hosts whose memory was being compacted), held for the whole staging by one build at a time
  CopyLane& lane = copy_lane();
  std::unique_lock<std::mutex> lane_lock(lane.mu, std::defer_lock);
  cudaStream_t* cs = lane.cs;
  // [0]: buffers ready, [1], [2]: lambda, mu arrived, [3 + 2c], [4 + 2c]: follower / leader
  // chunk c arrived
  std::vector<cudaEvent_t>& arrived = lane.ev;
  const int64_t chunk = (int64_t)1 << 25;
  const int64_t n_chunks = m > 0 ? ceil_div(m, chunk) : 0;
  auto release_copies = [&]() {
    if (!lane_lock.owns_lock()) return;
    for (int i = 0; i < 2; ++i) cudaStreamSynchronize(cs[i]);
    lane_lock.unlock();
  };
  struct CopyGuard {
    decltype(release_copies)& f;
    ~CopyGuard() { f(); }
  } copy_guard{release_copies};  // waits for the copies before the staging buffers go
  if (any_host) {
    lane_lock.lock();
    for (int i = 0; i < 2; ++i)
      if (!cs[i]) PSI_CUDA(cudaStreamCreateWithFlags(&cs[i], cudaStreamNonBlocking));
    while ((int64_t)arrived.size() < 3 + 2 * n_chunks) {
      cudaEvent_t ev;
      PSI_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      arrived.push_back(ev);
    }
    int next_ev = 0;
    cudaEvent_t ready = arrived[next_ev++];  // the staging buffers exist (stream-ordered allocation on s)
    PSI_CUDA(cudaEventRecord(ready, s));
    for (int i = 0; i < 2; ++i) PSI_CUDA(cudaStreamWaitEvent(cs[i], ready, 0));
    if (lam_host) PSI_CUDA(cudaMemcpyAsync(lam_buf.get(), lambda, sizeof(double) * n, cudaMemcpyHostToDevice, cs[0]));
    if (mu_host) PSI_CUDA(cudaMemcpyAsync(mu_buf.get(), mu, sizeof(double) * n, cudaMemcpyHostToDevice, cs[1]));
    auto mark = [&](cudaStream_t c) { PSI_CUDA(cudaEventRecord(arrived[next_ev++], c)); };
    mark(cs[0]);  // [1]: lambda
    mark(cs[1]);  // [2]: mu
    for (int64_t c = 0; c < n_chunks; ++c) {
      const int64_t e0 = c * chunk, len = std::min(chunk, m - e0);
      if (f_host)
        PSI_CUDA(cudaMemcpyAsync(fbuf.get() + e0, follower + e0, sizeof(int32_t) * len, cudaMemcpyHostToDevice,
                                 cs[0]));
      if (l_host)
        PSI_CUDA(cudaMemcpyAsync(lbuf.get() + e0, leader + e0, sizeof(int32_t) * len, cudaMemcpyHostToDevice,
                                 cs[1]));
      mark(cs[0]);
      mark(cs[1]);
    }
  }

  phases.next("psi build 1: validation");
  // ---- 1. validation and raw degrees
  DBuf<uint32_t> err(al, 8);  // [0] error bits, [1..4] class counts, [5] rows seen, [6..7] spare
  PSI_CUDA(cudaMemsetAsync(err.get(), 0, 8 * sizeof(uint32_t), s));
  DBuf<uint32_t> exp_range(al, 2);  // biased exponents of the nonzero rates: min, max
  PSI_CUDA(cudaMemsetAsync(exp_range.get(), 0xFF, sizeof(uint32_t), s));
  PSI_CUDA(cudaMemsetAsync(exp_range.get() + 1, 0, sizeof(uint32_t), s));
  DBuf<uint32_t> in_deg(al, (size_t)n), out_deg(al, (size_t)n);
  const size_t n_words = (size_t)ceil_div(n, 32);
  DBuf<uint32_t> fol_bits(al, n_words), lead_bits(al, n_words);
  PSI_CUDA(cudaMemsetAsync(in_deg.get(), 0, sizeof(uint32_t) * n, s));
  PSI_CUDA(cudaMemsetAsync(out_deg.get(), 0, sizeof(uint32_t) * n, s));
  PSI_CUDA(cudaMemsetAsync(fol_bits.get(), 0, sizeof(uint32_t) * n_words, s));
  PSI_CUDA(cudaMemsetAsync(lead_bits.get(), 0, sizeof(uint32_t) * n_words, s));
  if (any_host) {
    PSI_CUDA(cudaStreamWaitEvent(s, arrived[1], 0));
    PSI_CUDA(cudaStreamWaitEvent(s, arrived[2], 0));
  }
  k_check_rates<<<grid_for(n), 256, 0, s>>>(dlam, dmu, n, err.get(), exp_range.get());
  PSI_LAUNCHED();
  if (m > 0) {
    // degree sample: every edge up to 2^26 edges, then a fixed 1-in-2^k subset
    int64_t sample_mask = 0;
    while (m > ((sample_mask + 1) << 26)) sample_mask = 2 * sample_mask + 1;
    for (int64_t c = 0; c < n_chunks; ++c) {
      const int64_t e0 = c * chunk, len = std::min(chunk, m - e0);
      if (any_host) {
        PSI_CUDA(cudaStreamWaitEvent(s, arrived[3 + 2 * c], 0));
        PSI_CUDA(cudaStreamWaitEvent(s, arrived[4 + 2 * c], 0));
      }
      k_edges<<<grid_for(len), 256, 0, s>>>(df + e0, dl + e0, len, e0, n, g.opt.self_loops == PSI_DROP ? 1 : 0,
                                            sample_mask, fol_bits.get(), lead_bits.get(), in_deg.get(), out_deg.get(),
                                            err.get());
      PSI_LAUNCHED();
    }
  }
  const uint32_t ebits = read1(err.get(), s);
  PSI_REQUIRE(!(ebits & kErrId), PSI_ERR_OUT_OF_RANGE_ID, "an edge endpoint is outside [0, n)");
  PSI_REQUIRE(!(ebits & kErrSelf), PSI_ERR_SELF_LOOP, "a user follows itself (self_loops = PSI_REJECT)");
  PSI_REQUIRE(!(ebits & kErrRate), PSI_ERR_BAD_RATE, "lambda/mu must be finite, >= 0, with lambda + mu > 0");

  phases.next("psi build 2: renumbering");
  // ---- 2. renumbering by class and degree
  DBuf<uint32_t> perm32;
  {
    DBuf<uint32_t> k0(al, (size_t)n), k1(al, (size_t)n), v0(al, (size_t)n), v1(al, (size_t)n);
    k_node_keys<<<grid_for(n), 256, 0, s>>>(fol_bits.get(), lead_bits.get(), in_deg.get(), out_deg.get(), n,
                                            g.opt.reorder ? 1 : 0, hook ? hook->user_group() : nullptr, k0.get(),
                                            v0.get(), err.get() + 1);
    PSI_LAUNCHED();
    bool alt = radix_sort<uint32_t>(k0.get(), k1.get(), v0.get(), v1.get(), n, 25, al, s);
    perm32 = alt ? std::move(v1) : std::move(v0);
  }
  in_deg.release();
  out_deg.release();
  fol_bits.release();
  lead_bits.release();
  uint32_t cls[4], erange[2];
  PSI_CUDA(cudaMemcpyAsync(cls, err.get() + 1, sizeof(cls), cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaMemcpyAsync(erange, exp_range.get(), sizeof(erange), cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaStreamSynchronize(s));
  g.nX = (int32_t)cls[0];
  g.nR = (int32_t)cls[1];
  g.nU = (int32_t)cls[2];
  g.nZ = (int32_t)cls[3];
  g.n_rows = g.nX + g.nR;
  g.perm.reset(al, (size_t)n);
  PSI_CUDA(cudaMemcpyAsync(g.perm.get(), perm32.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));

  phases.next("psi build 3: edge sort and CSR");
  // ---- 3. sort, merge duplicates, transposed CSR.  Keys hold the leader row and the
  //         follower's gathered index: bits_for(n_rows - 1) + bits_for(nu) bits (the low
  //         field never reaches all ones, so the all-ones sentinel sorts last)
  const int64_t nu = (int64_t)g.nX + g.nU;
  const int bf = bits_for((uint64_t)nu);
  const int bl = g.n_rows > 1 ? bits_for((uint64_t)(g.n_rows - 1)) : 1;
  const int b = bf;  // width of the follower field (the follower sort below)
  const uint64_t sentinel = ((uint64_t)1 << (bl + bf)) - 1;
  int64_t mu_count = 0;
  DBuf<int32_t> li;
  // sigma and beta as exact sums (leader_sums.cuh) when the rates allow and no hook needs the
  // follower-grouped CSR: formed from the keys half-way through the sort, no such CSR built
  const bool exact = (hook == nullptr || !hook->follower_csr()) && nu > 0 && m > 0 && m < ((int64_t)1 << 31) &&
                     exact_sums_apply(erange[0], erange[1]);
  ExactLeaderSums xs;
  DBuf<double> lam_i(al, (size_t)n), mu_i(al, (size_t)n);
  k_permute_rates<<<grid_for(n), 256, 0, s>>>(dlam, dmu, perm32.get(), n, lam_i.get(), mu_i.get());
  PSI_LAUNCHED();
  if (exact) exact_sums_prepare(xs, lam_i.get(), mu_i.get(), g.n_rows, (int32_t)nu, erange[0], al, s);
  {
    DBuf<int32_t> inv(al, (size_t)n);
    k_invert<<<grid_for(n), 256, 0, s>>>(perm32.get(), n, inv.get());
    PSI_LAUNCHED();
    DBuf<uint64_t> k0(al, (size_t)m), k1(al, (size_t)m);
    if (m > 0) {
      k_edge_keys<<<grid_for(m), 256, 0, s>>>(df, dl, m, inv.get(), g.nX, g.nR, bf, sentinel, k0.get());
      PSI_LAUNCHED();
    }
    inv.release();
    fbuf.release();
    lbuf.release();
    bool alt;
    if (exact) {  // the follower field first; between the two halves the keys are grouped by follower
      const bool a1 = radix_sort_bits<uint64_t>(k0.get(), k1.get(), nullptr, nullptr, m, 0, bf, al, s);
      uint64_t* mid = a1 ? k1.get() : k0.get();
      // the group sums also count the digit of the sort's next pass
      DBuf<uint32_t> first_counts(al, (size_t)ceil_div(m, kRadixTileKeys) * 256);
      exact_sums_groups(xs, mid, m, bf, (int32_t)nu, radix_first_mask(bf, bf + bl), first_counts.get(), s);
      const bool a2 = radix_sort_bits<uint64_t>(mid, a1 ? k0.get() : k1.get(), nullptr, nullptr, m, bf, bf + bl, al, s,
                                                nullptr, nullptr, first_counts.get());
      alt = a1 != a2;
    } else {
      alt = radix_sort<uint64_t>(k0.get(), k1.get(), nullptr, nullptr, m, bl + bf, al, s);
    }
    const uint64_t* keys = alt ? k1.get() : k0.get();
    const int64_t uq_tiles = ceil_div(m, kUqTile);
    DBuf<uint32_t> uq_off(al, (size_t)(uq_tiles > 0 ? uq_tiles : 1));
    DBuf<uint32_t> total(al, 1);
    if (m > 0) {
      if (exact)
        k_unique_count<true><<<(unsigned)uq_tiles, kUqThreads, 0, s>>>(keys, m, sentinel, uq_off.get(), bf,
                                                                      xs.rows.get(), xs.s.get(), xs.b.get(),
                                                                      xs.cnt.get());
      else
        k_unique_count<false><<<(unsigned)uq_tiles, kUqThreads, 0, s>>>(keys, m, sentinel, uq_off.get(), bf, nullptr,
                                                                       nullptr, nullptr, nullptr);
      PSI_LAUNCHED();
      exclusive_scan_u32(uq_off.get(), uq_off.get(), uq_tiles, al, s, total.get());
      mu_count = read1(total.get(), s);
    } else {
      mu_count = 0;
    }
    g.m_unique = mu_count;
    g.tile = g.opt.spmv_tile > 0 ? g.opt.spmv_tile : spmv_tile_for(mu_count);
    g.num_tiles = (int32_t)ceil_div(mu_count, g.tile);
    const int64_t padded = ceil_div(mu_count, kSpmvTileMax) * kSpmvTileMax;
    g.col.reset(al, (size_t)(padded > 0 ? padded : 4));
    if (!exact) li.reset(al, (size_t)(mu_count > 0 ? mu_count : 1));  // leader rows, for the follower sort
    g.row_ptr.reset(al, (size_t)g.n_rows + 1);
    if (mu_count > 0) {
      k_unique_write<<<(unsigned)uq_tiles, kUqThreads, 0, s>>>(keys, m, sentinel, uq_off.get(), bf, li.get(),
                                                              g.col.get(), g.row_ptr.get(), err.get() + 5);
      PSI_LAUNCHED();
    }
    if (padded > mu_count) {
      k_fill_i32<<<grid_for(padded - mu_count), 256, 0, s>>>(g.col.get(), mu_count, padded, (int32_t)nu);
      PSI_LAUNCHED();
    }
  }
  {
    k_set_i32<<<1, 1, 0, s>>>(g.row_ptr.get() + g.n_rows, (int32_t)mu_count);
    PSI_LAUNCHED();
    const uint32_t rows_seen = read1(err.get() + 5, s);
    PSI_REQUIRE((int64_t)rows_seen == g.n_rows, PSI_ERR_CUDA, "internal: row count mismatch in CSR build");
    DBuf<int32_t> mx(al, 1);
    PSI_CUDA(cudaMemsetAsync(mx.get(), 0, sizeof(int32_t), s));
    if (g.n_rows > 0) {
      k_row_max<<<grid_for(g.n_rows), 256, 0, s>>>(g.row_ptr.get(), g.n_rows, mx.get());
      PSI_LAUNCHED();
    }
    g.max_followers = read1(mx.get(), s);
  }

  phases.next("psi build 4: sigma and beta");
  // ---- 4. leader sums per follower: (sigma, beta) = L (lambda + mu, lambda): exact sums
  //         (above), or one load-balanced product over the follower-grouped CSR (rows X then U)
  perm32.release();
  lam_buf.release();
  mu_buf.release();
  DBuf<double> sigma(al, (size_t)n), beta(al, (size_t)n);
  g.n_leaders.reset(al, (size_t)n);
  PSI_CUDA(cudaMemsetAsync(g.n_leaders.get(), 0, sizeof(int32_t) * n, s));
  PSI_CUDA(cudaMemsetAsync(sigma.get(), 0, sizeof(double) * n, s));
  PSI_CUDA(cudaMemsetAsync(beta.get(), 0, sizeof(double) * n, s));
  if (exact) {
    exact_sums_finish(xs, (int32_t)nu, g.nX, g.nR, sigma.get(), beta.get(), g.n_leaders.get(), s);
    xs = ExactLeaderSums();
  } else if (mu_count > 0) {
    const int64_t mc = mu_count;
    const int32_t n_f = g.nX + g.nU;  // followers: users with leaders
    const int32_t tiles_f = (int32_t)ceil_div(mc, kSpmvTileMax);
    DBuf<uint32_t> fk0(al, (size_t)mc), fk1(al, (size_t)mc);
    DBuf<uint32_t> lv0(al, (size_t)tiles_f * kSpmvTileMax), lv1(al, (size_t)mc);
    // keys: the followers' gathered indices (the transposed CSR's columns, left untouched);
    // values: the leader rows (non-negative int32, read as uint32)
    bool alt = radix_sort<uint32_t>(fk0.get(), fk1.get(), lv0.get(), lv1.get(), mc, b, al, s,
                                    reinterpret_cast<const uint32_t*>(g.col.get()),
                                    reinterpret_cast<const uint32_t*>(li.get()));
    li.release();
    uint32_t* fs = alt ? fk1.get() : fk0.get();
    uint32_t* ls = alt ? lv1.get() : lv0.get();
    DBuf<uint32_t> lpad;
    if (ls != lv0.get()) {  // the column array of the product needs whole tiles
      lpad = std::move(lv0);
      PSI_CUDA(cudaMemcpyAsync(lpad.get(), ls, sizeof(uint32_t) * mc, cudaMemcpyDeviceToDevice, s));
      ls = lpad.get();
    } else {
      lpad = std::move(lv0);
    }
    if ((int64_t)tiles_f * kSpmvTileMax > mc) {
      k_fill_i32<<<grid_for((int64_t)tiles_f * kSpmvTileMax - mc), 256, 0, s>>>(reinterpret_cast<int32_t*>(ls), mc,
                                                                            (int64_t)tiles_f * kSpmvTileMax, (int32_t)n);
      PSI_LAUNCHED();
    }
    DBuf<int32_t> rp_f(al, (size_t)n_f + 1);
    PSI_CUDA(cudaMemsetAsync(err.get() + 6, 0, sizeof(uint32_t), s));
    k_row_bounds<<<grid_for(mc), 256, 0, s>>>(reinterpret_cast<const int32_t*>(fs), mc, rp_f.get(), err.get() + 6);
    PSI_LAUNCHED();
    k_set_i32<<<1, 1, 0, s>>>(rp_f.get() + n_f, (int32_t)mc);
    PSI_LAUNCHED();
    const uint32_t frows = read1(err.get() + 6, s);
    PSI_REQUIRE((int64_t)frows == n_f, PSI_ERR_CUDA, "internal: follower row count mismatch");
    fk0.release();
    fk1.release();
    lv1.release();
    Schedule sch = make_schedule(rp_f.get(), n_f, mc, al, s, kSpmvTileMax);
    // sigma and beta: FP64 sums in the FP64 mode, float-pair sums otherwise (FP64 adds are
    // slow on this part; ~48-bit sums are far inside the FP32-series mode's accuracy)
    if (g.opt.precision == PSI_FP64) {
      DBuf<D2> w(al, (size_t)n + 1);
      k_leader_weights<<<grid_for(n + 1), 256, 0, s>>>(lam_i.get(), mu_i.get(), n, w.get());
      PSI_LAUNCHED();
      run_store_product(rp_f.get(), reinterpret_cast<const int32_t*>(ls), sch, n_f, mc, w.get(),
                        EpiStore2{sigma.get(), beta.get(), g.nX, g.nR}, al, s);
    } else {
      DBuf<DF2> w(al, (size_t)n + 1);
      k_leader_weights_df<<<grid_for(n + 1), 256, 0, s>>>(lam_i.get(), mu_i.get(), n, w.get());
      PSI_LAUNCHED();
      run_store_product(rp_f.get(), reinterpret_cast<const int32_t*>(ls), sch, n_f, mc, w.get(),
                        EpiStore2{sigma.get(), beta.get(), g.nX, g.nR}, al, s);
    }
    k_leader_counts<<<grid_for(n_f), 256, 0, s>>>(rp_f.get(), n_f, g.nX, g.nR, g.n_leaders.get());
    PSI_LAUNCHED();
    if (hook && hook->follower_csr()) {
      FollowerCsr fc{rp_f.get(), reinterpret_cast<const int32_t*>(ls), &sch, n_f, mc};
      hook->on_follower_csr(g, fc);
    }
  } else {
    li.release();
  }
  if (hook) hook->on_leader_sums(g, sigma.get(), beta.get());

  phases.next("psi build 5: constants");
  // ---- 5. per-user constants
  g.c64.reset(al, (size_t)n);
  g.d64.reset(al, (size_t)n);
  g.isig64.reset(al, (size_t)n);
  g.c32.reset(al, (size_t)n);
  g.mu32.reset(al, (size_t)n);
  g.isig32.reset(al, (size_t)n);
  DBuf<unsigned long long> norms(al, 2);
  PSI_CUDA(cudaMemsetAsync(norms.get(), 0, 2 * sizeof(unsigned long long), s));
  k_user_vectors<<<grid_for(n), 256, 0, s>>>(lam_i.get(), mu_i.get(), sigma.get(), beta.get(), n, g.c64.get(),
                                             g.d64.get(), g.isig64.get(), g.c32.get(), g.mu32.get(), g.isig32.get(),
                                             norms.get(), norms.get() + 1);
  PSI_LAUNCHED();
  g.lam64 = std::move(lam_i);
  g.mu64 = std::move(mu_i);
  {
    unsigned long long nb[2];
    PSI_CUDA(cudaMemcpyAsync(nb, norms.get(), sizeof(nb), cudaMemcpyDeviceToHost, s));
    PSI_CUDA(cudaStreamSynchronize(s));
    double v[2];
    memcpy(v, nb, sizeof(v));
    g.bnorm_inf = v[0];
    g.rho_inf = v[1];
  }

  phases.next("psi build 6: schedule");
  // ---- 6. tile schedule of the Power-psi product
  {
    Schedule sch = make_schedule(g.row_ptr.get(), g.n_rows, mu_count, al, s, g.tile);
    g.tile_row = std::move(sch.tile_row);
    g.fix_tile = std::move(sch.fix_tile);
    g.num_fix = sch.num_fix;
  }
  PSI_CUDA(cudaEventRecord(t1, s));
  PSI_CUDA(cudaStreamSynchronize(s));
  float ms = 0.f;
  PSI_CUDA(cudaEventElapsedTime(&ms, t0, t1));
  g.build_ms = ms;
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
}

}  // namespace psi
