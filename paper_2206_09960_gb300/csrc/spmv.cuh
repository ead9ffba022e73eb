// spmv.cuh -- the Power-psi sparse product, one launch per step.
//
// With a_ji = mu_i / sigma_j and b_ji = lambda_i / sigma_j (Sec. II) the operator
// factorises: s^T A = mu (.) G(s), s^T B = lambda (.) G(s), where
//     G(s)_i = sum_{j follows i} s_j / sigma_j = sum_{j in F(i)} u_j,   u = s (.) (1/sigma).
// So one step of Eq. 14 is a pattern-only pull over the followers F(i) of every user i
// (the transposed CSR: rows = leaders, columns = followers) followed by a per-row
// epilogue; no per-edge value is stored.
//
// Load balance is merge-based: the nonzeros are cut into fixed tiles (512 to 2048 per
// graph), one warp per tile; row boundaries inside a tile come from a bitmap of row ends built from
// the tile's slice of row_ptr, and partial row sums are joined by warp segmented scans and
// a register carried from step to step.  A row that starts in an earlier tile is closed by
// the fix-up kernel, which adds the tile carries in tile order.  Every sum therefore runs
// in an order fixed by the graph alone: results are bit-reproducible.
#pragma once

#include "common.cuh"
#include "df.cuh"

namespace psi {

// ------------------------------------------------------------------ value types
// A pair of FP64 sums carried through one product (16-byte gathers).
struct D2 {
  double a, b;
  D2() = default;
  __device__ __forceinline__ D2(int z) : a(z), b(z) {}
  __device__ __forceinline__ D2(double x, double y) : a(x), b(y) {}
};
__device__ __forceinline__ D2 operator+(D2 x, D2 y) { return D2(x.a + y.a, x.b + y.b); }
__device__ __forceinline__ D2& operator+=(D2& x, D2 y) {
  x.a += y.a;
  x.b += y.b;
  return x;
}
__device__ __forceinline__ D2 ld_gather(const D2* p, uint64_t pol) {
  double x, y;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;" : "=d"(x), "=d"(y) : "l"(p), "l"(pol));
  return D2(x, y);
}
// Four FP32 sums carried through one product (16-byte gathers).
struct F4 {
  float x, y, z, w;
  F4() = default;
  __device__ __forceinline__ F4(int v) : x((float)v), y((float)v), z((float)v), w((float)v) {}
  __device__ __forceinline__ F4(float a, float b, float c, float d) : x(a), y(b), z(c), w(d) {}
};
__device__ __forceinline__ F4 operator+(F4 a, F4 b) { return F4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ F4& operator+=(F4& a, F4 b) {
  a = a + b;
  return a;
}
__device__ __forceinline__ F4 ld_gather(const F4* p, uint64_t pol) {
  float a, b, c, d;
  asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
               : "=f"(a), "=f"(b), "=f"(c), "=f"(d)
               : "l"(p), "l"(pol));
  return F4(a, b, c, d);
}
template <typename T>
__device__ __forceinline__ T shfl_up_t(T v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
template <>
__device__ __forceinline__ D2 shfl_up_t<D2>(D2 v, int o) {
  return D2(__shfl_up_sync(0xffffffffu, v.a, o), __shfl_up_sync(0xffffffffu, v.b, o));
}
template <typename T>
__device__ __forceinline__ T shfl_xor_t(T v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
template <>
__device__ __forceinline__ D2 shfl_xor_t<D2>(D2 v, int o) {
  return D2(__shfl_xor_sync(0xffffffffu, v.a, o), __shfl_xor_sync(0xffffffffu, v.b, o));
}

template <>
__device__ __forceinline__ DF shfl_up_t<DF>(DF v, int o) {
  return DF(__shfl_up_sync(0xffffffffu, v.hi, o), __shfl_up_sync(0xffffffffu, v.lo, o));
}
template <>
__device__ __forceinline__ DF shfl_xor_t<DF>(DF v, int o) {
  return DF(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}
template <>
__device__ __forceinline__ DF2 shfl_up_t<DF2>(DF2 v, int o) {
  return DF2(shfl_up_t(v.a, o), shfl_up_t(v.b, o));
}
template <>
__device__ __forceinline__ DF2 shfl_xor_t<DF2>(DF2 v, int o) {
  return DF2(shfl_xor_t(v.a, o), shfl_xor_t(v.b, o));
}
template <>
__device__ __forceinline__ F4 shfl_xor_t<F4>(F4 v, int o) {
  return F4(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o),
            __shfl_xor_sync(0xffffffffu, v.z, o), __shfl_xor_sync(0xffffffffu, v.w, o));
}
template <>
__device__ __forceinline__ F4 shfl_up_t<F4>(F4 v, int o) {
  return F4(__shfl_up_sync(0xffffffffu, v.x, o), __shfl_up_sync(0xffffffffu, v.y, o),
            __shfl_up_sync(0xffffffffu, v.z, o), __shfl_up_sync(0xffffffffu, v.w, o));
}
template <typename T>
__device__ __forceinline__ T shfl_idx_t(T v, int src) { return __shfl_sync(0xffffffffu, v, src); }
template <>
__device__ __forceinline__ D2 shfl_idx_t<D2>(D2 v, int src) {
  return D2(__shfl_sync(0xffffffffu, v.a, src), __shfl_sync(0xffffffffu, v.b, src));
}
template <>
__device__ __forceinline__ DF shfl_idx_t<DF>(DF v, int src) {
  return DF(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
}
template <>
__device__ __forceinline__ DF2 shfl_idx_t<DF2>(DF2 v, int src) {
  return DF2(shfl_idx_t(v.a, src), shfl_idx_t(v.b, src));
}
template <>
__device__ __forceinline__ F4 shfl_idx_t<F4>(F4 v, int src) {
  return F4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
            __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
}

// ------------------------------------------------------------------ lane accumulators
// The sum of a lane's items between row ends.  For float pairs the high parts are added with
// Knuth's two-sum, whose error terms and the low parts collect in a second float, and the
// pair is renormalised only when the sum leaves the lane (at a row end, into the scan): the
// dependent chain per item is one FP32 add instead of a whole pair sum.  The result is the
// pair sum to within the FP32 rounding of the collected errors, about 2^-24 of a few ulps
// of the high part -- the accuracy of the pair sums themselves.
template <typename T>
struct LaneAcc {
  T v;
  __device__ __forceinline__ explicit LaneAcc(T x) : v(x) {}
  __device__ __forceinline__ void add(T x) { v += x; }
  __device__ __forceinline__ T get() const { return v; }
};
template <>
struct LaneAcc<DF> {
  float s, c;
  __device__ __forceinline__ explicit LaneAcc(DF x) : s(x.hi), c(x.lo) {}
  __device__ __forceinline__ void add(DF x) {
    const float t = s + x.hi;
    const float z = t - s;
    c += ((s - (t - z)) + (x.hi - z)) + x.lo;
    s = t;
  }
  __device__ __forceinline__ DF get() const {
    const float h = s + c;
    return DF(h, c - (h - s));
  }
};
template <>
struct LaneAcc<DF2> {
  LaneAcc<DF> a, b;
  __device__ __forceinline__ explicit LaneAcc(DF2 x) : a(x.a), b(x.b) {}
  __device__ __forceinline__ void add(DF2 x) {
    a.add(x.a);
    b.add(x.b);
  }
  __device__ __forceinline__ DF2 get() const { return DF2(a.get(), b.get()); }
};

// ------------------------------------------------------------------ epilogues
// row(r, y, gap): y = G(.)_r for row r (a user with followers); add |change| to gap.

// Algorithm 2 step in precision T: s_new = c + mu*y (Eq. 14), gap += |s_new - s_old|,
// u_new = s_new/sigma for users that have leaders.
template <typename T>
struct EpiPlain {
  const T* c;
  const T* mu;
  const T* isig;
  const T* s_old;
  T* s_new;
  T* u_new;
  int32_t nX;
  __device__ __forceinline__ void row(int32_t r, T y, double& gap, uint64_t pol_s, uint64_t pol_k) const {
    T s = ld_stream(c + r, pol_s) + ld_stream(mu + r, pol_s) * y;
    gap += fabs((double)s - (double)ld_stream(s_old + r, pol_s));
    s_new[r] = s;
    if (r < nX) st_keep(u_new + r, s * ld_stream(isig + r, pol_s), pol_k);
  }
};

// Series step (Eq. 13): term_t = mu * G(term_{t-1}) in FP32, s += term_t in FP64,
// gap += |term_t| (= |s_t - s_{t-1}|), v_new = term_t / sigma.
struct EpiSeries {
  const float* mu;
  const float* isig;
  double* s64;
  float* v_new;
  int32_t nX;
  __device__ __forceinline__ void row(int32_t r, float y, double& gap, uint64_t pol_s, uint64_t pol_k) const {
    float t = ld_stream(mu + r, pol_s) * y;
    s64[r] = ld_stream(s64 + r, pol_s) + (double)t;
    gap += fabs((double)t);
    if (r < nX) st_keep(v_new + r, t * ld_stream(isig + r, pol_s), pol_k);
  }
};

// y of a product, as FP64, and an FP64 value in a product's gather format
template <typename T>
__device__ __forceinline__ double as_double(T y) {
  return (double)y;
}
template <>
__device__ __forceinline__ double as_double<DF>(DF y) {
  return df_value(y);
}
template <typename G>
__device__ __forceinline__ G to_gather(double x) {
  return (G)x;
}
template <>
__device__ __forceinline__ DF to_gather<DF>(double x) {
  return df_from(x);
}

// Confirming step from the FP64 iterate: s_new = c + mu*y, r = s_new - s, gap += |r|,
// s = s_new, u_new = s_new/sigma (next gather), v32 = r/sigma (start of an FP32 correction
// series).  G is the product's gather and sum type: DF (float pairs) when the tolerance is
// far above their rounding, double otherwise; the row's update is FP64 either way.
template <typename G>
struct EpiResid {
  const double* c;
  const double* mu;
  const double* isig;
  double* s64;
  G* u_new;
  float* v32;
  int32_t nX;
  __device__ __forceinline__ void row(int32_t r, G yp, double& gap, uint64_t pol_s, uint64_t pol_k) const {
    const double y = as_double(yp);
    double sn = ld_stream(c + r, pol_s) + ld_stream(mu + r, pol_s) * y;
    double rr = sn - s64[r];
    gap += fabs(rr);
    s64[r] = sn;
    if (r < nX) {
      double is = ld_stream(isig + r, pol_s);
      st_keep(u_new + r, to_gather<G>(sn * is), pol_k);
      v32[r] = (float)(rr * is);
    }
  }
};

// Final step of Algorithm 2: psi_r = (lambda_r * G(s)_r + d_r) / N.
template <typename T>
struct EpiFinal {
  const double* lam;
  const double* d;
  double* psi;
  double n;
  __device__ __forceinline__ void row(int32_t r, T y, double& gap, uint64_t pol_s, uint64_t) const {
    psi[r] = (ld_stream(lam + r, pol_s) * as_double(y) + ld_stream(d + r, pol_s)) / n;
  }
};

// Plain product output of a pair of sums: out_a[user] = y.a, out_b[user] = y.b, with row r
// standing for user r < nX ? r : r + skip (per-user sums over a CSR whose rows skip a
// block of users).
struct EpiStore2 {
  double* out_a;
  double* out_b;
  int32_t nX;
  int32_t skip;
  __device__ __forceinline__ void row(int32_t r, D2 y, double&, uint64_t, uint64_t) const {
    const int32_t user = r < nX ? r : r + skip;
    out_a[user] = y.a;
    out_b[user] = y.b;
  }
  __device__ __forceinline__ void row(int32_t r, DF2 y, double&, uint64_t, uint64_t) const {
    const int32_t user = r < nX ? r : r + skip;
    out_a[user] = df_value(y.a);
    out_b[user] = df_value(y.b);
  }
};

struct SpmvArgs {
  const int32_t* row_ptr;
  const int32_t* col;
  const int32_t* tile_row;
  int32_t tile;           // nonzeros per tile: kSpmvTileMin .. kSpmvTileMax, a power of two
  int32_t num_tiles;
  int32_t hot;            // entries u[0, hot) staged in the block's shared memory (0: none)
  int32_t n_rows;
  int32_t* tile_ctr;      // tiles claimed at run time (4-byte sums only): {tiles claimed, warps
                          // done}, zero between launches (the last warp resets them); nullptr:
                          // a fixed stride
  int64_t m;
  const DevState* state;  // skip the step when state->done
  double* gap_part;       // [gridDim.x] (fixed stride)
  double* gap_tile;       // [num_tiles] the gap of each tile (claimed tiles)
  void* carry_head;       // [num_tiles] T
  void* carry_tail;       // [num_tiles] T
};

struct FixArgs {
  const int32_t* row_ptr;
  const int32_t* tile_row;
  int32_t tile;
  const int32_t* fix_tile;
  int32_t num_fix;
  const DevState* state;
  double* gap_fix;        // [gridDim.x]
  const void* carry_head;
  const void* carry_tail;
  const double* gap_tile; // the product's per-tile gaps, added in fixed slices (gap_tiles > 0)
  int32_t gap_tiles;
};

// An epilogue may declare `static constexpr bool kTileSkip = true` and a member
// `bool tile_on(int32_t tile) const`: tiles it turns off are neither gathered nor reduced
// (their rows get no epilogue call).  Used when several independent graphs share one
// product and some of them have stopped stepping.
template <typename E, typename = void>
struct tile_skip_of {
  static constexpr bool value = false;
};
template <typename E>
struct tile_skip_of<E, decltype((void)E::kTileSkip)> {
  static constexpr bool value = E::kTileSkip;
};

// Nonzeros per tile for a product over m nonzeros: the largest power of two up to
// kSpmvTileMax that still gives every resident warp of the series product (5 CTAs of 8 warps
// per SM) four tiles, at least kSpmvTileMin.
inline int32_t spmv_tile_for(int64_t m) {
  const int64_t tiles_wanted = num_sms() * 5 * kSpmvWarps * 4;
  int32_t t = kSpmvTileMax;
  while (t > kSpmvTileMin && m < (int64_t)t * tiles_wanted) t >>= 1;
  return t;
}

// Blocks for a product over `tiles` tiles: `per_sm` resident blocks on every SM, and no
// more blocks than the tiles fill (one tile per warp).
inline int spmv_blocks(int per_sm, int32_t tiles) {
  const int64_t cap = (int64_t)(per_sm > 0 ? per_sm : 1) * num_sms();
  const int64_t need = ceil_div(tiles > 0 ? tiles : 1, kSpmvWarps);
  return (int)(need < cap ? need : cap);
}

// Resident blocks per SM the register allocation must allow (measured at R-MAT scale 25):
// the products are bound by gather latency and gain from more warps, down to 48 registers
// for FP32 sums (5 blocks; 6 spill), 64 for 8-byte sums (4 blocks) and 128 for the
// 16-byte pair sums of the graph build (2 blocks).
template <typename T>
constexpr int spmv_min_blocks() {
  return sizeof(T) == 4 ? 5 : (sizeof(T) == 8 ? 4 : 2);
}

// Threads per block of the product with a shared-memory copy of the most gathered entries
// (one block per SM: the copy takes most of the SM's shared memory).
constexpr int kSpmvHotWarps = 32;

// One warp per tile.  With a.tile_ctr (FP32 sums), each warp takes its first two tiles by a
// grid-wide stride and claims every later one from a counter (the claim for the tile after
// next is issued when a tile starts and read when it ends, so its latency hides under the
// tile); SMs that run faster take more tiles, and the tile's gap is written per tile
// (a.gap_tile, a fixed lane tree) so that its sum keeps an order fixed by the graph.
// Without it the warps walk the tiles with a grid-wide stride and leave a per-block gap.  A
// tile's row ends are first marked in a bitmap in shared memory (bit q: nonzero nnz0 + q is
// the last one of its row) from the tile's slice of row_ptr.  Every row has at least one
// nonzero, so the k-th row end of the tile belongs to row tile_row[tile] + k.  Each step
// covers kSpmvStep nonzeros, kSpmvItems per lane: a lane sums its items and runs the
// epilogue of every row that begins and ends among them at once; the row of its first row
// end, which may have begun in earlier lanes, is completed by a warp segmented scan and
// closed by the same lane, and the sum of the row still open after the step is carried to
// the next step in a register.  Row indices come from the lanes' prefix counts of row ends
// (one ballot per item position) and the scan's segment flags from one ballot.  The
// gathers of the next step, and the column indices of the step after it, are issued before
// the current step is reduced.  No block barrier is taken inside the tile loop.
//
// The gathers are served by the L1 and, for entries that miss it, by L2 requests, whose
// rate bounds the product on large graphs.  With a.hot > 0 (WARPS = kSpmvHotWarps, one
// block per SM) each block first copies u[0, a.hot) -- the users gathered most, since the
// gathered index space is ordered by decreasing degree -- into shared memory and reads
// those entries there; the rest of the SM's on-chip memory stays L1 for the others.  With
// a.hot == 0 shared memory holds only the bitmaps and the whole of it serves as L1.
template <typename T, typename Epi, int WARPS = kSpmvWarps>
__global__ void __launch_bounds__(WARPS * 32, WARPS == kSpmvWarps ? spmv_min_blocks<T>() : 1)
    k_spmv(SpmvArgs a, const T* __restrict__ u, Epi epi) {
  constexpr bool kSkip = tile_skip_of<Epi>::value;
  constexpr int kWords = kSpmvTileMax / 32;  // bitmap words of the largest tile
  if (a.state->done) return;
  __shared__ uint32_t ends_sh[WARPS][kWords];
  __shared__ double gsh[WARPS];
  extern __shared__ __align__(16) unsigned char spmv_hot_dyn[];
  T* hot = reinterpret_cast<T*>(spmv_hot_dyn);
  const int32_t nhot = a.hot;
  if (nhot > 0) {
    for (int32_t i = threadIdx.x; i < nhot; i += WARPS * 32) hot[i] = u[i];
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* ends = ends_sh[warp];
  const uint64_t pol_s = policy_evict_first();
  const uint64_t pol_k = policy_evict_last();
  T* carry_head = static_cast<T*>(a.carry_head);
  T* carry_tail = static_cast<T*>(a.carry_tail);
  const int32_t stride = (int32_t)gridDim.x * WARPS;
  double gap = 0.0;

  // column indices of step k of a tile (this lane's kSpmvItems nonzeros; col is padded to
  // whole tiles, pad entries point at u[n] = 0) and their gathered values
  auto load_cols = [&](int32_t t, int k, int (&c)[kSpmvItems]) {
    ld_stream_v8(a.col + (int64_t)t * a.tile + k * kSpmvStep + lane * kSpmvItems, pol_s, c);
  };
  auto gather = [&](const int (&c)[kSpmvItems], T (&x)[kSpmvItems]) {
#pragma unroll
    for (int j = 0; j < kSpmvItems; ++j) x[j] = c[j] < nhot ? hot[c[j]] : ld_gather(u + c[j], pol_k);
  };
  // this warp's tiles, in order: first, first + stride, ... (all below 2^31: num_tiles +
  // 32 strides); with tile skipping, the gates of 32 candidates are tested at once (one per
  // lane) and a ballot gives the tiles to run
  const int32_t first = (int32_t)blockIdx.x * WARPS + warp;
  int32_t cand = first;  // next candidate tile (the first of the next batch when skipping)
  uint32_t on_bits = 0;  // tiles of the last batch still to run
  auto next_tile = [&]() -> int32_t {
    if constexpr (kSkip) {
      while (on_bits == 0) {
        if (cand >= a.num_tiles) return a.num_tiles;
        const int32_t tl = cand + lane * stride;
        on_bits = __ballot_sync(0xffffffffu, tl < a.num_tiles && epi.tile_on(tl));
        cand += 32 * stride;
      }
      const int b = __ffs(on_bits) - 1;
      on_bits &= on_bits - 1;
      return cand - (32 - b) * stride;
    } else {
      const int32_t t = cand;
      cand += stride;
      return t < a.num_tiles ? t : a.num_tiles;
    }
  };

  // claims only in the 4-byte products: the 8- and 16-byte sums need the registers
  constexpr bool kClaims = !kSkip && sizeof(T) == 4;
  const bool dyn = kClaims && a.tile_ctr != nullptr;
  int32_t tile = next_tile();
  int32_t nxt = kClaims ? next_tile() : 0;  // with claims the next tile is known a tile ahead
  // software pipeline: the values of the next step are in flight while a step is reduced,
  // and the column indices of the step after it, so its gathers issue without waiting
  T xn[kSpmvItems];
  int cn[kSpmvItems];
  const int steps = a.tile / kSpmvStep;  // >= 2: the index loads run two steps ahead
  const int words = a.tile / 32;
  if (tile < a.num_tiles) {
    int c0[kSpmvItems];
    load_cols(tile, 0, c0);
    gather(c0, xn);
    load_cols(tile, 1, cn);
  }
  while (tile < a.num_tiles) {
    const int32_t nnz0 = tile * a.tile;  // < m < 2^31
    const int32_t r0 = a.tile_row[tile];
    const int32_t nr = a.tile_row[tile + 1] - r0 + 1;  // rows touching the tile
    const int32_t next = kClaims ? nxt : next_tile();
    int32_t claim = a.num_tiles;
    if (dyn && lane == 0 && next < a.num_tiles) claim = 2 * stride + atomicAdd(a.tile_ctr, 1);
    for (int w = lane; w < words; w += 32) ends[w] = 0u;
    __syncwarp();
    const bool head_open = ld_stream(a.row_ptr + r0, pol_s) < nnz0;  // row r0 began earlier
    for (int i = lane; i < nr; i += 32) {
      const int32_t q = ld_stream(a.row_ptr + r0 + i + 1, pol_s) - 1 - nnz0;
      if ((uint32_t)q < (uint32_t)a.tile) atomicOr(ends + (q >> 5), 1u << (q & 31));
    }
    __syncwarp();

    T open = T(0);      // sum of the row left open by the last step
    int32_t done = 0;   // row ends of the tile in the steps before this one
#pragma unroll 1
    for (int k = 0; k < steps; ++k) {
      T x[kSpmvItems];
#pragma unroll
      for (int j = 0; j < kSpmvItems; ++j) x[j] = xn[j];
      if (k + 1 < steps || next < a.num_tiles) gather(cn, xn);
      if (k + 2 < steps) load_cols(tile, k + 2, cn);
      else if (next < a.num_tiles) load_cols(next, k + 2 - steps, cn);

      const int bit = k * kSpmvStep + lane * kSpmvItems;
      const uint32_t e = (ends[bit >> 5] >> (bit & 31)) & 0xffu;  // this lane's row ends
      const int cnt = __popc(e);
      // row ends in the lanes before this one and in the whole step, one ballot per item
      const uint32_t below = (1u << lane) - 1u;
      int before = 0, total = 0;
#pragma unroll
      for (int j = 0; j < kSpmvItems; ++j) {
        const uint32_t b = __ballot_sync(0xffffffffu, (e >> j) & 1u);
        before += __popc(b & below);
        total += __popc(b);
      }
      const int32_t j0 = done + before;  // index in the tile of this lane's first row end
      done += total;
      // rows that begin and end inside this lane are closed now; the head (up to the first
      // row end) waits for the sum carried in from the lanes before
      LaneAcc<T> acc(lane == 0 ? open : T(0));
      T head = T(0);
      int32_t jr = j0;
#pragma unroll
      for (int j = 0; j < kSpmvItems; ++j) {
        acc.add(x[j]);
        if ((e >> j) & 1u) {
          if (jr == j0) head = acc.get();
          else epi.row(r0 + jr, acc.get(), gap, pol_s, pol_k);
          ++jr;
          acc = LaneAcc<T>(T(0));
        }
      }
      // segmented inclusive scan of the sums after each lane's last row end: after offset o
      // a lane holds the sum over lanes max(lane - 2o + 1, last_end) .. lane, so it adds its
      // partner's value only while no row end lies in its own window
      const int last_end = 31 - __clz(__ballot_sync(0xffffffffu, cnt > 0) & (below | (1u << lane)));
      T v = acc.get();
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const T vu = shfl_up_t(v, o);
        if (lane >= o && last_end <= lane - o) v = vu + v;
      }
      T ve = shfl_up_t(v, 1);  // carried into this lane
      if (lane == 0) ve = T(0);
      open = shfl_idx_t(v, 31);
      // the first row end of a tile whose first row began in an earlier tile leaves its
      // partial for the fix-up kernel
      if (cnt > 0) {
        const T y = ve + head;
        if (j0 == 0 && head_open) carry_head[tile] = y;
        else epi.row(r0 + j0, y, gap, pol_s, pol_k);
      }
    }
    if (lane == 0) carry_tail[tile] = open;  // the sum after the tile's last row end
    __syncwarp();  // the bitmap is rewritten for the next tile
    if constexpr (kClaims) {
      if (dyn) {
        // the tile's gap, summed over the lanes in a fixed tree: the same whichever warp ran it
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gap += __shfl_xor_sync(0xffffffffu, gap, o);
        if (lane == 0) a.gap_tile[tile] = gap;
        gap = 0.0;
        const int32_t nn = __shfl_sync(0xffffffffu, claim, 0);
        nxt = (next < a.num_tiles && nn < a.num_tiles) ? nn : a.num_tiles;
      } else {
        nxt = next_tile();
      }
    }
    tile = next;
  }
  if (dyn && lane == 0) {
    // every claim of this warp is made before it counts itself done; the last warp to finish
    // leaves both counters at zero for the next launch
    __threadfence();
    if (atomicAdd(a.tile_ctr + 1, 1) == stride - 1) {
      atomicExch(a.tile_ctr, 0);
      atomicExch(a.tile_ctr + 1, 0);
    }
  }
  // per-CTA gap partial, fixed order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gap += __shfl_xor_sync(0xffffffffu, gap, o);
  if (lane == 0) gsh[warp] = gap;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < WARPS; ++w) t += gsh[w];
    a.gap_part[blockIdx.x] = t;
  }
}

constexpr int kFixThreads = 256;  // threads per fix-up block, one fix-up each

// Blocks for the fix-up of num_fix rows (at most 8 per SM: the gap_fix buffers' size).
inline int fix_blocks(int32_t num_fix) {
  const int64_t need = ceil_div(num_fix > 0 ? num_fix : 1, kFixThreads);
  const int64_t cap = num_sms() * 8;
  return (int)(need < cap ? need : cap);
}

// Rows spanning more tiles than this are summed by a whole warp in the fix-up.
constexpr int32_t kFixLongSpan = 128;

// Closes rows that began in an earlier tile: y = the sum of the carries of the tiles the row
// crosses, in tile order, plus the partial of the tile where it ends.  A row is one lane's
// task (four interleaved partial sums over its tiles, joined pairwise) unless it spans more
// than kFixLongSpan tiles; such a row (a leader with hundreds of thousands of followers and
// more) is summed by its whole warp -- lane l takes tiles l, l + 32, ... in order, then a
// fixed shuffle tree -- so its cost grows with span / 32 instead of span / 4.  Both orders are
// fixed by the graph: results stay bit-reproducible.
template <typename T, typename Epi>
__global__ void __launch_bounds__(kFixThreads) k_fixup(FixArgs a, Epi epi) {
  if (a.state->done) return;
  __shared__ double gsh[kFixThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t pol_s = policy_evict_first();
  const uint64_t pol_k = policy_evict_last();
  const T* ch = static_cast<const T*>(a.carry_head);
  const T* ct = static_cast<const T*>(a.carry_tail);
  double gap = 0.0;
  for (int32_t b = blockIdx.x * kFixThreads + warp * 32; b < a.num_fix; b += gridDim.x * kFixThreads) {
    const int32_t q = b + lane;
    int32_t k = 0, r0 = 0, kk0 = 0;
    if (q < a.num_fix) {
      k = a.fix_tile[q];
      r0 = a.tile_row[k];
      kk0 = a.row_ptr[r0] / a.tile;  // tile where row r0 begins
    }
    const bool is_long = q < a.num_fix && k - kk0 > kFixLongSpan;
    if (q < a.num_fix && !is_long) {
      int32_t kk = kk0;
      T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
      for (; kk + 4 <= k; kk += 4) {
        s0 += ct[kk];
        s1 += ct[kk + 1];
        s2 += ct[kk + 2];
        s3 += ct[kk + 3];
      }
      for (; kk < k; ++kk) s0 += ct[kk];
      epi.row(r0, ((s0 + s1) + (s2 + s3)) + ch[k], gap, pol_s, pol_k);
    }
    uint32_t longs = __ballot_sync(0xffffffffu, is_long);
    while (longs) {  // long rows of this batch, one after another, by the whole warp
      const int src = __ffs(longs) - 1;
      longs &= longs - 1;
      const int32_t kl = __shfl_sync(0xffffffffu, k, src);
      const int32_t rl = __shfl_sync(0xffffffffu, r0, src);
      const int32_t kb = __shfl_sync(0xffffffffu, kk0, src);
      T acc = T(0);
      for (int32_t kk = kb + lane; kk < kl; kk += 32) acc += ct[kk];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc = acc + shfl_xor_t(acc, o);
      if (lane == 0) epi.row(rl, acc + ch[kl], gap, pol_s, pol_k);
    }
  }
  if (a.gap_tiles > 0) {  // this block's fixed slice of the product's per-tile gaps
    const int32_t per = (int32_t)ceil_div(a.gap_tiles, gridDim.x);
    const int32_t t1 = min(a.gap_tiles, (int32_t)blockIdx.x * per + per);
    for (int32_t t = (int32_t)blockIdx.x * per + threadIdx.x; t < t1; t += kFixThreads) gap += a.gap_tile[t];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gap += __shfl_xor_sync(0xffffffffu, gap, o);
  if (lane == 0) gsh[warp] = gap;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kFixThreads / 32; ++w) t += gsh[w];
    a.gap_fix[blockIdx.x] = t;
  }
}

}  // namespace psi
