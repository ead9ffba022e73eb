// spmv.cuh -- the Power-psi sparse product, one launch per step.
//
// With a_ji = mu_i / sigma_j and b_ji = lambda_i / sigma_j (Sec. II) the operator
// factorises: s^T A = mu (.) G(s), s^T B = lambda (.) G(s), where
//     G(s)_i = sum_{j follows i} s_j / sigma_j = sum_{j in F(i)} u_j,   u = s (.) (1/sigma).
// So one step of Eq. 14 is a pattern-only pull over the followers F(i) of every user i
// (the transposed CSR: rows = leaders, columns = followers) followed by a per-row
// epilogue; no per-edge value is stored.
//
// Load balance is merge-based: the nonzeros are cut into fixed tiles of kSpmvTile (each
// thread owns kSpmvItems consecutive nonzeros, loaded as two 16-byte vectors), rows are
// found by a binary search over the tile's slice of row_ptr, and partial row sums are
// joined by a block-wide segmented scan.  A row that starts in an earlier tile is closed
// by the fix-up kernel, which adds the tile carries in tile order.  Every sum therefore
// runs in an order fixed by the graph alone: results are bit-reproducible.
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
  int32_t num_tiles;
  int32_t n_rows;
  int64_t m;
  const DevState* state;  // skip the step when state->done
  double* gap_part;       // [gridDim.x]
  void* carry_head;       // [num_tiles] T
  void* carry_tail;       // [num_tiles] T
};

struct FixArgs {
  const int32_t* row_ptr;
  const int32_t* tile_row;
  const int32_t* fix_tile;
  int32_t num_fix;
  const DevState* state;
  double* gap_fix;        // [gridDim.x]
  const void* carry_head;
  const void* carry_tail;
};

// Segmented scan element: f = a row ended inside the span, v = sum after the last row
// end.  Combining a left span L with the right span R that follows it:
//   (L.f | R.f, R.f ? R.v : L.v + R.v).
template <typename T>
__device__ __forceinline__ void seg_join(int lf, T lv, int& rf, T& rv) {  // R <- L . R
  if (!rf) rv = lv + rv;
  rf |= lf;
}

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

template <typename T, typename Epi>
__global__ void __launch_bounds__(kSpmvThreads) k_spmv(SpmvArgs a, const T* __restrict__ u, Epi epi) {
  constexpr bool kSkip = tile_skip_of<Epi>::value;
  if (a.state->done) return;
  __shared__ int32_t rp[kSpmvTile + 2];  // row_ptr slice of the tile's rows
  __shared__ T ys[kSpmvTile + 1];        // G(.) of every row that ends in the tile
  __shared__ int wf[kSpmvThreads / 32];
  __shared__ T wv[kSpmvThreads / 32];
  __shared__ double gsh[kSpmvThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t pol_s = policy_evict_first();
  const uint64_t pol_k = policy_evict_last();
  T* carry_head = static_cast<T*>(a.carry_head);
  T* carry_tail = static_cast<T*>(a.carry_tail);
  double gap = 0.0;

  // column indices and gathered values of one tile: this thread's kSpmvItems nonzeros
  // (col is padded to whole tiles, pad entries point at u[n] = 0)
  auto gather_tile = [&](int32_t t, T (&x)[kSpmvItems]) {
    const int* cp = a.col + (int64_t)t * kSpmvTile + (int64_t)threadIdx.x * kSpmvItems;
#pragma unroll
    for (int q = 0; q < kSpmvItems / 8; ++q) {
      int c[8];
      ld_stream_v8(cp + 8 * q, pol_s, c);
#pragma unroll
      for (int j = 0; j < 8; ++j) x[8 * q + j] = ld_gather(u + c[j], pol_k);
    }
  };
  T xn[kSpmvItems];
  if (!kSkip && (int32_t)blockIdx.x < a.num_tiles) gather_tile(blockIdx.x, xn);

  for (int32_t tile = blockIdx.x; tile < a.num_tiles; tile += gridDim.x) {
    if constexpr (kSkip) {
      if (!epi.tile_on(tile)) continue;  // uniform over the block
    }
    const int64_t nnz0 = (int64_t)tile * kSpmvTile;
    const int64_t nnz1 = nnz0 + kSpmvTile < a.m ? nnz0 + kSpmvTile : a.m;
    const int32_t r0 = a.tile_row[tile];
    const int32_t r_hi = a.tile_row[tile + 1];
    const int32_t nr = r_hi - r0 + 1;  // rows touching [nnz0, nnz0 + tile)
    __syncthreads();                    // shared buffers are reused across tiles
    if constexpr (kSkip) gather_tile(tile, xn);
    for (int i = threadIdx.x; i <= nr; i += kSpmvThreads) rp[i] = ld_stream(a.row_ptr + r0 + i, pol_s);
    const int64_t p0 = nnz0 + (int64_t)threadIdx.x * kSpmvItems;
    T x[kSpmvItems];
#pragma unroll
    for (int i = 0; i < kSpmvItems; ++i) x[i] = xn[i];
    const int32_t next = tile + gridDim.x;
    if (kSpmvPrefetch && !kSkip) {
      if (next < a.num_tiles) gather_tile(next, xn);
    } else {
      (void)next;
    }
    __syncthreads();
    // first row whose end lies beyond p0
    int lo = 0, hi = nr;
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if ((int64_t)rp[mid + 1] > p0) hi = mid; else lo = mid + 1;
    }
    int cur = lo;
    int64_t next_end = cur < nr ? (int64_t)rp[cur + 1] : INT64_MAX;
    T acc = T(0), first_val = T(0);
    int has_end = 0, first_row = 0;
#pragma unroll
    for (int i = 0; i < kSpmvItems; ++i) {
      acc += x[i];
      if (p0 + i + 1 == next_end) {  // row `cur` ends at nonzero p0 + i
        if (!has_end) {
          has_end = 1;
          first_row = cur;
          first_val = acc;
        } else {
          ys[cur] = acc;               // the row began inside this thread's span
        }
        acc = T(0);
        ++cur;
        next_end = cur < nr ? (int64_t)rp[cur + 1] : INT64_MAX;
      }
    }
    // block-wide segmented scan of (has_end, acc) in thread order
    int f = has_end;
    T v = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int fu = __shfl_up_sync(0xffffffffu, f, o);
      T vu = shfl_up_t(v, o);
      if (lane >= o) seg_join(fu, vu, f, v);
    }
    if (lane == 31) { wf[warp] = f; wv[warp] = v; }
    int fe = __shfl_up_sync(0xffffffffu, f, 1);  // exclusive within the warp
    T ve = shfl_up_t(v, 1);
    if (lane == 0) { fe = 0; ve = T(0); }
    __syncthreads();
    int fw = 0;  // inclusive prefix of the warps before this one
    T vw = T(0);
    for (int w = 0; w < warp; ++w) {
      int g = wf[w];
      T gv = wv[w];
      seg_join(fw, vw, g, gv);
      fw = g;
      vw = gv;
    }
    seg_join(fw, vw, fe, ve);  // exclusive prefix of this thread
    if (has_end) ys[first_row] = ve + first_val;
    if (threadIdx.x == kSpmvThreads - 1) {
      seg_join(fw, vw, f, v);  // inclusive prefix of the whole tile
      carry_tail[tile] = v;
    }
    __syncthreads();
    // epilogues of the rows that end in this tile, one row per thread, coalesced; a first
    // row that began in an earlier tile leaves its partial for the fix-up kernel
    const bool head_open = (int64_t)rp[0] < nnz0;
    for (int i = threadIdx.x; i < nr; i += kSpmvThreads) {
      if ((int64_t)rp[i + 1] > nnz1) break;  // this row and the next ones end later
      if (i == 0 && head_open) carry_head[tile] = ys[0];
      else epi.row(r0 + i, ys[i], gap, pol_s, pol_k);
    }
    if (!kSpmvPrefetch && !kSkip && next < a.num_tiles) gather_tile(next, xn);
  }
  // per-CTA gap partial, fixed order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gap += __shfl_xor_sync(0xffffffffu, gap, o);
  if (lane == 0) gsh[warp] = gap;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kSpmvThreads / 32; ++w) t += gsh[w];
    a.gap_part[blockIdx.x] = t;
  }
}

constexpr int kFixWarps = 8;  // warps per fix-up block

// Closes rows that began in an earlier tile: y = sum of the tile carries in tile order
// plus the partial of the tile where the row ends.
template <typename T, typename Epi>
__global__ void __launch_bounds__(kFixWarps * 32) k_fixup(FixArgs a, Epi epi) {
  if (a.state->done) return;
  __shared__ double gsh[kFixWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t pol_s = policy_evict_first();
  const uint64_t pol_k = policy_evict_last();
  const T* ch = static_cast<const T*>(a.carry_head);
  const T* ct = static_cast<const T*>(a.carry_tail);
  double gap = 0.0;
  for (int32_t q = blockIdx.x * kFixWarps + warp; q < a.num_fix; q += gridDim.x * kFixWarps) {
    const int32_t k = a.fix_tile[q];
    const int32_t r0 = a.tile_row[k];
    const int32_t ks = a.row_ptr[r0] / kSpmvTile;  // tile where row r0 begins
    T acc = T(0);
    for (int32_t kk = ks + lane; kk < k; kk += 32) acc += ct[kk];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += shfl_xor_t(acc, o);
    if (lane == 0) epi.row(r0, acc + ch[k], gap, pol_s, pol_k);
  }
  if (lane == 0) gsh[warp] = gap;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kFixWarps; ++w) t += gsh[w];
    a.gap_fix[blockIdx.x] = t;
  }
}

}  // namespace psi
