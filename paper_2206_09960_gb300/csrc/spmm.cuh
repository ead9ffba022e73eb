// spmm.cuh -- the Power-psi product for S activity scenarios on one graph at once.
//
// The follower pattern is the same for every scenario; only the per-user constants differ
// (sigma, c, mu, lambda, d per scenario).  The gathered values of all scenarios of one user
// are stored contiguously (row j of a [users x S] matrix), so one column index feeds S
// values: for S = 64, one fully used 256-byte row per nonzero.
//
// Load balance: the nonzeros are cut into chunks of kSpmmChunk; one warp owns a chunk and
// walks it nonzero by nonzero, all lanes together (row boundaries are warp-uniform, so no
// divergence), lane l holding scenarios 2l and 2l+1.  A row that began in an earlier chunk
// leaves its partial sums (S values) for the fix-up kernel, which adds the chunk carries
// in chunk order: results are bit-reproducible.  Scenarios are masked out individually once
// they have met their stop test.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "df.cuh"

namespace psi {

constexpr int kSpmmChunk = 512;  // nonzeros per warp task (a divisor of kSpmvTileMax)
constexpr int kSpmmMaxS = 64;    // scenarios per launch (lane l: 2l, 2l+1)

struct SpmmArgs {
  const int32_t* row_ptr;
  const int32_t* col;          // padded to whole chunks with the zero entry
  const int32_t* chunk_row;    // [num_chunks + 1]: row holding the chunk's first nonzero
  int32_t num_chunks;
  int32_t n_rows;
  int64_t m;
  int32_t S;                   // padded scenario count (64)
  const int32_t* active;       // [S]: 1 while a scenario still steps
  const int32_t* done;         // nonzero: no scenario steps, skip the launch
  double* gap_part;            // [warps][S] (fixed stride)
  int32_t* chunk_ctr;          // chunks claimed at run time (FP32 products): {claimed, warps
                               // done}, zero between launches; nullptr: a fixed stride
  double* gap_chunk;           // [num_chunks][S] the gaps of each chunk (claimed chunks)
  float2* carry_head;          // [num_chunks][S/2] (FP32 products)
  float2* carry_tail;
  double2* carry_head64;       // FP64 products
  double2* carry_tail64;
};

// Series step for S scenarios: t = mu_s * y_s, s_s += t (FP64), v_s = t / sigma_s.
// Every epilogue loads a row's operands in pre(), issued when the warp starts the row, so
// that they arrive while its gathers are summed; row() applies them at the row's end.
struct EpiSeriesS {
  const float2* mu;     // [users][S/2]
  const float2* isig;
  double2* s64;         // [users][S/2] as double pairs
  float2* v_new;        // [gathered][S/2]
  int32_t nX;
  struct Pre {
    float2 m, is;
    double2 s;
  };
  __device__ __forceinline__ Pre pre(int32_t r, int lane) const {
    const int64_t o = (int64_t)r * 32 + lane;
    return Pre{mu[o], r < nX ? isig[o] : make_float2(0.f, 0.f), s64[o]};
  }
  __device__ __forceinline__ void row(int32_t r, int lane, float2 y, const int* act, double2& gap, const Pre& p) const {
    const int64_t o = (int64_t)r * 32 + lane;
    float2 t = make_float2(act[0] ? p.m.x * y.x : 0.f, act[1] ? p.m.y * y.y : 0.f);
    double2 s = p.s;
    s.x += (double)t.x;
    s.y += (double)t.y;
    s64[o] = s;
    gap.x += fabs((double)t.x);
    gap.y += fabs((double)t.y);
    if (r < nX) v_new[o] = make_float2(t.x * p.is.x, t.y * p.is.y);
  }
};

// Confirming step for S scenarios: s_new = c + mu*y, r = s_new - s, s = s_new,
// u_new = s_new/sigma (next gather, float pairs), v32 = r/sigma (start of the next series);
// inactive scenarios keep their state.  The product sums float pairs; the update is FP64.
__device__ __forceinline__ double2 pair_value(double2 y) { return y; }
__device__ __forceinline__ double2 pair_value(DF2 y) { return make_double2(df_value(y.a), df_value(y.b)); }
template <typename V>
__device__ __forceinline__ V pair_gather(double x, double y);
template <>
__device__ __forceinline__ double2 pair_gather<double2>(double x, double y) { return make_double2(x, y); }
template <>
__device__ __forceinline__ DF2 pair_gather<DF2>(double x, double y) { return DF2{df_from(x), df_from(y)}; }

// V = DF2 (float pairs) when the tolerance is far above their rounding, double2 otherwise.
template <typename V>
struct EpiResidS {
  const double2* c;
  const double2* mu;
  const double2* isig;
  double2* s64;
  V* u_new;
  float2* v32;
  int32_t nX;
  struct Pre {
    double2 cc, mm, s, is;
  };
  __device__ __forceinline__ Pre pre(int32_t r, int lane) const {
    const int64_t o = (int64_t)r * 32 + lane;
    return Pre{c[o], mu[o], s64[o], r < nX ? isig[o] : make_double2(0.0, 0.0)};
  }
  __device__ __forceinline__ void row(int32_t r, int lane, V yp, const int* act, double2& gap, const Pre& p) const {
    const int64_t o = (int64_t)r * 32 + lane;
    const double2 y = pair_value(yp);
    const double2 cc = p.cc, mm = p.mm, s = p.s;
    double2 sn = make_double2(cc.x + mm.x * y.x, cc.y + mm.y * y.y);
    if (!act[0]) sn.x = s.x;
    if (!act[1]) sn.y = s.y;
    const double2 rr = make_double2(sn.x - s.x, sn.y - s.y);
    gap.x += fabs(rr.x);
    gap.y += fabs(rr.y);
    s64[o] = sn;
    if (r < nX) {
      const double2 is = p.is;
      u_new[o] = pair_gather<V>(sn.x * is.x, sn.y * is.y);
      v32[o] = make_float2((float)(rr.x * is.x), (float)(rr.y * is.y));
    }
  }
};

// psi_s = (lambda_s * G(s_s) + d_s) / N for every scenario.
template <typename V>
struct EpiFinalS {
  const double2* lam;
  const double2* d;
  double2* psi;
  double n;
  struct Pre {
    double2 l, dd;
  };
  __device__ __forceinline__ Pre pre(int32_t r, int lane) const {
    const int64_t o = (int64_t)r * 32 + lane;
    return Pre{lam[o], d[o]};
  }
  __device__ __forceinline__ void row(int32_t r, int lane, V yp, const int*, double2&, const Pre& p) const {
    const int64_t o = (int64_t)r * 32 + lane;
    const double2 y = pair_value(yp);
    psi[o] = make_double2((p.l.x * y.x + p.dd.x) / n, (p.l.y * y.y + p.dd.y) / n);
  }
};

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 add2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ DF2 add2(DF2 a, DF2 b) { return DF2{a.a + b.a, a.b + b.b}; }
template <typename V>
__device__ __forceinline__ V zero2();
template <>
__device__ __forceinline__ float2 zero2<float2>() { return make_float2(0.f, 0.f); }
template <>
__device__ __forceinline__ double2 zero2<double2>() { return make_double2(0.0, 0.0); }
template <>
__device__ __forceinline__ DF2 zero2<DF2>() { return DF2{DF(0), DF(0)}; }

__device__ __forceinline__ float2 ld_row(const float2* p, uint64_t pol) {
  float2 v;
  asm("ld.global.nc.L2::cache_hint.v2.f32 {%0,%1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double2 ld_row(const double2* p, uint64_t pol) {
  double2 v;
  asm("ld.global.nc.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ DF2 ld_row(const DF2* p, uint64_t pol) {
  DF2 v;
  asm("ld.global.nc.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
      : "=f"(v.a.hi), "=f"(v.a.lo), "=f"(v.b.hi), "=f"(v.b.lo)
      : "l"(p), "l"(pol));
  return v;
}

template <typename V>
__device__ __forceinline__ V* carry_of(const SpmmArgs& a, bool head);
template <>
__device__ __forceinline__ float2* carry_of<float2>(const SpmmArgs& a, bool head) {
  return head ? a.carry_head : a.carry_tail;
}
template <>
__device__ __forceinline__ double2* carry_of<double2>(const SpmmArgs& a, bool head) {
  return head ? a.carry_head64 : a.carry_tail64;
}
template <>
__device__ __forceinline__ DF2* carry_of<DF2>(const SpmmArgs& a, bool head) {  // the 16-byte carries
  return reinterpret_cast<DF2*>(head ? a.carry_head64 : a.carry_tail64);
}

// V = float2 (FP32 gathers) or DF2 (float-pair gathers); u is [gathered + 1][S/2] pairs.
// With a.chunk_ctr (FP32 only) each warp takes its first two chunks by a grid-wide stride
// and claims every later one from a counter (the claim for the chunk after next issued when
// a chunk starts, read when it ends); each chunk's gaps go to a.gap_chunk and the fix-up
// adds them in fixed slices, so the sums keep an order fixed by the graph.
template <typename V, typename Epi>
__device__ __forceinline__ void spmm_run(const SpmmArgs& a, const V* __restrict__ u, const Epi& epi) {
  if (*a.done) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  constexpr bool kClaims = std::is_same<V, float2>::value;
  const bool dyn = kClaims && a.chunk_ctr != nullptr;
  const uint64_t pol_s = policy_evict_first();
  const uint64_t pol_k = policy_evict_last();
  const int act[2] = {a.active[2 * lane], a.active[2 * lane + 1]};
  V* ch = carry_of<V>(a, true);
  V* ct = carry_of<V>(a, false);
  double2 gap = make_double2(0.0, 0.0);
  int64_t nxt = warp_id + n_warps;  // the next chunk (known a chunk ahead with claims)
  for (int64_t c = warp_id; c < a.num_chunks;) {
    int32_t claim = a.num_chunks;
    if constexpr (kClaims) {
      if (dyn && lane == 0 && nxt < a.num_chunks) claim = (int32_t)(2 * n_warps) + atomicAdd(a.chunk_ctr, 1);
    }
    const int64_t p0 = c * kSpmmChunk;
    const int64_t p1 = p0 + kSpmmChunk < a.m ? p0 + kSpmmChunk : a.m;
    int32_t r = a.chunk_row[c];
    const bool head_open = (int64_t)a.row_ptr[r] < p0;
    int64_t next_end = a.row_ptr[r + 1];
    typename Epi::Pre pre = epi.pre(r, lane);
    bool first = true;
    V acc = zero2<V>();
    // col is padded to whole chunks with the zero entry, so groups of 8 never run short
    for (int64_t q = p0; q < p1; q += 32) {
      const int my_col = ld_stream(a.col + q + lane, pol_s);
#pragma unroll 1
      for (int i0 = 0; i0 < 32 && q + i0 < p1; i0 += 8) {
        V x[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {  // eight row gathers in flight per lane
          const int j = __shfl_sync(0xffffffffu, my_col, i0 + i);
          x[i] = ld_row(u + (int64_t)j * 32 + lane, pol_k);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          acc = add2(acc, x[i]);
          if (q + i0 + i + 1 == next_end) {  // row r ends at this nonzero (warp-uniform)
            if (first && head_open) ch[c * 32 + lane] = acc;
            else epi.row(r, lane, acc, act, gap, pre);
            first = false;
            acc = zero2<V>();
            ++r;
            next_end = r < a.n_rows ? (int64_t)a.row_ptr[r + 1] : INT64_MAX;
            if (r < a.n_rows) pre = epi.pre(r, lane);
          }
        }
      }
    }
    ct[c * 32 + lane] = acc;  // the part of a row that continues into the next chunk
    if constexpr (kClaims) {
      if (dyn) {
        a.gap_chunk[c * a.S + 2 * lane] = gap.x;
        a.gap_chunk[c * a.S + 2 * lane + 1] = gap.y;
        gap = make_double2(0.0, 0.0);
        const int32_t nn = __shfl_sync(0xffffffffu, claim, 0);
        c = nxt;
        nxt = (nxt < a.num_chunks && nn < a.num_chunks) ? nn : a.num_chunks;
      } else {
        c += n_warps;
      }
    } else {
      (void)claim;
      c += n_warps;
    }
  }
  if (kClaims && dyn && lane == 0) {
    // every claim of this warp is made before it counts itself done; the last warp to finish
    // leaves both counters at zero for the next launch
    __threadfence();
    if (atomicAdd(a.chunk_ctr + 1, 1) == (int32_t)n_warps - 1) {
      atomicExch(a.chunk_ctr, 0);
      atomicExch(a.chunk_ctr + 1, 0);
    }
  }
  a.gap_part[warp_id * a.S + 2 * lane] = gap.x;
  a.gap_part[warp_id * a.S + 2 * lane + 1] = gap.y;
}

// The product with a fixed stride (the 8- and 16-byte sums take the registers they need).
template <typename V, typename Epi>
__global__ void __launch_bounds__(256) k_spmm(SpmmArgs a, const V* __restrict__ u, Epi epi) {
  spmm_run<V, Epi>(a, u, epi);
}

// The FP32 product with chunk claims, held to 64 registers (four blocks per SM).
template <typename Epi>
__global__ void __launch_bounds__(256, 4) k_spmm_claims(SpmmArgs a, const float2* __restrict__ u, Epi epi) {
  spmm_run<float2, Epi>(a, u, epi);
}

// Rows that began in an earlier chunk: y = carries of the chunks in order + head partial.
template <typename V, typename Epi>
__global__ void __launch_bounds__(256) k_spmm_fixup(SpmmArgs a, const int32_t* __restrict__ fix_chunk,
                                                   int32_t num_fix, double* gap_fix, Epi epi) {
  if (*a.done) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int act[2] = {a.active[2 * lane], a.active[2 * lane + 1]};
  const V* ch = carry_of<V>(a, true);
  const V* ct = carry_of<V>(a, false);
  double2 gap = make_double2(0.0, 0.0);
  for (int64_t q = warp_id; q < num_fix; q += n_warps) {
    const int32_t c = fix_chunk[q];
    const int32_t r = a.chunk_row[c];
    const int32_t cs = a.row_ptr[r] / kSpmmChunk;
    V acc = zero2<V>();
#pragma unroll 8
    for (int32_t k = cs; k < c; ++k) acc = add2(acc, ct[(int64_t)k * 32 + lane]);
    acc = add2(acc, ch[(int64_t)c * 32 + lane]);
    epi.row(r, lane, acc, act, gap, epi.pre(r, lane));
  }
  if (a.gap_chunk) {  // this warp's fixed slice of the product's per-chunk gaps, in order
    const int64_t per = (a.num_chunks + n_warps - 1) / n_warps;
    const int64_t c1 = min((int64_t)a.num_chunks, warp_id * per + per);
    for (int64_t c = warp_id * per; c < c1; ++c) {
      gap.x += a.gap_chunk[c * a.S + 2 * lane];
      gap.y += a.gap_chunk[c * a.S + 2 * lane + 1];
    }
  }
  gap_fix[warp_id * a.S + 2 * lane] = gap.x;
  gap_fix[warp_id * a.S + 2 * lane + 1] = gap.y;
}

}  // namespace psi
