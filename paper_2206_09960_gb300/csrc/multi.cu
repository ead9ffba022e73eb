// multi.cu -- many independent follower graphs solved together.
//
// The graphs are joined into one block-diagonal graph (ids offset per graph) and built
// once; the renumbering keeps each graph's users contiguous inside every class, so a
// graph's rows are two ranges (its X users, then its R users).  Each graph keeps its own N
// (psi = (.)/N_g, the psi-tolerance eps/N_g), gap, stop test, step count and FP64
// confirming step, i.e. runs exactly the single-graph schedule (FP32 series of Eq. 13, then
// one FP64 step of Eq. 14 whose gap is tested, Algorithm 2's stop rule):
//   * a graph is in one of three phases: SERIES, CONFIRM (its series met the test; the
//     next FP64 step checks it) or DONE;
//   * every step pair is one series product (rows of SERIES graphs) and one FP64 product
//     (rows of CONFIRM graphs); tiles holding no row of a graph in the product's phase are
//     skipped, so a graph that is waiting or done costs nothing;
//   * the epilogues write one gap entry per row; fixed slices of each graph's rows are summed
//     by their own blocks and one block adds each graph's slice sums in order and moves the
//     graph between phases (bit-reproducible);
//   * the step pairs are captured once into a CUDA graph and replayed until every graph is
//     DONE, with no host work between steps.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <cstring>
#include <vector>

#include "build.cuh"
#include "trace.cuh"
#include "primitives.cuh"
#include "solve.cuh"
#include "spmv.cuh"

namespace psi {

namespace {

#define MGRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

int mgrid(int64_t n) {
  int64_t g = ceil_div(n > 0 ? n : 1, 256);
  int64_t cap = num_sms() * 16;
  return (int)(g < cap ? g : cap);
}

constexpr int32_t kDone = 0, kSeries = 1, kConfirm = 2;
constexpr int kMaxGraphs = 1024;  // group ids take 10 bits of the renumbering key

// Shared loop state.  gate[0].done: no graph in SERIES (series launches exit at once);
// gate[1].done: no graph in CONFIRM; gate[2] stays open (final product).
struct MState {
  int32_t n_series;
  int32_t n_confirm;
  int32_t max_iter;
  int32_t pad0_;
  double eps;
  int32_t all_done;
  int32_t pad_;
};

// Tile -> graphs it touches: rows [r0, r_hi] of a tile cover the graph id range [x, y]
// among X rows and [z, w] among R rows (empty when x > y).  A tile is on when a graph of
// either range is in the product's phase: cnt is the prefix count of such graphs.
struct TileGate {
  const int4* tile_g;
  const int32_t* cnt;  // [G + 1]
  __device__ __forceinline__ bool on(int32_t tile) const {
    const int4 t = tile_g[tile];
    bool any = false;
    if (t.x <= t.y) any = cnt[t.y + 1] - cnt[t.x] > 0;
    if (t.z <= t.w) any = any || cnt[t.w + 1] - cnt[t.z] > 0;
    return any;
  }
};

// ---------------------------------------------------------------- epilogues
// Series step (Eq. 13) for the rows of SERIES graphs: t = mu * y in FP32, s += t in FP64,
// v_new = t / sigma.  Rows of other graphs add nothing and leave their gap entry at 0.
struct EpiSeriesM {
  static constexpr bool kTileSkip = true;
  const float* mu;
  const float* isig;
  double* s64;
  float* v_new;
  int32_t nX;
  const int32_t* gid;
  const int32_t* phase;
  double* gap_row;
  TileGate gate;
  __device__ __forceinline__ bool tile_on(int32_t tile) const { return gate.on(tile); }
  __device__ __forceinline__ void row(int32_t r, float y, double&, uint64_t pol_s, uint64_t pol_k) const {
    const bool on = phase[gid[r]] == kSeries;
    const float t = on ? ld_stream(mu + r, pol_s) * y : 0.f;  // a select: y of an idle row is not used
    if (on) s64[r] += (double)t;
    gap_row[r] = fabs((double)t);
    if (r < nX && on) st_keep(v_new + r, t * ld_stream(isig + r, pol_s), pol_k);
  }
};

// Confirming step (Eq. 14) for the rows of CONFIRM graphs: s_new = c + mu * y, r = s_new - s,
// s = s_new; v_next = r / sigma starts the graph's next series if the test fails.  The
// product sums float pairs or FP64 (G, chosen per solve as in the single-graph path); the
// row update is FP64.
template <typename G>
struct EpiResidM {
  static constexpr bool kTileSkip = true;
  const double* c;
  const double* mu;
  const double* isig;
  double* s64;
  float* v_next;
  int32_t nX;
  const int32_t* gid;
  const int32_t* phase;
  double* gap_row;
  TileGate gate;
  __device__ __forceinline__ bool tile_on(int32_t tile) const { return gate.on(tile); }
  __device__ __forceinline__ void row(int32_t r, G yp, double&, uint64_t pol_s, uint64_t) const {
    if (phase[gid[r]] != kConfirm) {
      gap_row[r] = 0.0;
      return;
    }
    const double y = as_double(yp);
    const double s = s64[r];
    const double sn = ld_stream(c + r, pol_s) + ld_stream(mu + r, pol_s) * y;
    const double rr = sn - s;
    gap_row[r] = fabs(rr);
    s64[r] = sn;
    if (r < nX) v_next[r] = (float)(rr * ld_stream(isig + r, pol_s));
  }
};

// Final step of Algorithm 2 for every graph: psi_r = (lambda_r * G(s)_r + d_r) / N_g.
template <typename G>
struct EpiFinalM {
  const double* lam;
  const double* d;
  double* psi;
  const int32_t* gid;
  const double* n_of;
  __device__ __forceinline__ void row(int32_t r, G y, double&, uint64_t pol_s, uint64_t) const {
    psi[r] = (ld_stream(lam + r, pol_s) * as_double(y) + ld_stream(d + r, pol_s)) / n_of[gid[r]];
  }
};

// ---------------------------------------------------------------- per-graph stop test
// Two kernels per step.  k_group_partial: kGapSlices blocks per graph; block (g, b) sums
// the gap entries of slice b of graph g's rows (its X range, then its R range, cut into
// kGapSlices equal slices) with several loads in flight per thread.  k_group_step: one
// block; thread g adds graph g's slice sums in order, counts the step and moves the graph:
//   series (mode 0): test met (or the next step predicted to meet it) and steps < max_iter
//                    -> CONFIRM; steps >= max_iter -> DONE;
//   FP64   (mode 1): test met -> DONE, converged; steps >= max_iter -> DONE; else SERIES;
// then the block recounts the phases into the prefix counts and the gates.
constexpr int kGapSlices = 8;

__global__ void __launch_bounds__(256) k_group_partial(int mode, const DevState* gate, const int4* __restrict__ ranges,
                                                      const double* __restrict__ gap_row,
                                                      const int32_t* __restrict__ phase, double* part) {
  if (gate[mode].done) return;
  const int g = blockIdx.x / kGapSlices, b = blockIdx.x % kGapSlices;
  if (phase[g] != (mode == 0 ? kSeries : kConfirm)) return;
  __shared__ double sh[256];
  const int4 rg = ranges[g];
  const int64_t nx = rg.y - rg.x, total = nx + (rg.w - rg.z);
  const int64_t lo = total * b / kGapSlices, hi = total * (b + 1) / kGapSlices;
  auto at = [&](int64_t v) { return v < nx ? gap_row[rg.x + v] : gap_row[rg.z + (v - nx)]; };
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int64_t v = lo + threadIdx.x;
  for (; v + 768 < hi; v += 1024) {
    a0 += at(v);
    a1 += at(v + 256);
    a2 += at(v + 512);
    a3 += at(v + 768);
  }
  for (; v < hi; v += 256) a0 += at(v);
  sh[threadIdx.x] = (a0 + a1) + (a2 + a3);
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(1024) k_group_step(int mode, MState* st, DevState* gate,
                                                    const double* __restrict__ part, int32_t* phase, int32_t* iters,
                                                    int32_t* phase_it, int32_t* converged, int32_t* refinements,
                                                    double* gap_last,
                                                    const double* __restrict__ scale, int32_t* cnt_series,
                                                    int32_t* cnt_confirm, int G) {
  if (gate[mode].done) return;
  __shared__ int32_t ws[2][32];
  const int g = threadIdx.x;
  int32_t p = kDone;
  if (g < G) {
    p = phase[g];
    if (p == (mode == 0 ? kSeries : kConfirm)) {
      double gap = 0.0;
      for (int b = 0; b < kGapSlices; ++b) gap += part[g * kGapSlices + b];
      const double prev = gap_last[g];
      gap_last[g] = gap;
      const int32_t it = iters[g] + 1;
      iters[g] = it;
      const double scaled = gap * scale[g];
      const bool met = scaled <= st->eps;
      if (mode == 0) {
        // as in the single-graph path: a series also stops one step early when the next gap,
        // predicted from the last two with a 1.2x margin, meets the test
        const int32_t pit = phase_it[g] + 1;
        phase_it[g] = pit;
        const bool next_passes = pit >= 2 && gap < prev && 1.2 * (gap / prev) * scaled <= st->eps;
        p = ((met || next_passes) && it < st->max_iter) ? kConfirm : (it >= st->max_iter ? kDone : kSeries);
      } else {
        refinements[g] += 1;
        if (met) converged[g] = 1;
        p = met || it >= st->max_iter ? kDone : kSeries;
        if (p == kSeries) phase_it[g] = 0;  // a new series starts from the residual
      }
      phase[g] = p;
    }
  }
  // exclusive prefix counts of the new phases over the graphs, block-wide
  const int32_t a = p == kSeries, c = p == kConfirm;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t ia = a, ic = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t ua = __shfl_up_sync(0xffffffffu, ia, o), uc = __shfl_up_sync(0xffffffffu, ic, o);
    if (lane >= o) {
      ia += ua;
      ic += uc;
    }
  }
  if (lane == 31) {
    ws[0][warp] = ia;
    ws[1][warp] = ic;
  }
  __syncthreads();
  int32_t oa = 0, oc = 0;
  for (int w = 0; w < warp; ++w) {
    oa += ws[0][w];
    oc += ws[1][w];
  }
  if (g < G) {
    cnt_series[g] = oa + ia - a;
    cnt_confirm[g] = oc + ic - c;
  }
  if (g == (int)blockDim.x - 1) {
    const int32_t ns = oa + ia, nc = oc + ic;
    cnt_series[G] = ns;
    cnt_confirm[G] = nc;
    st->n_series = ns;
    st->n_confirm = nc;
    st->all_done = (ns == 0 && nc == 0) ? 1 : 0;
    gate[0].done = ns == 0 ? 1 : 0;
    gate[1].done = nc == 0 ? 1 : 0;
  }
}

// Gathered vector of the CONFIRM graphs' X users: u = s / sigma (other graphs' entries are
// read only by their own rows, which ignore them in this step).  kGapSlices blocks per
// graph over its X range; blocks of graphs in another phase return at once.
template <typename G>
__global__ void __launch_bounds__(256) k_confirm_u(const DevState* gate, const double* __restrict__ s64,
                                                  const double* __restrict__ isig, const int4* __restrict__ ranges,
                                                  const int32_t* __restrict__ phase, G* u) {
  if (gate[1].done) return;
  const int g = blockIdx.x / kGapSlices, b = blockIdx.x % kGapSlices;
  if (phase[g] != kConfirm) return;
  const int4 rg = ranges[g];
  const int64_t nx = rg.y - rg.x;
  const int64_t lo = rg.x + nx * b / kGapSlices, hi = rg.x + nx * (b + 1) / kGapSlices;
  for (int64_t j = lo + threadIdx.x; j < hi; j += blockDim.x) u[j] = to_gather<G>(s64[j] * isig[j]);
}

// gathered vector of the confirming / final products: dst[j] = s[user(j)] * isig[user(j)]
template <typename G>
__global__ void k_to_gathered_g(G* dst, const double* __restrict__ s, const double* __restrict__ isig, int32_t nX,
                                int32_t nR, int64_t lo, int64_t hi) {
  MGRID_STRIDE(i, hi - lo) {
    const int64_t j = lo + i;
    const int64_t user = j < nX ? j : j + nR;
    dst[j] = to_gather<G>(s[user] * isig[user]);
  }
}

// ---------------------------------------------------------------- setup kernels
// graph holding element e of a concatenation with offsets off[0..G] (largest g, off[g] <= e)
__device__ __forceinline__ int owner_of(const int64_t* __restrict__ off, int G, int64_t e) {
  int lo = 0, hi = G - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// union ids from per-graph local ids; an id outside its graph's [0, N_g) is reported
__global__ void k_union_edges(const int32_t* __restrict__ f, const int32_t* __restrict__ l, int64_t m,
                              const int64_t* __restrict__ moff, const int64_t* __restrict__ noff, int G, int32_t* uf,
                              int32_t* ul, uint32_t* bad) {
  uint32_t b = 0;
  MGRID_STRIDE(e, m) {
    const int g = owner_of(moff, G, e);
    const int64_t ng = noff[g + 1] - noff[g];
    const int32_t a = f[e], c = l[e];
    if (a < 0 || a >= ng || c < 0 || c >= ng) {
      b = 1;
      uf[e] = ul[e] = 0;
    } else {
      uf[e] = (int32_t)(noff[g] + a);
      ul[e] = (int32_t)(noff[g] + c);
    }
  }
  if (b) atomicOr(bad, 1u);
}

__global__ void k_user_groups(const int64_t* __restrict__ noff, int G, int64_t n, int32_t* group) {
  MGRID_STRIDE(i, n) group[i] = owner_of(noff, G, i);
}

// graph id of every internal user
__global__ void k_internal_groups(const int32_t* __restrict__ group_in, const int32_t* __restrict__ perm, int64_t n,
                                  int32_t* gid) {
  MGRID_STRIDE(k, n) gid[k] = group_in[perm[k]];
}

// ranges[g] = {X begin, X end, R begin, R end}: gid is non-decreasing inside each class
__global__ void k_group_ranges(const int32_t* __restrict__ gid, int32_t nX, int32_t n_rows, int4* ranges) {
  MGRID_STRIDE(r, n_rows) {
    const int g = gid[r];
    const bool in_x = r < nX;
    const int64_t lo = in_x ? 0 : nX, hi = in_x ? nX : n_rows;
    if (r == lo || gid[r - 1] != g) {
      if (in_x) ranges[g].x = (int)r; else ranges[g].z = (int)r;
    }
    if (r + 1 == hi || gid[r + 1] != g) {
      if (in_x) ranges[g].y = (int)r + 1; else ranges[g].w = (int)r + 1;
    }
  }
}

// graph id ranges of the rows [tile_row[t], tile_row[t + 1]] of every tile
__global__ void k_tile_groups(const int32_t* __restrict__ tile_row, int32_t tiles, const int32_t* __restrict__ gid,
                              int32_t nX, int4* tile_g) {
  MGRID_STRIDE(t, tiles) {
    const int32_t r0 = tile_row[t], r1 = tile_row[t + 1];
    int4 o = make_int4(0, -1, 0, -1);
    if (r0 < nX) o.x = gid[r0], o.y = gid[r1 < nX ? r1 : nX - 1];
    if (r1 >= nX) o.z = gid[r0 >= nX ? r0 : nX], o.w = gid[r1];
    tile_g[t] = o;
  }
}

// ||B||_inf of each graph: max over its users with leaders of beta_j / sigma_j
__global__ void k_group_bnorm(const double* __restrict__ sigma, const double* __restrict__ beta,
                              const int32_t* __restrict__ group_in, const int32_t* __restrict__ perm, int64_t n,
                              unsigned long long* bits) {
  MGRID_STRIDE(k, n) {
    const double sg = sigma[k];
    if (sg > 0.0) {
      const double b = beta[k] / sg;  // non-negative doubles order like their bit patterns
      atomicMax(bits + group_in[perm[k]], (unsigned long long)__double_as_longlong(b));
    }
  }
}

// gathered index space: X at [0, nX), U at [nX, nX + nU) (user j + nR)
template <typename T>
__global__ void k_to_gathered(T* dst, const T* __restrict__ s, const T* __restrict__ isig, int32_t nX, int32_t nR,
                              int64_t lo, int64_t hi) {
  MGRID_STRIDE(i, hi - lo) {
    const int64_t j = lo + i;
    const int64_t user = j < nX ? j : j + nR;
    dst[j] = s[user] * isig[user];
  }
}

template <typename T>
__global__ void k_fill_m(T* x, int64_t n, T v) {
  MGRID_STRIDE(i, n) x[i] = v;
}

__global__ void k_psi_nonrow_m(double* psi, const double* __restrict__ d, const int32_t* __restrict__ gid,
                               const double* __restrict__ n_of, int64_t lo, int64_t n) {
  MGRID_STRIDE(i, n - lo) {
    const int64_t k = lo + i;
    psi[k] = d[k] / n_of[gid[k]];
  }
}

__global__ void k_scatter_m(const double* __restrict__ in, const int32_t* __restrict__ perm, int64_t n, double* out) {
  MGRID_STRIDE(k, n) out[perm[k]] = in[k];
}

// one block per graph: sum of psi over its users (input order, contiguous), fixed order
__global__ void __launch_bounds__(256) k_group_sums(const double* __restrict__ x, const int64_t* __restrict__ noff,
                                                   double* out) {
  __shared__ double sh[256];
  const int g = blockIdx.x;
  double acc = 0.0;
  for (int64_t i = noff[g] + threadIdx.x; i < noff[g + 1]; i += blockDim.x) acc += x[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[g] = sh[0];
}

}  // namespace

// ------------------------------------------------------------------ the multi-graph object
struct Multi {
  Graph g;  // the block-diagonal union
  int G = 0;
  std::vector<int64_t> h_noff;         // [G + 1] user offsets of the graphs (input order)
  DBuf<int64_t> noff;
  DBuf<double> n_of, scale, bnorm;     // [G]
  DBuf<int32_t> gid;                   // [n] graph of every internal user
  DBuf<int4> ranges;                   // [G] row ranges
  DBuf<int4> tile_g;                   // [tiles] graph ranges of the tiles
  // loop state
  DBuf<int32_t> phase, iters, phase_it, converged, refinements, cnt_series, cnt_confirm;
  DBuf<double> gap_last;
  DBuf<double> gap_part;               // [G][kGapSlices] slice sums of the per-row gaps
  DBuf<MState> st;
  DBuf<DevState> gate;                 // [3]
  MState* host = nullptr;              // pinned, 2 slots
  // vectors
  DBuf<double> s64, u64, gap_row, psi, psi_sum;  // u64 holds float pairs (8 bytes per entry)
  template <typename G>
  G* u64as() const {
    return reinterpret_cast<G*>(u64.get());
  }
  DBuf<float> v0, va, vb;
  // graph-build scratch of the hook
  DBuf<unsigned long long> bnorm_bits;
  // captured step pairs
  cudaGraphExec_t exec[2] = {nullptr, nullptr};  // captured step pairs: [0] FP64, [1] float-pair products
  int pairs_per_replay = 4;
  int launches_per_replay[2] = {0, 0};
  bool solved = false;
  bool tile_fixed = false;  // psi_options.spmv_tile chose the tile
  bool tuned = false;
};

// Per-graph ||B||_inf from the build's sigma and beta.
struct MultiHook final : BuildHook {
  Multi& mg;
  const int32_t* group_in;
  MultiHook(Multi& m, const int32_t* gr) : mg(m), group_in(gr) {}
  const int32_t* user_group() const override { return group_in; }
  void on_leader_sums(Graph& g, const double* sigma, const double* beta) override {
    const int64_t n = g.n;
    k_group_bnorm<<<mgrid(n), 256, 0, g.stream>>>(sigma, beta, group_in, g.perm.get(), n, mg.bnorm_bits.get());
    PSI_LAUNCHED();
  }
};

namespace {

// Per-graph top k in one launch: one block per graph selects, over the graph's psi values
// (input order), the k largest of the 96-bit keys (bits(psi) << 32 | ~local id), i.e. the
// ranking by psi descending, then local id ascending.  MSB-first radix select (8-bit digits),
// then the k keys above the threshold are gathered and ranked by counting.
constexpr int kMultiTopkMax = 1024;

__device__ __forceinline__ void topk_key(const double* psi, int64_t i, int64_t base, uint64_t& hi, uint32_t& lo) {
  hi = (uint64_t)__double_as_longlong(psi[i]);  // psi >= 0: bit patterns order like the values
  lo = ~(uint32_t)(i - base);
}

__global__ void __launch_bounds__(256) k_multi_topk(const double* __restrict__ psi, const int64_t* __restrict__ noff,
                                                   int32_t k, int32_t* ids, double* vals) {
  __shared__ uint32_t hist[256];
  __shared__ uint64_t p_hi;
  __shared__ uint32_t p_lo;
  __shared__ int32_t k_rem, level_end, n_cand;
  __shared__ uint64_t c_hi[kMultiTopkMax];
  __shared__ uint32_t c_lo[kMultiTopkMax];
  const int g = blockIdx.x;
  const int64_t b0 = noff[g], b1 = noff[g + 1];
  if (threadIdx.x == 0) {
    p_hi = 0;
    p_lo = 0;
    k_rem = k;
    level_end = 12;
    n_cand = 0;
  }
  __syncthreads();
  for (int level = 0; level < 12; ++level) {
    if (level >= level_end) break;  // uniform (shared, written before the barrier)
    hist[threadIdx.x] = 0;
    __syncthreads();
    // the top `level` digits must equal the prefix
    const int done_bits = level * 8;
    const uint64_t m_hi = done_bits >= 64 ? ~0ull : (done_bits == 0 ? 0ull : ~0ull << (64 - done_bits));
    const uint32_t m_lo = done_bits <= 64 ? 0u : ~0u << (96 - done_bits);
    const uint64_t ph = p_hi;
    const uint32_t pl = p_lo;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
      uint64_t hi;
      uint32_t lo;
      topk_key(psi, i, b0, hi, lo);
      if ((hi & m_hi) != ph || (lo & m_lo) != pl) continue;
      const uint32_t d = level < 8 ? (uint32_t)(hi >> (56 - 8 * level)) & 255u : (lo >> (24 - 8 * (level - 8))) & 255u;
      atomicAdd(&hist[d], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t above = 0;
      int b = 255;
      for (; b > 0; --b) {
        if (above + (int32_t)hist[b] >= k_rem) break;
        above += (int32_t)hist[b];
      }
      k_rem -= above;
      if (level < 8) p_hi |= (uint64_t)b << (56 - 8 * level);
      else p_lo |= (uint32_t)b << (24 - 8 * (level - 8));
      if ((int32_t)hist[b] == k_rem) level_end = level + 1;  // the whole bin is taken
    }
    __syncthreads();
  }
  // keys >= the threshold (the prefix followed by zeros): exactly k of them
  const uint64_t th = p_hi;
  const uint32_t tl = p_lo;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    uint64_t hi;
    uint32_t lo;
    topk_key(psi, i, b0, hi, lo);
    if (hi > th || (hi == th && lo >= tl)) {
      const int32_t q = atomicAdd(&n_cand, 1);
      if (q < kMultiTopkMax) {
        c_hi[q] = hi;
        c_lo[q] = lo;
      }
    }
  }
  __syncthreads();
  const int32_t nc = n_cand < k ? n_cand : k;
  for (int32_t q = threadIdx.x; q < nc; q += blockDim.x) {
    const uint64_t h = c_hi[q];
    const uint32_t l = c_lo[q];
    int32_t rank = 0;
    for (int32_t j = 0; j < nc; ++j) rank += (c_hi[j] > h || (c_hi[j] == h && c_lo[j] > l)) ? 1 : 0;
    ids[(int64_t)g * k + rank] = (int32_t)~l;
    vals[(int64_t)g * k + rank] = __longlong_as_double((long long)h);
  }
}

void multi_buffers(Multi& M) {
  Graph& g = M.g;
  Allocator& al = g.al;
  const size_t n = (size_t)g.n;
  const size_t nu = (size_t)g.nX + (size_t)g.nU;
  const size_t G = (size_t)M.G;
  M.phase.reset(al, G);
  M.iters.reset(al, G);
  M.phase_it.reset(al, G);
  M.converged.reset(al, G);
  M.refinements.reset(al, G);
  M.cnt_series.reset(al, G + 1);
  M.cnt_confirm.reset(al, G + 1);
  M.gap_last.reset(al, G);
  M.gap_part.reset(al, G * kGapSlices);
  M.st.reset(al, 1);
  M.gate.reset(al, 3);
  if (!M.host) PSI_CUDA(cudaMallocHost((void**)&M.host, 2 * sizeof(MState)));
  M.s64.reset(al, n);
  M.u64.reset(al, nu + 1);
  M.gap_row.reset(al, (size_t)(g.n_rows > 0 ? g.n_rows : 1));
  M.psi.reset(al, n);
  M.psi_sum.reset(al, G);
  M.v0.reset(al, nu + 1);
  M.va.reset(al, nu + 1);
  M.vb.reset(al, nu + 1);
  const size_t nt = (size_t)(g.num_tiles > 0 ? g.num_tiles : 1);
  g.carry_head.reset(al, nt);
  g.carry_tail.reset(al, nt);
  g.gap_part.reset(al, (size_t)num_sms() * 32);
  g.gap_fix.reset(al, (size_t)num_sms() * 8);
}

template <typename T, typename Epi>
int multi_spmv_grid(int tiles) {
  static const int per_sm = [] {  // once, thread-safe
    int b = 0;
    PSI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_spmv<T, Epi>, kSpmvThreads, 0));
    return b > 0 ? b : 1;
  }();
  return spmv_blocks(per_sm, tiles);
}

// product + fix-up of one step, skipped on the device when gate->done
template <typename T, typename Epi>
int multi_product(Multi& M, cudaStream_t s, const T* u, const Epi& epi, const DevState* gate) {
  Graph& g = M.g;
  int launches = 0;
  if (g.num_tiles > 0) {
    SpmvArgs a{};
    a.row_ptr = g.row_ptr.get();
    a.col = g.col.get();
    a.tile_row = g.tile_row.get();
    a.tile = g.tile;
    a.num_tiles = g.num_tiles;
    a.n_rows = g.n_rows;
    a.m = g.m_unique;
    a.state = gate;
    a.gap_part = g.gap_part.get();
    a.carry_head = g.carry_head.get();
    a.carry_tail = g.carry_tail.get();
    k_spmv<T, Epi><<<multi_spmv_grid<T, Epi>(g.num_tiles), kSpmvThreads, 0, s>>>(a, u, epi);
    PSI_LAUNCHED();
    ++launches;
  }
  if (g.num_fix > 0) {
    FixArgs f{};
    f.row_ptr = g.row_ptr.get();
    f.tile_row = g.tile_row.get();
    f.tile = g.tile;
    f.fix_tile = g.fix_tile.get();
    f.num_fix = g.num_fix;
    f.state = gate;
    f.gap_fix = g.gap_fix.get();
    f.carry_head = g.carry_head.get();
    f.carry_tail = g.carry_tail.get();
    int fgrid = fix_blocks(g.num_fix);
    k_fixup<T, Epi><<<fgrid, kFixThreads, 0, s>>>(f, epi);
    PSI_LAUNCHED();
    ++launches;
  }
  return launches;
}

int group_step(Multi& M, cudaStream_t s, int mode) {
  k_group_partial<<<M.G * kGapSlices, 256, 0, s>>>(mode, M.gate.get(), M.ranges.get(), M.gap_row.get(), M.phase.get(),
                                                   M.gap_part.get());
  PSI_LAUNCHED();
  // gate[mode] is read before any thread writes a gate (only the last thread does, after
  // the block's barrier), and all threads of the block see the same value
  k_group_step<<<1, 1024, 0, s>>>(mode, M.st.get(), M.gate.get(), M.gap_part.get(), M.phase.get(), M.iters.get(),
                                  M.phase_it.get(), M.converged.get(), M.refinements.get(), M.gap_last.get(),
                                  M.scale.get(),
                                  M.cnt_series.get(), M.cnt_confirm.get(), M.G);
  PSI_LAUNCHED();
  return 2;
}

// One step pair: a series step of the SERIES graphs reading v_in and writing v_out, their
// stop tests, then the FP64 step of the CONFIRM graphs (whose residual, if the test fails,
// is written to v_out for the next series step) and their tests.  Returns the launches.
template <typename G>
int step_pair(Multi& M, cudaStream_t s, const float* v_in, float* v_out) {
  Graph& g = M.g;
  int launches = 0;
  EpiSeriesM es{g.mu32.get(), g.isig32.get(), M.s64.get(), v_out, g.nX, M.gid.get(), M.phase.get(), M.gap_row.get(),
                TileGate{M.tile_g.get(), M.cnt_series.get()}};
  launches += multi_product<float>(M, s, v_in, es, M.gate.get() + 0);
  launches += group_step(M, s, 0);
  k_confirm_u<G><<<M.G * kGapSlices, 256, 0, s>>>(M.gate.get(), M.s64.get(), g.isig64.get(), M.ranges.get(),
                                                  M.phase.get(), M.u64as<G>());
  PSI_LAUNCHED();
  ++launches;
  EpiResidM<G> er{g.c64.get(), g.mu64.get(), g.isig64.get(), M.s64.get(), v_out, g.nX, M.gid.get(), M.phase.get(),
               M.gap_row.get(), TileGate{M.tile_g.get(), M.cnt_confirm.get()}};
  launches += multi_product<G>(M, s, M.u64as<G>(), er, M.gate.get() + 1);
  launches += group_step(M, s, 1);
  return launches;
}

template <typename T>
void read_vec_m(std::vector<T>& h, const T* d, size_t k, cudaStream_t s) {
  h.resize(k);
  PSI_CUDA(cudaMemcpyAsync(h.data(), d, sizeof(T) * k, cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaStreamSynchronize(s));
}

// Captures pairs_per_replay step pairs (an even number: buffers alternate va -> vb -> va)
// into a CUDA graph on a private stream.  Kernel arguments are device pointers only, so the
// graph serves every later solve of the object.
template <typename G>
int capture_pairs(Multi& M, cudaGraphExec_t* exec) {
  cudaStream_t cs = nullptr;
  PSI_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  int launches = 0;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    throw_cuda(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
  }
  try {
    for (int p = 0; p < M.pairs_per_replay; ++p) {
      float* in = (p & 1) ? M.va.get() : M.vb.get();
      float* out = (p & 1) ? M.vb.get() : M.va.get();
      launches += step_pair<G>(M, cs, in, out);
    }
  } catch (...) {
    cudaStreamEndCapture(cs, &graph);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    cudaGetLastError();
    throw;
  }
  e = cudaStreamEndCapture(cs, &graph);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) throw_cuda(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) throw_cuda(e, "cudaGraphInstantiate", __FILE__, __LINE__);
  return launches;
}

}  // namespace

psi_status multi_solve_once(Multi& M, double eps, int32_t max_iter, psi_solve_info* info) {
  NvtxRange nvtx_range("psi_multi_solve");
  PSI_REQUIRE(max_iter >= 0 && !std::isnan(eps), PSI_ERR_INVALID_ARG, "bad eps or max_iter");
  Graph& g = M.g;
  cudaStream_t s = g.stream;
  const int64_t n = g.n;
  const int32_t nX = g.nX, nR = g.nR;
  const int64_t nu = (int64_t)g.nX + g.nU;
  const int G = M.G;
  M.solved = false;
  // float pairs in the confirming and final products when every graph's tolerance is far
  // above their rounding (as in the single-graph path), FP64 otherwise
  bool pairs = true;
  {
    std::vector<double> sc;
    read_vec_m(sc, M.scale.get(), (size_t)G, s);
    for (int q = 0; q < G; ++q)
      pairs = pairs && eps / sc[q] >= std::ldexp(1.0, -30) * (double)(M.h_noff[q + 1] - M.h_noff[q]);
  }
  const int variant = pairs ? 1 : 0;
  auto to_gathered = [&](const double* src, int64_t lo, int64_t hi) {
    if (hi <= lo) return;
    if (pairs) k_to_gathered_g<DF><<<mgrid(hi - lo), 256, 0, s>>>(M.u64as<DF>(), src, g.isig64.get(), nX, nR, lo, hi);
    else k_to_gathered_g<double><<<mgrid(hi - lo), 256, 0, s>>>(M.u64as<double>(), src, g.isig64.get(), nX, nR, lo, hi);
    PSI_LAUNCHED();
  };
  cudaEvent_t t0, t1;
  PSI_CUDA(cudaEventCreate(&t0));
  PSI_CUDA(cudaEventCreate(&t1));
  PSI_CUDA(cudaEventRecord(t0, s));
  // s_0 = c; the first series term c / sigma on X and U; later terms vanish on U; the FP64
  // gathered vector holds c / sigma on U throughout
  PSI_CUDA(cudaMemcpyAsync(M.s64.get(), g.c64.get(), sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  k_fill_m<float><<<mgrid(nu + 1), 256, 0, s>>>(M.v0.get(), nu + 1, 0.f);
  PSI_LAUNCHED();
  k_fill_m<float><<<mgrid(nu + 1), 256, 0, s>>>(M.va.get(), nu + 1, 0.f);
  PSI_LAUNCHED();
  k_fill_m<float><<<mgrid(nu + 1), 256, 0, s>>>(M.vb.get(), nu + 1, 0.f);
  PSI_LAUNCHED();
  k_fill_m<double><<<mgrid(nu + 1), 256, 0, s>>>(M.u64.get(), nu + 1, 0.0);
  PSI_LAUNCHED();
  if (nu > 0) {
    k_to_gathered<float><<<mgrid(nu), 256, 0, s>>>(M.v0.get(), g.c32.get(), g.isig32.get(), nX, nR, 0, nu);
    PSI_LAUNCHED();
  }
  if (g.nU > 0) to_gathered(g.c64.get(), nX, nu);
  const bool iterate = (1.0 > eps) && max_iter > 0;  // Algorithm 2's loop test with gap = 1
  {
    // every graph starts in SERIES; prefix counts and gates to match
    std::vector<int32_t> ph((size_t)G, iterate ? kSeries : kDone), cs((size_t)G + 1), cc((size_t)G + 1, 0);
    for (int q = 0; q <= G; ++q) cs[q] = iterate ? q : 0;
    PSI_CUDA(cudaMemcpyAsync(M.phase.get(), ph.data(), sizeof(int32_t) * G, cudaMemcpyHostToDevice, s));
    PSI_CUDA(cudaMemcpyAsync(M.cnt_series.get(), cs.data(), sizeof(int32_t) * (G + 1), cudaMemcpyHostToDevice, s));
    PSI_CUDA(cudaMemcpyAsync(M.cnt_confirm.get(), cc.data(), sizeof(int32_t) * (G + 1), cudaMemcpyHostToDevice, s));
    PSI_CUDA(cudaMemsetAsync(M.iters.get(), 0, sizeof(int32_t) * G, s));
    PSI_CUDA(cudaMemsetAsync(M.phase_it.get(), 0, sizeof(int32_t) * G, s));
    PSI_CUDA(cudaMemsetAsync(M.converged.get(), 0, sizeof(int32_t) * G, s));
    PSI_CUDA(cudaMemsetAsync(M.refinements.get(), 0, sizeof(int32_t) * G, s));
    PSI_CUDA(cudaMemsetAsync(M.gap_last.get(), 0, sizeof(double) * G, s));
    MState h{};
    h.n_series = iterate ? G : 0;
    h.max_iter = max_iter;
    h.eps = eps;
    h.all_done = iterate ? 0 : 1;
    M.host[0] = h;
    PSI_CUDA(cudaMemcpyAsync(M.st.get(), M.host, sizeof(MState), cudaMemcpyHostToDevice, s));
    DevState gt[3]{};
    gt[0].done = iterate ? 0 : 1;
    gt[1].done = 1;
    gt[2].done = 0;
    PSI_CUDA(cudaMemcpyAsync(M.gate.get(), gt, sizeof(gt), cudaMemcpyHostToDevice, s));
    PSI_CUDA(cudaStreamSynchronize(s));  // host staging above lives on this stack frame
  }
  if (iterate) {
    // first pair from v0 (plain launches), then replays of the captured pairs
    if (pairs) step_pair<DF>(M, s, M.v0.get(), M.vb.get());
    else step_pair<double>(M, s, M.v0.get(), M.vb.get());
    if (!M.exec[variant]) {
      M.launches_per_replay[variant] =
          pairs ? capture_pairs<DF>(M, &M.exec[variant]) : capture_pairs<double>(M, &M.exec[variant]);
      count_launches(-M.launches_per_replay[variant]);  // captured, not run
    }
    // every pair advances each graph that is not DONE by one step, so max_iter pairs end
    // the loop; the bound below only guards against a broken state
    const int64_t max_replays = (int64_t)max_iter / M.pairs_per_replay + 3;
    const int per_replay = M.launches_per_replay[variant];
    cudaEvent_t evs[2];
    PSI_CUDA(cudaEventCreateWithFlags(&evs[0], cudaEventDisableTiming));
    PSI_CUDA(cudaEventCreateWithFlags(&evs[1], cudaEventDisableTiming));
    auto replay = [&](int slot) {
      PSI_CUDA(cudaGraphLaunch(M.exec[variant], s));
      for (int q = 0; q < per_replay; ++q) count_launch();
      PSI_CUDA(cudaMemcpyAsync(M.host + slot, M.st.get(), sizeof(MState), cudaMemcpyDeviceToHost, s));
      PSI_CUDA(cudaEventRecord(evs[slot], s));
    };
    replay(0);
    int64_t r = 1;
    bool finished = false;
    for (; r < max_replays + 1; ++r) {
      replay((int)(r & 1));
      PSI_CUDA(cudaEventSynchronize(evs[(r - 1) & 1]));
      if (M.host[(r - 1) & 1].all_done) {
        finished = true;
        break;
      }
    }
    PSI_CUDA(cudaEventSynchronize(evs[r & 1]));
    cudaEventDestroy(evs[0]);
    cudaEventDestroy(evs[1]);
    PSI_REQUIRE(finished || M.host[r & 1].all_done, PSI_ERR_CUDA, "internal: the step loop did not finish");
  }
  // final step of Algorithm 2 for every graph: psi = (s B + d) / N_g, one more product
  if (nX > 0) to_gathered(M.s64.get(), 0, nX);
  if (pairs) {
    EpiFinalM<DF> ef{g.lam64.get(), g.d64.get(), M.psi.get(), M.gid.get(), M.n_of.get()};
    multi_product<DF>(M, s, M.u64as<DF>(), ef, M.gate.get() + 2);
  } else {
    EpiFinalM<double> ef{g.lam64.get(), g.d64.get(), M.psi.get(), M.gid.get(), M.n_of.get()};
    multi_product<double>(M, s, M.u64as<double>(), ef, M.gate.get() + 2);
  }
  if (g.n_rows < n) {
    k_psi_nonrow_m<<<mgrid(n - g.n_rows), 256, 0, s>>>(M.psi.get(), g.d64.get(), M.gid.get(), M.n_of.get(), g.n_rows, n);
    PSI_LAUNCHED();
  }
  // psi in input order (graphs contiguous) and per-graph sums
  DBuf<double> psi_in(g.al, (size_t)n);
  k_scatter_m<<<mgrid(n), 256, 0, s>>>(M.psi.get(), g.perm.get(), n, psi_in.get());
  PSI_LAUNCHED();
  k_group_sums<<<G, 256, 0, s>>>(psi_in.get(), M.noff.get(), M.psi_sum.get());
  PSI_LAUNCHED();
  PSI_CUDA(cudaEventRecord(t1, s));
  std::swap(M.psi.ptr, psi_in.ptr);  // keep psi in input order
  std::vector<int32_t> it, cv, rf;
  std::vector<double> gp, ps, bn, sc;
  read_vec_m(it, M.iters.get(), (size_t)G, s);
  read_vec_m(cv, M.converged.get(), (size_t)G, s);
  read_vec_m(rf, M.refinements.get(), (size_t)G, s);
  read_vec_m(gp, M.gap_last.get(), (size_t)G, s);
  read_vec_m(ps, M.psi_sum.get(), (size_t)G, s);
  read_vec_m(bn, M.bnorm.get(), (size_t)G, s);
  read_vec_m(sc, M.scale.get(), (size_t)G, s);
  float ms = 0.f;
  PSI_CUDA(cudaEventElapsedTime(&ms, t0, t1));
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  M.solved = true;
  bool all_conv = true;
  for (int q = 0; q < G; ++q) {
    const int32_t conv = iterate ? cv[q] : 1;
    all_conv = all_conv && conv;
    if (info) {
      psi_solve_info& o = info[q];
      std::memset(&o, 0, sizeof(o));
      const double nq = (double)(M.h_noff[q + 1] - M.h_noff[q]);
      o.iters = it[q];
      o.converged = conv;
      o.refinements = rf[q];
      o.spmv_launches = it[q] + 1;
      o.gap_s_l1 = gp[q];
      o.gap_scaled = gp[q] * sc[q];
      o.gap_psi_bound = gp[q] * bn[q] / nq;
      o.psi_sum = ps[q];
      o.ms = ms;
    }
  }
  return all_conv ? PSI_OK : PSI_ERR_NOT_CONVERGED;
}

// Cuts the union's nonzeros into tiles of `tile` (schedule, carries, the graph ranges of
// every tile) and drops the captured step pairs, which hold the old schedule.
void multi_retile(Multi& M, int32_t tile) {
  Graph& g = M.g;
  cudaStream_t s = g.stream;
  PSI_CUDA(cudaStreamSynchronize(s));
  for (auto& e : M.exec) {
    if (e) cudaGraphExecDestroy(e);
    e = nullptr;
  }
  Schedule sc = make_schedule(g.row_ptr.get(), g.n_rows, g.m_unique, g.al, s, tile);
  g.tile = sc.tile;
  g.num_tiles = sc.tiles;
  g.num_fix = sc.num_fix;
  g.tile_row = std::move(sc.tile_row);
  g.fix_tile = std::move(sc.fix_tile);
  const size_t nt = (size_t)(g.num_tiles > 0 ? g.num_tiles : 1);
  g.carry_head.reset(g.al, nt);
  g.carry_tail.reset(g.al, nt);
  M.tile_g.reset(g.al, nt);
  if (g.num_tiles > 0) {
    k_tile_groups<<<mgrid(g.num_tiles), 256, 0, s>>>(g.tile_row.get(), g.num_tiles, M.gid.get(), g.nX, M.tile_g.get());
    PSI_LAUNCHED();
  }
}

// The autotuner of the independent-graph object: its product has one free parameter, the
// tile, and how well a tile fits depends on how the graphs stop one after another (a
// stopped graph's tiles are skipped), so each candidate is timed on a whole solve of the
// object (the first solve's eps and step cap), and the fastest is kept for this object and
// remembered for objects of the same sizes.
std::mutex g_mtune_mu;
std::map<std::tuple<int32_t, int64_t, int64_t>, int32_t> g_mtune_cache;

void multi_autotune(Multi& M, double eps, int32_t max_iter) {
  Graph& g = M.g;
  M.tuned = true;
  if (!g.opt.autotune || M.tile_fixed || g.m_unique < ((int64_t)1 << 22)) return;
  const auto key = std::make_tuple((int32_t)M.G, (int64_t)g.n, (int64_t)g.m_unique);
  int32_t pick = 0;
  {
    std::lock_guard<std::mutex> lock(g_mtune_mu);
    auto it = g_mtune_cache.find(key);
    if (it != g_mtune_cache.end()) pick = it->second;
  }
  if (pick == 0) {
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<psi_solve_info> inf((size_t)M.G);
    double best = 0.0;
    for (int32_t tile : {kSpmvTileMin, 2 * kSpmvTileMin, kSpmvTileMax}) {
      if (tile != g.tile) multi_retile(M, tile);
      multi_solve_once(M, eps, max_iter, inf.data());
      if (pick == 0 || inf[0].ms < best) {
        best = inf[0].ms;
        pick = tile;
      }
    }
    g.tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    std::lock_guard<std::mutex> lock(g_mtune_mu);
    g_mtune_cache[key] = pick;
  }
  if (pick != g.tile) multi_retile(M, pick);
}

psi_status multi_solve(Multi& M, double eps, int32_t max_iter, psi_solve_info* info) {
  if (!M.tuned) multi_autotune(M, eps, max_iter);
  return multi_solve_once(M, eps, max_iter, info);
}

}  // namespace psi

namespace psi {
namespace {

template <typename F>
psi_status multi_guard(F&& f) {
  try {
    f();
    return PSI_OK;
  } catch (const PsiError& e) {
    set_last_error(e.what());
    return e.status;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return PSI_ERR_CUDA;
  } catch (...) {
    set_last_error("unknown failure");
    return PSI_ERR_CUDA;
  }
}

// device copy of a host or device array (owned by `buf` when staged)
template <typename T>
const T* on_device(const T* p, size_t count, DBuf<T>& buf, Allocator& al, cudaStream_t s) {
  if (count == 0 || is_device_pointer(p)) return p;
  buf.reset(al, count);
  copy_in(buf.get(), p, sizeof(T) * count, s);
  return buf.get();
}

void release_multi(Multi* M) {
  if (!M) return;
  cudaStreamSynchronize(M->g.stream);
  for (auto& e : M->exec) {
    if (e) cudaGraphExecDestroy(e);
    e = nullptr;
  }
  if (M->host) cudaFreeHost(M->host);
  M->host = nullptr;
  if (M->g.host_state) cudaFreeHost(M->g.host_state);
  M->g.host_state = nullptr;
}

}  // namespace
}  // namespace psi

struct psi_multi {
  psi::Multi m;
};

extern "C" {

psi_status psi_multi_create(int32_t G, const int64_t* n_g, const int64_t* m_g, const int32_t* follower,
                            const int32_t* leader, const double* lambda, const double* mu, const psi_options* opt,
                            psi_multi** out) {
  using namespace psi;
  if (out) *out = nullptr;
  psi_multi* h = nullptr;
  psi_status st = multi_guard([&] {
    PSI_REQUIRE(out, PSI_ERR_INVALID_ARG, "out is NULL");
    PSI_REQUIRE(G >= 1 && G <= kMaxGraphs, PSI_ERR_INVALID_ARG, "G must be in [1, 1024]");
    PSI_REQUIRE(n_g && m_g, PSI_ERR_INVALID_ARG, "n_g and m_g are required (host arrays of G entries)");
    PSI_REQUIRE(lambda && mu, PSI_ERR_INVALID_ARG, "lambda and mu are required");
    std::vector<int64_t> noff((size_t)G + 1, 0), moff((size_t)G + 1, 0);
    for (int q = 0; q < G; ++q) {
      PSI_REQUIRE(n_g[q] >= 1, PSI_ERR_INVALID_ARG, "every graph needs n_g >= 1");
      PSI_REQUIRE(m_g[q] >= 0, PSI_ERR_INVALID_ARG, "m_g must be >= 0");
      noff[q + 1] = noff[q] + n_g[q];
      moff[q + 1] = moff[q] + m_g[q];
      PSI_REQUIRE(noff[q + 1] < ((int64_t)1 << 31) - 1, PSI_ERR_INVALID_ARG, "sum of n_g must be below 2^31 - 1");
      PSI_REQUIRE(moff[q + 1] < ((int64_t)1 << 31) - 1, PSI_ERR_INVALID_ARG, "sum of m_g must be below 2^31 - 1");
    }
    const int64_t n = noff[G], m = moff[G];
    PSI_REQUIRE(m == 0 || (follower && leader), PSI_ERR_INVALID_ARG, "follower/leader are NULL");
    psi_options o;
    psi_options_default(&o);
    if (opt) o = *opt;
    PSI_REQUIRE(o.tol_mode == PSI_TOL_PSI || o.tol_mode == PSI_TOL_S_ABS, PSI_ERR_INVALID_ARG, "unknown tol_mode");
    PSI_REQUIRE(o.bnorm_mode == PSI_BNORM_NONE || o.bnorm_mode == PSI_BNORM_INF, PSI_ERR_INVALID_ARG,
                "unknown bnorm_mode");
    PSI_REQUIRE(o.self_loops == PSI_REJECT || o.self_loops == PSI_DROP, PSI_ERR_INVALID_ARG, "unknown self_loops");
    PSI_REQUIRE(o.spmv_tile == 0 || o.spmv_tile == 512 || o.spmv_tile == 1024 || o.spmv_tile == 2048,
                PSI_ERR_INVALID_ARG, "spmv_tile must be 0, 512, 1024 or 2048");
    o.precision = PSI_FP32_REFINE;
    // small tiles: once most graphs have stopped, the few still stepping own few nonzeros,
    // and every tile is walked by one warp (the autotuner may pick another on the first solve)
    const bool tile_fixed = o.spmv_tile != 0;
    if (o.spmv_tile == 0) o.spmv_tile = 512;
    h = new psi_multi();
    Multi& M = h->m;
    Graph& g = M.g;
    g.opt = o;
    g.stream = static_cast<cudaStream_t>(o.stream);
    g.al.stream = g.stream;
    if (o.allocator) {
      PSI_REQUIRE(o.allocator->alloc && o.allocator->free, PSI_ERR_INVALID_ARG, "allocator callbacks are NULL");
      g.al.user = *o.allocator;
      g.al.has_user = true;
    }
    cudaStream_t s = g.stream;
    M.G = G;
    M.tile_fixed = tile_fixed;
    M.h_noff = noff;
    M.noff.reset(g.al, (size_t)G + 1);
    PSI_CUDA(cudaMemcpyAsync(M.noff.get(), noff.data(), sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice, s));
    DBuf<int64_t> dmoff(g.al, (size_t)G + 1);
    PSI_CUDA(cudaMemcpyAsync(dmoff.get(), moff.data(), sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice, s));
    // union edge list, graph of every user
    DBuf<int32_t> fbuf, lbuf, uf(g.al, (size_t)m), ul(g.al, (size_t)m), group_in(g.al, (size_t)n);
    DBuf<double> lbuf_d, mbuf_d;
    DBuf<uint32_t> bad(g.al, 1);
    PSI_CUDA(cudaMemsetAsync(bad.get(), 0, sizeof(uint32_t), s));
    if (m > 0) {
      const int32_t* df = on_device(follower, (size_t)m, fbuf, g.al, s);
      const int32_t* dl = on_device(leader, (size_t)m, lbuf, g.al, s);
      k_union_edges<<<mgrid(m), 256, 0, s>>>(df, dl, m, dmoff.get(), M.noff.get(), G, uf.get(), ul.get(), bad.get());
      PSI_LAUNCHED();
    }
    k_user_groups<<<mgrid(n), 256, 0, s>>>(M.noff.get(), G, n, group_in.get());
    PSI_LAUNCHED();
    uint32_t hb = 0;
    PSI_CUDA(cudaMemcpyAsync(&hb, bad.get(), sizeof(hb), cudaMemcpyDeviceToHost, s));
    PSI_CUDA(cudaStreamSynchronize(s));
    PSI_REQUIRE(!hb, PSI_ERR_OUT_OF_RANGE_ID, "an edge endpoint is outside [0, n_g) of its graph");
    fbuf.release();
    lbuf.release();
    const double* dlam = on_device(lambda, (size_t)n, lbuf_d, g.al, s);
    const double* dmu = on_device(mu, (size_t)n, mbuf_d, g.al, s);
    M.bnorm_bits.reset(g.al, (size_t)G);
    PSI_CUDA(cudaMemsetAsync(M.bnorm_bits.get(), 0, sizeof(unsigned long long) * G, s));
    MultiHook hook(M, group_in.get());
    build_graph(g, n, m, uf.get(), ul.get(), dlam, dmu, &hook);
    uf.release();
    ul.release();
    // graph of every internal user, row ranges, graph ranges of the tiles
    M.gid.reset(g.al, (size_t)n);
    k_internal_groups<<<mgrid(n), 256, 0, s>>>(group_in.get(), g.perm.get(), n, M.gid.get());
    PSI_LAUNCHED();
    M.ranges.reset(g.al, (size_t)G);
    PSI_CUDA(cudaMemsetAsync(M.ranges.get(), 0, sizeof(int4) * G, s));
    if (g.n_rows > 0) {
      k_group_ranges<<<mgrid(g.n_rows), 256, 0, s>>>(M.gid.get(), g.nX, g.n_rows, M.ranges.get());
      PSI_LAUNCHED();
    }
    M.tile_g.reset(g.al, (size_t)(g.num_tiles > 0 ? g.num_tiles : 1));
    if (g.num_tiles > 0) {
      k_tile_groups<<<mgrid(g.num_tiles), 256, 0, s>>>(g.tile_row.get(), g.num_tiles, M.gid.get(), g.nX,
                                                        M.tile_g.get());
      PSI_LAUNCHED();
    }
    // N, ||B||_inf and the gap scale of every graph
    std::vector<unsigned long long> bits((size_t)G);
    PSI_CUDA(cudaMemcpyAsync(bits.data(), M.bnorm_bits.get(), sizeof(unsigned long long) * G, cudaMemcpyDeviceToHost,
                             s));
    PSI_CUDA(cudaStreamSynchronize(s));
    M.bnorm_bits.release();
    std::vector<double> nq((size_t)G), bn((size_t)G), sc((size_t)G);
    for (int q = 0; q < G; ++q) {
      nq[q] = (double)n_g[q];
      std::memcpy(&bn[q], &bits[q], sizeof(double));
      sc[q] = (o.bnorm_mode == PSI_BNORM_INF ? bn[q] : 1.0) * (o.tol_mode == PSI_TOL_PSI ? 1.0 / nq[q] : 1.0);
    }
    M.n_of.reset(g.al, (size_t)G);
    M.bnorm.reset(g.al, (size_t)G);
    M.scale.reset(g.al, (size_t)G);
    PSI_CUDA(cudaMemcpyAsync(M.n_of.get(), nq.data(), sizeof(double) * G, cudaMemcpyHostToDevice, s));
    PSI_CUDA(cudaMemcpyAsync(M.bnorm.get(), bn.data(), sizeof(double) * G, cudaMemcpyHostToDevice, s));
    PSI_CUDA(cudaMemcpyAsync(M.scale.get(), sc.data(), sizeof(double) * G, cudaMemcpyHostToDevice, s));
    multi_buffers(M);
    PSI_CUDA(cudaStreamSynchronize(s));
  });
  if (st != PSI_OK) {
    if (h) {
      release_multi(&h->m);
      cudaGetLastError();
      delete h;
    }
    return st;
  }
  *out = h;
  return PSI_OK;
}

psi_status psi_multi_solve(psi_multi* h, double eps, int32_t max_iter, psi_solve_info* info) {
  using namespace psi;
  if (!h) {
    set_last_error("multi is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  psi_status result = PSI_OK;
  psi_status st = multi_guard([&] { result = multi_solve(h->m, eps, max_iter, info); });
  if (st != PSI_OK) return st;
  if (result == PSI_ERR_NOT_CONVERGED) set_last_error("max_iter reached before every graph met its stop test");
  return result;
}

psi_status psi_multi_scores(const psi_multi* h, double* psi_out) {
  using namespace psi;
  if (!h || !psi_out) {
    set_last_error("multi or output is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  if (!h->m.solved) {
    set_last_error("psi_multi_solve has not produced scores yet");
    return PSI_ERR_NOT_SOLVED;
  }
  return multi_guard([&] {
    const Graph& g = h->m.g;
    copy_out(psi_out, h->m.psi.get(), sizeof(double) * (size_t)g.n, g.stream);
    PSI_CUDA(cudaStreamSynchronize(g.stream));
  });
}

psi_status psi_multi_topk(const psi_multi* h, int32_t k, int32_t* ids_out, double* vals_out) {
  using namespace psi;
  if (!h || !ids_out) {
    set_last_error("multi or ids_out is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  if (!h->m.solved) {
    set_last_error("psi_multi_solve has not produced scores yet");
    return PSI_ERR_NOT_SOLVED;
  }
  int64_t n_min = INT64_MAX;
  for (int q = 0; q < h->m.G; ++q) n_min = std::min<int64_t>(n_min, h->m.h_noff[q + 1] - h->m.h_noff[q]);
  if (k < 1 || k > kMultiTopkMax || (int64_t)k > n_min) {
    set_last_error("k must be in [1, min(1024, smallest n_g)]");
    return PSI_ERR_INVALID_ARG;
  }
  return multi_guard([&] {
    Multi& M = const_cast<Multi&>(h->m);
    Graph& g = M.g;
    const size_t total = (size_t)M.G * (size_t)k;
    DBuf<int32_t> di(g.al, total);
    DBuf<double> dv(g.al, total);
    k_multi_topk<<<M.G, 256, 0, g.stream>>>(M.psi.get(), M.noff.get(), k, di.get(), dv.get());
    PSI_LAUNCHED();
    copy_out(ids_out, di.get(), sizeof(int32_t) * total, g.stream);
    if (vals_out) copy_out(vals_out, dv.get(), sizeof(double) * total, g.stream);
    PSI_CUDA(cudaStreamSynchronize(g.stream));
  });
}

psi_status psi_multi_get_stats(const psi_multi* h, psi_graph_stats* st) {
  if (!h || !st) {
    psi::set_last_error("multi or stats is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  psi::fill_graph_stats(h->m.g, st);
  return PSI_OK;
}

void psi_multi_destroy(psi_multi* h) {
  if (!h) return;
  psi::release_multi(&h->m);
  delete h;
  cudaGetLastError();
}

}  // extern "C"
