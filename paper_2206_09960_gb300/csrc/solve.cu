// solve.cu -- Power-psi (Algorithm 2) on the device: step kernels, the device-side stop
// test, the three precision modes and the final psi.
#include <cmath>
#include <map>
#include <mutex>
#include <chrono>
#include <tuple>
#include <type_traits>

#include "build.cuh"
#include "primitives.cuh"
#include "trace.cuh"
#include "solve.cuh"
#include "spmv.cuh"

namespace psi {

namespace {

// Sums the step's gap partials in a fixed order and applies the stop test of
// Algorithm 2: stop when scale * ||s_t - s_{t-1}||_1 <= eps (Eqs. 15-16) or at max_iter.
__global__ void __launch_bounds__(1024) k_finalize(DevState* st, const double* __restrict__ gp, int ngp,
                                                  const double* __restrict__ gf, int ngf) {
  if (st->done) return;
  __shared__ double sh[1024];
  double acc = 0.0;
  for (int i = threadIdx.x; i < ngp; i += blockDim.x) acc += gp[i];
  for (int i = threadIdx.x; i < ngf; i += blockDim.x) acc += gf[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double gap = sh[0] + st->extra_gap;
    const double prev = st->gap;  // the previous step's gap (same phase when phase_iters >= 1)
    st->extra_gap = 0.0;
    st->gap = gap;
    st->gap_scaled = gap * st->scale;
    st->total_iters += 1;
    st->phase_iters += 1;
    // In an FP32 series phase the terms shrink geometrically; when the next gap, predicted
    // from the last two with a 1.2x margin, meets the test, the series stops one step early
    // and the FP64 confirming step that follows is that next step (its gap is still the one
    // tested, so the stop rule of Algorithm 2 is unchanged; a wrong guess costs a series).
    const bool next_passes = st->predict && st->phase_iters >= 2 && gap < prev &&
                             1.2 * (gap / prev) * st->gap_scaled <= st->eps;
    if (st->gap_scaled <= st->eps || (next_passes && st->total_iters < st->max_iter)) {
      st->done = 1;
      st->converged = 1;
    } else if (st->total_iters >= st->max_iter) {
      st->done = 1;
      st->converged = 0;
    }
  }
}

__global__ void k_phase_begin(DevState* st, int predict) {
  st->phase_iters = 0;
  st->converged = 0;
  st->predict = predict;
  st->done = st->total_iters >= st->max_iter ? 1 : 0;
}

template <typename T>
__global__ void k_fill(T* x, int64_t n, T v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = v;
}

template <typename D, typename S>
__global__ void k_convert(D* dst, const S* src, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (D)src[i];
}

// Gathered vectors live in their own index space: users with leaders only, X at [0, nX)
// and U at [nX, nX + nU) (user nX + nR + j at nX + j), plus a zero pad entry at nX + nU.
// dst[i] = s[user(i)] * isig[user(i)] for i in [lo, hi).
template <typename T, typename S>
__global__ void k_to_u(T* dst, const S* s, const T* isig, int32_t nX, int32_t nR, int64_t lo, int64_t hi) {
  for (int64_t i = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t user = i < nX ? i : i + nR;
    dst[i] = (T)s[user] * isig[user];
  }
}

// the same into the gathered vector of a confirming or final product (FP64 or float pairs)
template <typename G>
__global__ void k_to_u_g(G* dst, const double* s, const double* isig, int32_t nX, int32_t nR, int64_t lo,
                         int64_t hi) {
  for (int64_t i = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t user = i < nX ? i : i + nR;
    dst[i] = to_gather<G>(s[user] * isig[user]);
  }
}

// out[k] = in[perm[k]] (gather into internal order)
__global__ void k_gather_f64(double* out, const double* in, const int32_t* perm, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[perm[i]];
}

// non-row users of a warm start: their s_1 = c; the change |c - s_0| joins the first gap
__global__ void k_nonrow_start(double* s, const double* c, int64_t lo, int64_t n, double* part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int64_t i = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    acc += fabs(c[i] - s[i]);
    s[i] = c[i];
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_set_extra_gap(DevState* st, const double* part, int np) {
  double acc = 0.0;
  for (int i = 0; i < np; ++i) acc += part[i];
  st->extra_gap = acc;
}

// psi of users without followers: G = 0, psi = d / N
__global__ void k_psi_nonrow(double* psi, const double* d, int64_t lo, int64_t n) {
  for (int64_t i = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    psi[i] = d[i] / (double)n;
}

int elementwise_grid(int64_t n) {
  int64_t g = ceil_div(n > 0 ? n : 1, 256);
  int64_t cap = num_sms() * 8;
  return (int)(g < cap ? g : cap);
}

template <typename T>
void fill(T* x, int64_t n, T v, cudaStream_t s) {
  if (n <= 0) return;
  k_fill<T><<<elementwise_grid(n), 256, 0, s>>>(x, n, v);
  PSI_LAUNCHED();
}

template <typename T, typename Epi>
int spmv_grid(int32_t tiles) {
  static const int per_sm = [] {  // once, thread-safe
    int b = 0;
    PSI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_spmv<T, Epi>, kSpmvThreads, 0));
    return b > 0 ? b : 1;
  }();
  return spmv_blocks(per_sm, tiles);
}

constexpr int32_t kHotMax = 32768;  // largest shared-memory copy of the series product (FP32 entries)

// One block per SM of the series product with a shared-memory copy (no more blocks than
// the tiles fill)
int hot_series_grid(int32_t tiles) {
  static const bool configured = [] {  // once, thread-safe
    PSI_CUDA(cudaFuncSetAttribute(k_spmv<float, EpiSeries, kSpmvHotWarps>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(float) * kHotMax)));
    return true;
  }();
  (void)configured;
  const int64_t need = ceil_div(tiles > 0 ? tiles : 1, kSpmvHotWarps);
  return (int)(need < num_sms() ? need : num_sms());
}

// ------------------------------------------------------------------ autotuner
// The FP32 series product (the step that takes nearly all of a solve) has two free
// parameters: the tile (512, 1024 or 2048 nonzeros per warp task) and the number of
// most-gathered entries read from shared memory instead of L1/L2 (0, or a copy of 24K-32K
// entries with one 32-warp block per SM).  Which is fastest depends on the graph's size
// and degree distribution, so on the first solve of a large graph every candidate is
// timed on the graph itself (CUDA events, a warm-up launch then three timed ones, on the
// solver's own buffers before they are initialised) and the fastest is kept.  The choice is
// remembered per graph signature for the process, so later graphs of the same sizes skip
// the timing.
struct TuneKey {
  int64_t n_rows, nu, m, max_followers;
  int32_t tile_req, hot_req;  // what the options fixed
  bool operator<(const TuneKey& o) const {
    return std::tie(n_rows, nu, m, max_followers, tile_req, hot_req) <
           std::tie(o.n_rows, o.nu, o.m, o.max_followers, o.tile_req, o.hot_req);
  }
};
struct TuneChoice {
  int32_t tile, hot;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune_cache;

constexpr int64_t kTuneMinNnz = (int64_t)1 << 22;  // smaller graphs keep the fixed rule

// average time of one FP32 series step (product + fix-up) with the given schedule and copy
float time_series_step(Graph& g, const Schedule& sc, int32_t hot, cudaStream_t s) {
  Allocator& al = g.al;
  DBuf<float> ch(al, (size_t)sc.tiles), ct(al, (size_t)sc.tiles);
  DBuf<double> gt(al, (size_t)sc.tiles);
  SpmvArgs a{};
  a.row_ptr = g.row_ptr.get();
  a.col = g.col.get();
  a.tile_row = sc.tile_row.get();
  a.tile = sc.tile;
  a.num_tiles = sc.tiles;
  a.hot = hot;
  a.n_rows = g.n_rows;
  a.m = g.m_unique;
  a.state = g.state.get();
  a.gap_part = g.gap_part.get();
  a.tile_ctr = g.tile_ctr.get();
  a.gap_tile = gt.get();
  a.carry_head = ch.get();
  a.carry_tail = ct.get();
  FixArgs f{};
  f.row_ptr = g.row_ptr.get();
  f.tile_row = sc.tile_row.get();
  f.tile = sc.tile;
  f.fix_tile = sc.fix_tile.get();
  f.num_fix = sc.num_fix;
  f.state = g.state.get();
  f.gap_fix = g.gap_fix.get();
  f.carry_head = ch.get();
  f.carry_tail = ct.get();
  f.gap_tile = gt.get();
  f.gap_tiles = sc.tiles;
  // scratch output: the series term goes to u32b, the sums to s64 (both initialised by the
  // solve that follows)
  EpiSeries epi{g.mu32.get(), g.isig32.get(), g.s64.get(), g.u32b.get(), g.nX};
  auto launch = [&]() {
    if (hot > 0) {
      k_spmv<float, EpiSeries, kSpmvHotWarps>
          <<<hot_series_grid(sc.tiles), kSpmvHotWarps * 32, sizeof(float) * (size_t)hot, s>>>(a, g.u32a.get(), epi);
    } else {
      k_spmv<float, EpiSeries><<<spmv_grid<float, EpiSeries>(sc.tiles), kSpmvThreads, 0, s>>>(a, g.u32a.get(), epi);
    }
    PSI_LAUNCHED();
    // the fix-up also adds the per-tile gaps, so it runs on every step
    k_fixup<float, EpiSeries><<<fix_blocks(std::max(sc.num_fix, sc.tiles)), kFixThreads, 0, s>>>(f, epi);
    PSI_LAUNCHED();
  };
  cudaEvent_t e0, e1;
  PSI_CUDA(cudaEventCreate(&e0));
  PSI_CUDA(cudaEventCreate(&e1));
  launch();
  PSI_CUDA(cudaEventRecord(e0, s));
  for (int i = 0; i < 3; ++i) launch();
  PSI_CUDA(cudaEventRecord(e1, s));
  PSI_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  PSI_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / 3.f;
}

void apply_schedule(Graph& g, Schedule&& sc) {
  g.tile = sc.tile;
  g.num_tiles = sc.tiles;
  g.num_fix = sc.num_fix;
  g.tile_row = std::move(sc.tile_row);
  g.fix_tile = std::move(sc.fix_tile);
  g.carry_head.reset(g.al, (size_t)(g.num_tiles > 0 ? g.num_tiles : 1));
  g.carry_tail.reset(g.al, (size_t)(g.num_tiles > 0 ? g.num_tiles : 1));
  if (g.allocated_iter) g.gap_tile.reset(g.al, (size_t)(g.num_tiles > 0 ? g.num_tiles : 1));
}

void autotune_series(Graph& g, cudaStream_t s) {
  g.tuned = true;
  const int64_t nu = (int64_t)g.nX + g.nU;
  // a requested copy, never longer than the gathered vector (u holds nu entries and a pad)
  const int32_t hot_req = g.opt.spmv_hot < 0 ? -1 : (int32_t)std::min<int64_t>(g.opt.spmv_hot, nu);
  if (g.opt.precision != PSI_FP32_REFINE) return;
  if (!g.opt.autotune || g.m_unique < kTuneMinNnz || (g.opt.spmv_tile > 0 && hot_req >= 0)) {
    g.series_hot = hot_req > 0 ? hot_req : 0;
    return;
  }
  const TuneKey key{g.n_rows, nu, g.m_unique, g.max_followers, g.opt.spmv_tile, hot_req};
  TuneChoice pick{g.tile, hot_req > 0 ? hot_req : 0};
  bool cached = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      pick = it->second;
      cached = true;
    }
  }
  if (g.opt.spmv_tile > 0) pick.tile = g.opt.spmv_tile;
  if (!cached) {
    NvtxRange range("psi solve: autotune");
    const auto t0 = std::chrono::steady_clock::now();
    PSI_CUDA(cudaMemsetAsync(g.state.get(), 0, sizeof(DevState), s));
    PSI_CUDA(cudaMemsetAsync(g.u32a.get(), 0, sizeof(float) * (size_t)(nu + 1), s));
    PSI_CUDA(cudaMemsetAsync(g.s64.get(), 0, sizeof(double) * (size_t)g.n, s));
    // the copy first, on the rule's tile; then the tile, with the best copy
    const int32_t hots[4] = {0, 24576, 28672, kHotMax};
    std::map<int32_t, Schedule> scheds;
    auto sched_for = [&](int32_t tile) -> const Schedule& {
      auto it = scheds.find(tile);
      if (it == scheds.end())
        it = scheds.emplace(tile, make_schedule(g.row_ptr.get(), g.n_rows, g.m_unique, g.al, s, tile)).first;
      return it->second;
    };
    float best = 0.f;
    bool first = true;
    for (int32_t h : hots) {
      if (hot_req >= 0 && h != 0) break;  // the copy is fixed by the options
      if (hot_req >= 0) h = hot_req;
      if (hot_req < 0 && h > 0 && nu < 8 * (int64_t)h) continue;  // a copy pays only as a small part of the vector
      const float ms = time_series_step(g, sched_for(pick.tile), h, s);
      if (first || ms < best) {
        best = ms;
        pick.hot = h;
        first = false;
      }
    }
    if (g.opt.spmv_tile == 0) {
      const int32_t tiles[3] = {kSpmvTileMin, 2 * kSpmvTileMin, kSpmvTileMax};
      const int32_t rule = pick.tile;
      for (int32_t t : tiles) {
        if (t == rule) continue;
        const float ms = time_series_step(g, sched_for(t), pick.hot, s);
        if (ms < best) {
          best = ms;
          pick.tile = t;
        }
      }
    }
    if (pick.tile != g.tile) apply_schedule(g, std::move(scheds.at(pick.tile)));
    g.tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = pick;
  } else if (pick.tile != g.tile) {
    apply_schedule(g, make_schedule(g.row_ptr.get(), g.n_rows, g.m_unique, g.al, s, pick.tile));
  }
  g.series_hot = pick.hot;
}

}  // namespace

// ------------------------------------------------------------------ step launch
struct Stepper {
  Graph& g;
  cudaStream_t s;
  bool profile;
  std::vector<cudaEvent_t>& ev;   // pairs (start, stop) per product
  std::vector<int>& ev_phase;     // phase-local index of each pair
  int phase_step = 0;
  int launches = 0;

  template <typename T, typename Epi>
  void step(const T* u, const Epi& epi) {
    SpmvArgs a{};
    a.row_ptr = g.row_ptr.get();
    a.col = g.col.get();
    a.tile_row = g.tile_row.get();
    a.tile = g.tile;
    a.num_tiles = g.num_tiles;
    a.n_rows = g.n_rows;
    a.m = g.m_unique;
    a.state = g.state.get();
    a.gap_part = g.gap_part.get();
    // FP32 products claim their tiles at run time (their gaps then reach k_finalize through
    // the fix-up's fixed slices); the 8- and 16-byte products keep the fixed stride
    constexpr bool claims = sizeof(T) == 4;
    a.tile_ctr = claims ? g.tile_ctr.get() : nullptr;
    a.gap_tile = claims ? g.gap_tile.get() : nullptr;
    a.carry_head = g.carry_head.get();
    a.carry_tail = g.carry_tail.get();
    int grid = 0, fgrid = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (profile) {
      PSI_CUDA(cudaEventCreate(&e0));
      PSI_CUDA(cudaEventCreate(&e1));
      PSI_CUDA(cudaEventRecord(e0, s));
    }
    if (g.num_tiles > 0) {
      if constexpr (std::is_same<Epi, EpiSeries>::value) {
        if (g.series_hot > 0) {
          a.hot = g.series_hot;
          grid = hot_series_grid(g.num_tiles);
          k_spmv<float, EpiSeries, kSpmvHotWarps>
              <<<grid, kSpmvHotWarps * 32, sizeof(float) * (size_t)g.series_hot, s>>>(a, u, epi);
          PSI_LAUNCHED();
        }
      }
      if (a.hot == 0) {
        grid = spmv_grid<T, Epi>(g.num_tiles);
        k_spmv<T, Epi><<<grid, kSpmvThreads, 0, s>>>(a, u, epi);
        PSI_LAUNCHED();
      }
    }
    // the fix-up closes rows that span tiles and, after claimed tiles, adds the product's
    // per-tile gaps in fixed slices (no per-block gap then has a fixed order)
    if (claims ? g.num_tiles > 0 : g.num_fix > 0) {
      FixArgs f{};
      f.row_ptr = g.row_ptr.get();
      f.tile_row = g.tile_row.get();
      f.tile = g.tile;
      f.fix_tile = g.fix_tile.get();
      f.num_fix = g.num_fix;
      f.state = g.state.get();
      f.gap_fix = g.gap_fix.get();
      f.carry_head = g.carry_head.get();
      f.carry_tail = g.carry_tail.get();
      f.gap_tile = claims ? g.gap_tile.get() : nullptr;
      f.gap_tiles = claims ? g.num_tiles : 0;
      fgrid = fix_blocks(claims ? std::max(g.num_fix, g.num_tiles) : g.num_fix);
      k_fixup<T, Epi><<<fgrid, kFixThreads, 0, s>>>(f, epi);
      PSI_LAUNCHED();
    }
    if (profile) {
      PSI_CUDA(cudaEventRecord(e1, s));
      ev.push_back(e0);
      ev.push_back(e1);
      ev_phase.push_back(phase_step);
    }
    k_finalize<<<1, 1024, 0, s>>>(g.state.get(), g.gap_part.get(), claims ? 0 : grid, g.gap_fix.get(), fgrid);
    PSI_LAUNCHED();
    ++phase_step;
    ++launches;
  }
};

// Runs one phase of steps; step(k) launches phase step k.  Keeps two batches in flight
// and stops when the device reports done.  Returns the steps executed.
template <typename F>
static int run_phase(Graph& g, cudaStream_t s, Stepper& st, F&& step_k, int batch, int predict = 0) {
  NvtxRange range("psi solve: steps");
  k_phase_begin<<<1, 1, 0, s>>>(g.state.get(), predict);
  PSI_LAUNCHED();
  st.phase_step = 0;
  cudaEvent_t evs[2];
  PSI_CUDA(cudaEventCreateWithFlags(&evs[0], cudaEventDisableTiming));
  PSI_CUDA(cudaEventCreateWithFlags(&evs[1], cudaEventDisableTiming));
  DevState* hs = g.host_state;  // two pinned slots
  int k = 0;
  auto launch_batch = [&](int slot) {
    for (int i = 0; i < batch; ++i) step_k(k++);
    PSI_CUDA(cudaMemcpyAsync(hs + slot, g.state.get(), sizeof(DevState), cudaMemcpyDeviceToHost, s));
    PSI_CUDA(cudaEventRecord(evs[slot], s));
  };
  launch_batch(0);
  int b = 1;
  int executed = 0;
  for (;;) {
    launch_batch(b & 1);
    PSI_CUDA(cudaEventSynchronize(evs[(b - 1) & 1]));
    if (hs[(b - 1) & 1].done) {
      PSI_CUDA(cudaEventSynchronize(evs[b & 1]));
      executed = hs[b & 1].phase_iters;
      break;
    }
    ++b;
  }
  cudaEventDestroy(evs[0]);
  cudaEventDestroy(evs[1]);
  return executed;
}

// One step outside the batched loop (the FP64 refinement step): run it and read the state.
template <typename F>
static DevState run_single(Graph& g, cudaStream_t s, Stepper& st, F&& step_0) {
  NvtxRange range("psi solve: FP64 step");
  k_phase_begin<<<1, 1, 0, s>>>(g.state.get(), 0);
  PSI_LAUNCHED();
  st.phase_step = 0;
  step_0();
  PSI_CUDA(cudaMemcpyAsync(g.host_state, g.state.get(), sizeof(DevState), cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaStreamSynchronize(s));
  return g.host_state[0];
}

static DevState read_state(Graph& g, cudaStream_t s) {
  PSI_CUDA(cudaMemcpyAsync(g.host_state, g.state.get(), sizeof(DevState), cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaStreamSynchronize(s));
  return g.host_state[0];
}

void ensure_iteration_buffers(Graph& g) {
  if (g.allocated_iter) return;
  Allocator& al = g.al;
  const size_t n = (size_t)g.n;
  const size_t nu = (size_t)g.nX + (size_t)g.nU;  // gathered entries; pad at nu
  const int prec = g.opt.precision;
  if (prec == PSI_FP32_REFINE || prec == PSI_FP64) {
    g.s64.reset(al, n);
    g.u64a.reset(al, nu + 1);
    g.u64b.reset(al, nu + 1);
  }
  if (prec == PSI_FP64) g.s64b.reset(al, n);
  if (prec == PSI_FP32) {
    g.s32a.reset(al, n);
    g.s32b.reset(al, n);
  }
  if (prec == PSI_FP32 || prec == PSI_FP32_REFINE) {
    g.u32a.reset(al, nu + 1);
    g.u32b.reset(al, nu + 1);
  }
  if (prec == PSI_FP32_REFINE) g.u32c.reset(al, nu + 1);
  g.psi64.reset(al, n);
  const size_t nt = (size_t)(g.num_tiles > 0 ? g.num_tiles : 1);
  g.carry_head.reset(al, nt);
  g.carry_tail.reset(al, nt);
  g.gap_part.reset(al, (size_t)num_sms() * 32);
  g.gap_fix.reset(al, (size_t)num_sms() * 8);
  g.gap_tile.reset(al, nt);
  g.tile_ctr.reset(al, 2);
  PSI_CUDA(cudaMemsetAsync(g.tile_ctr.get(), 0, 2 * sizeof(int32_t), g.stream));
  g.state.reset(al, 1);
  if (!g.host_state) PSI_CUDA(cudaMallocHost((void**)&g.host_state, 2 * sizeof(DevState)));
  g.allocated_iter = true;
}

static void init_state(Graph& g, cudaStream_t s, double eps, int32_t max_iter, double scale) {
  DevState h{};
  h.max_iter = max_iter;
  h.eps = eps;
  h.scale = scale;
  g.host_state[0] = h;
  PSI_CUDA(cudaMemcpyAsync(g.state.get(), g.host_state, sizeof(DevState), cudaMemcpyHostToDevice, s));
  PSI_CUDA(cudaStreamSynchronize(s));  // the pinned slot is reused below
}

// s_dst (internal order) = the caller's warm start (input order, host or device)
static void load_init(Graph& g, cudaStream_t s, const double* init_s, double* s_dst) {
  const int64_t n = g.n;
  DBuf<double> tmp(g.al, (size_t)n);
  copy_in(tmp.get(), init_s, sizeof(double) * n, s);
  k_gather_f64<<<elementwise_grid(n), 256, 0, s>>>(s_dst, tmp.get(), g.perm.get(), n);
  PSI_LAUNCHED();
}

// Users without followers have s_t = c for t >= 1; with a warm start their change
// |c - s_0| belongs to the first step's gap.  Sets s to c there and queues that change.
static void nonrow_start(Graph& g, cudaStream_t s, double* s64, const double* c64) {
  const int64_t n = g.n;
  if (g.n_rows >= n) return;
  const int blocks = 64;
  DBuf<double> part(g.al, blocks);
  k_nonrow_start<<<blocks, 256, 0, s>>>(s64, c64, g.n_rows, n, part.get());
  PSI_LAUNCHED();
  k_set_extra_gap<<<1, 1, 0, s>>>(g.state.get(), part.get(), blocks);
  PSI_LAUNCHED();
}

psi_status solve_with(Graph& g, const SolveConsts& K, const SolveTarget& T, double eps, int32_t max_iter,
                      const double* init_s, psi_solve_info* info) {
  PSI_REQUIRE(max_iter >= 0, PSI_ERR_INVALID_ARG, "max_iter must be >= 0");
  PSI_REQUIRE(!std::isnan(eps), PSI_ERR_INVALID_ARG, "eps is NaN");
  cudaStream_t s = g.stream;
  ensure_iteration_buffers(g);
  if (!g.tuned) autotune_series(g, s);
  if (T.final_psi) g.solved = false;
  const int64_t n = g.n;
  const int32_t nX = g.nX;
  const int32_t nR = g.nR;
  const int64_t nu = (int64_t)g.nX + g.nU;        // gathered entries (X, then U); pad at nu
  const int prec = g.opt.precision;
  const int batch = g.m_unique > ((int64_t)1 << 24) ? 2 : 8;
  const int eg = elementwise_grid(n);

  cudaEvent_t t0, t1;
  PSI_CUDA(cudaEventCreate(&t0));
  PSI_CUDA(cudaEventCreate(&t1));
  init_state(g, s, eps, max_iter, T.scale);
  PSI_CUDA(cudaEventRecord(t0, s));

  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_phase;
  struct Timed { size_t first; int steps; bool refine; };
  std::vector<Timed> timed;  // event pairs of each phase: first pair, steps executed, FP64 refinement?
  Stepper st{g, s, g.opt.profile != 0, ev, ev_phase};
  // Algorithm 2 enters its loop only while gap (initially 1) > eps
  const bool iterate = (1.0 > eps) && max_iter > 0;
  int refinements = 0;
  const double* u_final64 = nullptr;
  const DF* u_final_df = nullptr;
  const float* u_final32 = nullptr;
  // gathered vector of s_0 when a warm start is given (U users use s_0 in step 1 only)
  DBuf<double> u0_64;
  DBuf<float> u0_32;

  if (prec == PSI_FP64) {
    double* sb[2] = {g.s64.get(), g.s64b.get()};
    double* ub[2] = {g.u64a.get(), g.u64b.get()};
    for (int b = 0; b < 2; ++b) {  // X from s_0 = c, U = c/sigma (s_t = c there for t >= 1)
      fill<double>(ub[b], nu + 1, 0.0, s);
      k_to_u<double, double><<<eg, 256, 0, s>>>(ub[b], K.c64, K.isig64, nX, nR, 0, nu);
      PSI_LAUNCHED();
    }
    const double* u_first = ub[0];
    if (init_s) {
      load_init(g, s, init_s, sb[0]);
      u0_64.reset(g.al, (size_t)nu + 1);
      fill<double>(u0_64.get(), nu + 1, 0.0, s);
      k_to_u<double, double><<<eg, 256, 0, s>>>(u0_64.get(), sb[0], K.isig64, nX, nR, 0, nu);
      PSI_LAUNCHED();
      if (iterate) nonrow_start(g, s, sb[0], K.c64);
      u_first = u0_64.get();
    } else {
      PSI_CUDA(cudaMemcpyAsync(sb[0], K.c64, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    }
    PSI_CUDA(cudaMemcpyAsync(sb[1], sb[0], sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    int steps = 0;
    if (iterate) {
      size_t first = ev_phase.size();
      steps = run_phase(g, s, st, [&](int k) {
        EpiPlain<double> e{K.c64, K.mu64, K.isig64, sb[k & 1], sb[(k + 1) & 1], ub[(k + 1) & 1], nX};
        st.step<double>(k == 0 ? u_first : ub[k & 1], e);
      }, batch);
      timed.push_back({first, steps, false});
    }
    g.last_s_kind = (steps & 1) ? 1 : 0;
    u_final64 = (steps == 0) ? u_first : ub[steps & 1];
  } else if (prec == PSI_FP32) {
    float* sb[2] = {g.s32a.get(), g.s32b.get()};
    float* ub[2] = {g.u32a.get(), g.u32b.get()};
    for (int b = 0; b < 2; ++b) {
      fill<float>(ub[b], nu + 1, 0.0f, s);
      k_to_u<float, float><<<eg, 256, 0, s>>>(ub[b], K.c32, K.isig32, nX, nR, 0, nu);
      PSI_LAUNCHED();
    }
    const float* u_first = ub[0];
    if (init_s) {
      DBuf<double> s0(g.al, (size_t)n);
      load_init(g, s, init_s, s0.get());
      DBuf<double> u0(g.al, (size_t)nu + 1);
      fill<double>(u0.get(), nu + 1, 0.0, s);
      k_to_u<double, double><<<eg, 256, 0, s>>>(u0.get(), s0.get(), K.isig64, nX, nR, 0, nu);
      PSI_LAUNCHED();
      u0_32.reset(g.al, (size_t)nu + 1);
      k_convert<float, double><<<eg, 256, 0, s>>>(u0_32.get(), u0.get(), nu + 1);
      PSI_LAUNCHED();
      if (iterate) nonrow_start(g, s, s0.get(), K.c64);
      k_convert<float, double><<<eg, 256, 0, s>>>(sb[0], s0.get(), n);
      PSI_LAUNCHED();
      u_first = u0_32.get();
    } else {
      k_convert<float, double><<<eg, 256, 0, s>>>(sb[0], K.c64, n);
      PSI_LAUNCHED();
    }
    PSI_CUDA(cudaMemcpyAsync(sb[1], sb[0], sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    int steps = 0;
    if (iterate) {
      size_t first = ev_phase.size();
      steps = run_phase(g, s, st, [&](int k) {
        EpiPlain<float> e{K.c32, K.mu32, K.isig32, sb[k & 1], sb[(k + 1) & 1], ub[(k + 1) & 1], nX};
        st.step<float>(k == 0 ? u_first : ub[k & 1], e);
      }, batch);
      timed.push_back({first, steps, false});
    }
    g.last_s_kind = (steps & 1) ? 3 : 2;
    u_final32 = (steps == 0) ? u_first : ub[steps & 1];
  } else {  // PSI_FP32_REFINE
    auto refine = [&](auto gather_tag) {
      using G = decltype(gather_tag);
    double* s64 = g.s64.get();
    // gathered vectors of the confirming and final products in the FP64 buffers (8 bytes
    // per entry either way)
    G* ub[2] = {reinterpret_cast<G*>(g.u64a.get()), reinterpret_cast<G*>(g.u64b.get())};
    float* v0 = g.u32c.get();
    float* vb[2] = {g.u32a.get(), g.u32b.get()};
    for (int b = 0; b < 2; ++b) {
      fill<double>(reinterpret_cast<double*>(ub[b]), nu + 1, 0.0, s);  // zero bits: a zero pair
      k_to_u_g<G><<<eg, 256, 0, s>>>(ub[b], K.c64, K.isig64, nX, nR, nX, nu);  // U = c/sigma
      PSI_LAUNCHED();
      fill<float>(vb[b], nu + 1, 0.0f, s);  // series terms of U users vanish after the first
    }
    fill<float>(v0, nu + 1, 0.0f, s);
    int cur_u = 0;            // FP64 buffer that will hold u of the current s64
    bool u_current = false;   // whether it does now
    const G* u_resid_in = nullptr;
    bool resid_first = false;
    if (init_s) {
      load_init(g, s, init_s, s64);
      u0_64.reset(g.al, (size_t)nu + 1);
      fill<double>(u0_64.get(), nu + 1, 0.0, s);
      k_to_u_g<G><<<eg, 256, 0, s>>>(reinterpret_cast<G*>(u0_64.get()), s64, K.isig64, nX, nR, 0, nu);
      PSI_LAUNCHED();
      if (iterate) nonrow_start(g, s, s64, K.c64);
      u_resid_in = reinterpret_cast<const G*>(u0_64.get());  // the first step is an FP64 step from s_0
      resid_first = true;
    } else {
      PSI_CUDA(cudaMemcpyAsync(s64, K.c64, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      // the first series term is c itself: v0 = c/sigma on X and U
      k_to_u<float, float><<<eg, 256, 0, s>>>(v0, K.c32, K.isig32, nX, nR, 0, nu);
      PSI_LAUNCHED();
    }
    bool v0_u_cleared = false;
    if (iterate) {
      for (;;) {
        if (!resid_first) {
          // FP32 series from v0 (Eq. 13), terms summed into s64
          size_t first = ev_phase.size();
          int steps = run_phase(g, s, st, [&](int k) {
            const float* vin = (k == 0) ? v0 : vb[(k + 1) & 1];
            EpiSeries e{K.mu32, K.isig32, s64, vb[k & 1], nX};
            st.step<float>(vin, e);
          }, batch, /*predict=*/1);
          timed.push_back({first, steps, false});
          if (steps > 0) u_current = false;
          DevState h = read_state(g, s);
          if (!h.converged) break;  // the step cap came first
          // FP64 gathered vector of the series' s64 (X users; U hold c/sigma)
          k_to_u_g<G><<<eg, 256, 0, s>>>(ub[cur_u], s64, K.isig64, nX, nR, 0, nX);
          PSI_LAUNCHED();
          u_current = true;
          u_resid_in = ub[cur_u];
        }
        resid_first = false;
        if (!v0_u_cleared && g.nU > 0) {  // later series start from a residual: U terms are 0
          fill<float>(v0 + nX, g.nU, 0.0f, s);
          v0_u_cleared = true;
        }
        // one FP64 step s <- s A + c from s64; its gap is the one tested
        size_t first = ev_phase.size();
        G* u_out = ub[cur_u ^ 1];
        DevState h = run_single(g, s, st, [&]() {
          EpiResid<G> e{K.c64, K.mu64, K.isig64, s64, u_out, v0, nX};
          st.step<G>(u_resid_in, e);
        });
        timed.push_back({first, h.phase_iters, true});
        if (h.phase_iters == 0) break;  // the step cap came first
        ++refinements;
        cur_u ^= 1;
        u_current = true;
        if (h.converged || h.total_iters >= max_iter) break;
      }
    }
    if (!u_current) {  // psi from the current s64 (after a capped series, or no loop)
      k_to_u_g<G><<<eg, 256, 0, s>>>(ub[cur_u], s64, K.isig64, nX, nR, 0, nX);
      PSI_LAUNCHED();
    }
    g.last_s_kind = 0;
    // without any step, psi comes from s_0 itself (a warm start reaches U users too)
    const G* u_fin = (!iterate && init_s) ? reinterpret_cast<const G*>(u0_64.get()) : ub[cur_u];
    if constexpr (std::is_same<G, DF>::value) u_final_df = u_fin;
    else u_final64 = u_fin;
    };
    // The confirming and final products sum float pairs (~48 bits) when the tolerance is
    // far above their rounding (about 2^-46 of ||s||_1 per step); for tighter tolerances,
    // such as an absolute s-tolerance of 1e-9 on millions of users, they sum in FP64.
    const bool use_pairs = eps / T.scale >= std::ldexp(1.0, -30) * (double)n;
    if (use_pairs) refine(DF{});
    else refine(double{});
  }
  // final step of Algorithm 2: psi^T = (s^T B + d^T) / N, one more product
  NvtxRange final_range("psi solve: final");
  const DevState h = read_state(g, s);
  {
    DevState run = h;
    run.done = 0;
    run.max_iter = INT32_MAX;
    g.host_state[1] = run;
    PSI_CUDA(cudaMemcpyAsync(g.state.get(), &g.host_state[1], sizeof(DevState), cudaMemcpyHostToDevice, s));
  }
  st.phase_step = 0;
  if (T.final_psi) {
    if (u_final_df) {
      EpiFinal<DF> e{K.lam64, K.d64, T.out, (double)n};
      st.step<DF>(u_final_df, e);
    } else if (u_final64) {
      EpiFinal<double> e{K.lam64, K.d64, T.out, (double)n};
      st.step<double>(u_final64, e);
    } else {
      EpiFinal<float> e{K.lam64, K.d64, T.out, (double)n};
      st.step<float>(u_final32, e);
    }
    if (g.n_rows < n) {
      k_psi_nonrow<<<elementwise_grid(n - g.n_rows), 256, 0, s>>>(T.out, K.d64, g.n_rows, n);
      PSI_LAUNCHED();
    }
  } else if (g.last_s_kind <= 1) {  // the result is the iterate itself
    const double* sp = g.last_s_kind == 0 ? g.s64.get() : g.s64b.get();
    PSI_CUDA(cudaMemcpyAsync(T.out, sp, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  } else {
    const float* sp = g.last_s_kind == 2 ? g.s32a.get() : g.s32b.get();
    k_convert<double, float><<<eg, 256, 0, s>>>(T.out, sp, n);
    PSI_LAUNCHED();
  }
  PSI_CUDA(cudaEventRecord(t1, s));
  DBuf<double> dsum(g.al, 1);
  sum_f64(T.out, n, dsum.get(), g.al, s);
  PSI_CUDA(cudaMemcpyAsync(&g.host_state[0].gap, dsum.get(), sizeof(double), cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaStreamSynchronize(s));
  const double psi_sum = g.host_state[0].gap;
  float ms = 0.f;
  PSI_CUDA(cudaEventElapsedTime(&ms, t0, t1));
  double spmv_ms = 0.0, refine_ms = 0.0;
  int timed_n = 0, refine_n = 0;
  for (const Timed& ph : timed) {
    for (int q = 0; q < ph.steps; ++q) {
      size_t idx = ph.first + (size_t)q;
      if (idx >= ev_phase.size()) break;
      float e = 0.f;
      PSI_CUDA(cudaEventElapsedTime(&e, ev[2 * idx], ev[2 * idx + 1]));
      if (ph.refine) {
        refine_ms += e;
        ++refine_n;
      } else {
        spmv_ms += e;
        ++timed_n;
      }
    }
  }
  for (auto e : ev) cudaEventDestroy(e);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (T.final_psi) g.solved = true;
  if (info) {
    info->iters = h.total_iters;
    info->converged = iterate ? h.converged : 1;
    info->refinements = refinements;
    info->spmv_launches = h.total_iters + 1;
    info->gap_s_l1 = h.gap;
    info->gap_scaled = h.gap_scaled;
    info->gap_psi_bound = T.final_psi ? h.gap * g.bnorm_inf / (double)n : h.gap;
    info->psi_sum = psi_sum;
    info->ms = ms;
    info->spmv_ms = spmv_ms;
    info->spmv_timed = timed_n;
    info->refine_timed = refine_n;
    info->refine_ms = refine_ms;
  }
  if (!iterate) return PSI_OK;  // Algorithm 2 with gap = 1 <= eps: psi from s_0
  return h.converged ? PSI_OK : PSI_ERR_NOT_CONVERGED;
}

SolveConsts graph_consts(const Graph& g) {
  return SolveConsts{g.c64.get(), g.mu64.get(), g.isig64.get(), g.lam64.get(), g.d64.get(),
                     g.c32.get(), g.mu32.get(), g.isig32.get()};
}

psi_status solve(Graph& g, double eps, int32_t max_iter, const double* init_s, psi_solve_info* info) {
  ensure_iteration_buffers(g);
  const double bn = g.opt.bnorm_mode == PSI_BNORM_INF ? g.bnorm_inf : 1.0;
  const SolveTarget T{bn * (g.opt.tol_mode == PSI_TOL_PSI ? 1.0 / (double)g.n : 1.0), g.psi64.get(), true};
  return solve_with(g, graph_consts(g), T, eps, max_iter, init_s, info);
}

}  // namespace psi
