// batch.cu -- Power-psi for S activity scenarios (lambda, mu sets) on one graph, solved
// together: one product per step serves every scenario (spmm.cuh), each scenario with its
// own constants, gap, stop test and step count (Algorithm 2 per scenario, FP32 series +
// FP64 confirming step as in the single-graph path).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "build.cuh"
#include "trace.cuh"
#include "primitives.cuh"
#include "solve.cuh"
#include "spmm.cuh"

namespace psi {

namespace {

#define BGRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

int bgrid(int64_t n) {
  int64_t g = ceil_div(n > 0 ? n : 1, 256);
  int64_t cap = num_sms() * 16;
  return (int)(g < cap ? g : cap);
}

// out[k] = in[perm[k]] (one scenario's rates into internal order)
__global__ void k_b_permute(const double* __restrict__ in, const int32_t* __restrict__ perm, int64_t n, double* out) {
  BGRID_STRIDE(k, n) out[k] = in[perm[k]];
}

__global__ void k_b_weights(const double* __restrict__ lam, const double* __restrict__ mu, int64_t n, D2* w) {
  BGRID_STRIDE(k, n + 1) w[k] = k < n ? D2(lam[k] + mu[k], lam[k]) : D2(0.0, 0.0);
}

// one scenario's constants, scenario-major [S][n]; bnorm_s = max beta/sigma
__global__ void k_b_consts(const double* __restrict__ lam, const double* __restrict__ mu,
                           const double* __restrict__ sigma, const double* __restrict__ beta, int64_t n, double* c,
                           double* d, double* isig, unsigned long long* bnorm_bits) {
  double bn = 0.0;
  BGRID_STRIDE(k, n) {
    // the single-graph build's formulas: two FP64 divisions per user
    const double x = lam[k], y = mu[k], sg = sigma[k];
    const double inv = 1.0 / (x + y);
    const double is = sg > 0.0 ? 1.0 / sg : 0.0;
    c[k] = y * inv;
    d[k] = x * inv;
    isig[k] = is;
    if (sg > 0.0) bn = fmax(bn, beta[k] * is);
  }
  atomicMax(bnorm_bits, (unsigned long long)__double_as_longlong(bn));
}

// [S][n] (scenario-major) -> [n][Sp] (user-major), padding scenarios set to `pad`
template <typename D, typename Src>
__global__ void k_b_transpose(const Src* __restrict__ in, int S, int Sp, int64_t n, D* out, D pad) {
  __shared__ D tile[32][33];
  const int64_t k0 = (int64_t)blockIdx.x * 32;
  const int s0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int r = ty; r < 32; r += 8) {
    const int s = s0 + r;
    const int64_t k = k0 + tx;
    tile[r][tx] = (s < S && k < n) ? (D)in[(int64_t)s * n + k] : pad;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t k = k0 + r;
    const int s = s0 + tx;
    if (k < n && s < Sp) out[k * Sp + s] = tile[tx][r];
  }
}

// gathered [nu + 1][Sp] from user-major [n][Sp]: X -> same row, U -> row - nR; pad row 0
template <typename T, typename S>
__global__ void k_b_to_u(T* dst, const S* s, const T* isig, int32_t nX, int32_t nR, int64_t lo, int64_t hi, int Sp) {
  BGRID_STRIDE(idx, (hi - lo) * Sp) {
    const int64_t i = lo + idx / Sp;
    const int c = (int)(idx % Sp);
    const int64_t user = i < nX ? i : i + nR;
    dst[i * Sp + c] = (T)s[user * Sp + c] * isig[user * Sp + c];
  }
}

// the same into the gathered matrix of the confirming and final products (FP64 or float pairs)
template <typename E>
__global__ void k_b_to_u_g(E* dst, const double* s, const double* isig, int32_t nX, int32_t nR, int64_t lo,
                           int64_t hi, int Sp) {
  BGRID_STRIDE(idx, (hi - lo) * Sp) {
    const int64_t i = lo + idx / Sp;
    const int c = (int)(idx % Sp);
    const int64_t user = i < nX ? i : i + nR;
    dst[i * Sp + c] = to_gather<E>(s[user * Sp + c] * isig[user * Sp + c]);
  }
}

template <typename T>
__global__ void k_b_fill(T* x, int64_t n, T v) {
  BGRID_STRIDE(i, n) x[i] = v;
}

struct BatchState {
  int32_t done;     // no scenario is stepping
  int32_t mode;     // 0: series (stop a scenario when its gap meets eps), 1: one FP64 step each
  int32_t max_iter;
  int32_t pad_;
  double eps;
};

// Per-scenario gap sums (fixed order) and stop tests; one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_b_finalize(BatchState* st, int32_t* active, int32_t* iters,
                                                    int32_t* phase_it, int32_t* ok, int32_t* converged,
                                                    double* gap_last,
                                                    const double* __restrict__ scale, const double* __restrict__ gp,
                                                    int ngp, const double* __restrict__ gf, int ngf, int Sp) {
  if (st->done) return;
  __shared__ double sh[1024];
  __shared__ int any;
  const int s = threadIdx.x % Sp;
  const int part = threadIdx.x / Sp;
  const int parts = blockDim.x / Sp;
  double acc = 0.0;
  for (int b = part; b < ngp; b += parts) acc += gp[(int64_t)b * Sp + s];
  for (int b = part; b < ngf; b += parts) acc += gf[(int64_t)b * Sp + s];
  sh[threadIdx.x] = acc;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  if (threadIdx.x < Sp) {
    double gsum = 0.0;
    for (int p = 0; p < parts; ++p) gsum += sh[p * Sp + s];
    if (active[s]) {
      const double prev = gap_last[s];
      gap_last[s] = gsum;
      iters[s] += 1;
      const double scaled = gsum * scale[s];
      const bool met = scaled <= st->eps;
      if (st->mode == 0) {
        // as in the single-graph path: stop the series one step early when the next gap,
        // predicted from the last two with a 1.2x margin, meets the test (the FP64 step that
        // follows is tested as usual)
        phase_it[s] += 1;
        const bool next_passes =
            phase_it[s] >= 2 && gsum < prev && 1.2 * (gsum / prev) * scaled <= st->eps && iters[s] < st->max_iter;
        if (met || next_passes) { active[s] = 0; ok[s] = 1; }
        else if (iters[s] >= st->max_iter) active[s] = 0;
      } else {
        if (met) converged[s] = 1;
        active[s] = 0;
      }
    }
    if (active[s]) atomicOr(&any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0 && !any) st->done = 1;
}

__global__ void k_b_psi_nonrow(double* psi, const double* d, int64_t lo, int64_t n, int Sp) {
  BGRID_STRIDE(idx, (n - lo) * Sp) {
    const int64_t i = lo * Sp + idx;
    psi[i] = d[i] / (double)n;
  }
}

// out[s][perm[k]] = in[k][s] for s < S
__global__ void k_b_scatter(const double* __restrict__ in, const int32_t* __restrict__ perm, int64_t n, int S, int Sp,
                            double* out) {
  BGRID_STRIDE(idx, n * Sp) {
    const int64_t k = idx / Sp;
    const int s = (int)(idx % Sp);
    if (s < S) out[(int64_t)s * n + perm[k]] = in[idx];
  }
}

// column sums (per scenario) in a fixed order: blocks of users, then the partials
__global__ void k_b_colsum(const double* __restrict__ x, int64_t n, int Sp, double* part) {
  __shared__ double sh[256];
  const int s = threadIdx.x % Sp;
  const int lanes = blockDim.x / Sp;
  const int r = threadIdx.x / Sp;
  double acc = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * lanes + r; k < n; k += (int64_t)gridDim.x * lanes) acc += x[k * Sp + s];
  sh[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < Sp) {
    double t = 0.0;
    for (int q = 0; q < lanes; ++q) t += sh[q * Sp + s];
    part[(int64_t)blockIdx.x * Sp + s] = t;
  }
}

// one column of [n][Sp] into a contiguous vector
__global__ void k_b_column(const double* __restrict__ x, int64_t n, int Sp, int s, double* out) {
  BGRID_STRIDE(k, n) out[k] = x[k * Sp + s];
}

}  // namespace

// ------------------------------------------------------------------ the batch object
constexpr int kSp = kSpmmMaxS;  // scenarios are padded to 64 (two per lane)

struct Batch {
  Graph g;          // the shared follower structure (built with scenario 0's rates)
  int32_t S = 0;
  // per-user, per-scenario constants, user-major [n][kSp]
  DBuf<double> c64, mu64, isig64, lam64, d64;
  DBuf<float> mu32, isig32, c32;
  DBuf<double> scale;   // [kSp] gap scale of each scenario
  DBuf<double> bnorm;   // [kSp] ||B||_inf of each scenario
  // iteration state
  DBuf<double> s64, psi;          // [n][kSp]
  DBuf<double> u64a, u64b;        // [nu + 1][kSp]
  DBuf<float> v0, va, vb;         // [nu + 1][kSp]
  DBuf<int32_t> active, iters, phase_it, ok, converged;  // phase_it: steps of the current series phase
  DBuf<double> gap_last;
  DBuf<BatchState> state;
  BatchState* host = nullptr;
  // chunk schedule of the shared product
  Schedule sched;
  DBuf<float2> carry_head, carry_tail;
  DBuf<double2> carry_head64, carry_tail64;
  DBuf<double> gap_part, gap_fix;
  DBuf<double> gap_chunk;      // [chunks][S] per-chunk gaps of the FP32 product
  DBuf<int32_t> chunk_ctr;     // its chunk claims {claimed, warps done}
  int grid = 0, fgrid = 0;
  bool solved = false;
};

// Per-scenario sigma, beta and constants, formed while the follower-grouped CSR exists.
struct BatchHook final : BuildHook {
  Batch& b;
  const double* lamS;  // [S][n] input order, device
  const double* muS;
  explicit BatchHook(Batch& bb, const double* l, const double* m) : b(bb), lamS(l), muS(m) {}

  bool follower_csr() const override { return true; }  // one product per scenario over it
  void on_follower_csr(Graph& g, const FollowerCsr& fc) override { form(g, &fc); }

  void form(Graph& g, const FollowerCsr* fc) {
    Allocator& al = g.al;
    cudaStream_t s = g.stream;
    const int64_t n = g.n;
    const int S = b.S;
    DBuf<double> lam_s(al, (size_t)n), mu_s(al, (size_t)n), sig(al, (size_t)n), bet(al, (size_t)n);
    DBuf<double> cS(al, (size_t)S * n), dS(al, (size_t)S * n), iS(al, (size_t)S * n), lS(al, (size_t)S * n),
        mS(al, (size_t)S * n);
    DBuf<D2> w(al, (size_t)n + 1);
    DBuf<unsigned long long> bn(al, kSp);
    PSI_CUDA(cudaMemsetAsync(bn.get(), 0, kSp * sizeof(unsigned long long), s));
    for (int q = 0; q < S; ++q) {
      k_b_permute<<<bgrid(n), 256, 0, s>>>(lamS + (int64_t)q * n, g.perm.get(), n, lam_s.get());
      PSI_LAUNCHED();
      k_b_permute<<<bgrid(n), 256, 0, s>>>(muS + (int64_t)q * n, g.perm.get(), n, mu_s.get());
      PSI_LAUNCHED();
      PSI_CUDA(cudaMemsetAsync(sig.get(), 0, sizeof(double) * n, s));
      PSI_CUDA(cudaMemsetAsync(bet.get(), 0, sizeof(double) * n, s));
      if (fc) {
        k_b_weights<<<bgrid(n + 1), 256, 0, s>>>(lam_s.get(), mu_s.get(), n, w.get());
        PSI_LAUNCHED();
        run_store_product(fc->row_ptr, fc->col, *fc->sched, fc->n_rows, fc->m, w.get(),
                          EpiStore2{sig.get(), bet.get(), g.nX, g.nR}, al, s);
      }
      k_b_consts<<<bgrid(n), 256, 0, s>>>(lam_s.get(), mu_s.get(), sig.get(), bet.get(), n, cS.get() + q * n,
                                          dS.get() + q * n, iS.get() + q * n, bn.get() + q);
      PSI_LAUNCHED();
      PSI_CUDA(cudaMemcpyAsync(lS.get() + q * n, lam_s.get(), sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      PSI_CUDA(cudaMemcpyAsync(mS.get() + q * n, mu_s.get(), sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    }
    const size_t nS = (size_t)n * kSp;
    b.c64.reset(al, nS);
    b.d64.reset(al, nS);
    b.isig64.reset(al, nS);
    b.lam64.reset(al, nS);
    b.mu64.reset(al, nS);
    b.c32.reset(al, nS);
    b.mu32.reset(al, nS);
    b.isig32.reset(al, nS);
    dim3 tg((unsigned)ceil_div(n, 32), kSp / 32);
    // padding scenarios: lambda = 1, mu = 0 (c = 0, d = 1): harmless and never reported
    k_b_transpose<double, double><<<tg, 256, 0, s>>>(cS.get(), S, kSp, n, b.c64.get(), 0.0);
    k_b_transpose<double, double><<<tg, 256, 0, s>>>(dS.get(), S, kSp, n, b.d64.get(), 1.0);
    k_b_transpose<double, double><<<tg, 256, 0, s>>>(iS.get(), S, kSp, n, b.isig64.get(), 0.0);
    k_b_transpose<double, double><<<tg, 256, 0, s>>>(lS.get(), S, kSp, n, b.lam64.get(), 1.0);
    k_b_transpose<double, double><<<tg, 256, 0, s>>>(mS.get(), S, kSp, n, b.mu64.get(), 0.0);
    k_b_transpose<float, double><<<tg, 256, 0, s>>>(cS.get(), S, kSp, n, b.c32.get(), 0.f);
    k_b_transpose<float, double><<<tg, 256, 0, s>>>(mS.get(), S, kSp, n, b.mu32.get(), 0.f);
    k_b_transpose<float, double><<<tg, 256, 0, s>>>(iS.get(), S, kSp, n, b.isig32.get(), 0.f);
    for (int t = 0; t < 7; ++t) count_launch();
    PSI_LAUNCHED();
    unsigned long long hb[kSp];
    PSI_CUDA(cudaMemcpyAsync(hb, bn.get(), sizeof(hb), cudaMemcpyDeviceToHost, s));
    PSI_CUDA(cudaStreamSynchronize(s));
    double bnv[kSp];
    std::memcpy(bnv, hb, sizeof(bnv));
    double sc[kSp];
    for (int q = 0; q < kSp; ++q) {
      const double bnorm_q = g.opt.bnorm_mode == PSI_BNORM_INF ? bnv[q] : 1.0;
      sc[q] = bnorm_q * (g.opt.tol_mode == PSI_TOL_PSI ? 1.0 / (double)n : 1.0);
    }
    b.bnorm.reset(al, kSp);
    b.scale.reset(al, kSp);
    PSI_CUDA(cudaMemcpyAsync(b.bnorm.get(), bnv, sizeof(bnv), cudaMemcpyHostToDevice, s));
    PSI_CUDA(cudaMemcpyAsync(b.scale.get(), sc, sizeof(sc), cudaMemcpyHostToDevice, s));
    PSI_CUDA(cudaStreamSynchronize(s));
    formed = true;
  }
  bool formed = false;
};

namespace {

void batch_buffers(Batch& b) {
  Graph& g = b.g;
  Allocator& al = g.al;
  const size_t n = (size_t)g.n;
  const size_t nu = (size_t)g.nX + (size_t)g.nU;
  b.s64.reset(al, n * kSp);
  b.psi.reset(al, n * kSp);
  b.u64a.reset(al, (nu + 1) * kSp);
  b.u64b.reset(al, (nu + 1) * kSp);
  b.v0.reset(al, (nu + 1) * kSp);
  b.va.reset(al, (nu + 1) * kSp);
  b.vb.reset(al, (nu + 1) * kSp);
  b.active.reset(al, kSp);
  b.iters.reset(al, kSp);
  b.phase_it.reset(al, kSp);
  b.ok.reset(al, kSp);
  b.converged.reset(al, kSp);
  b.gap_last.reset(al, kSp);
  b.state.reset(al, 1);
  if (!b.host) PSI_CUDA(cudaMallocHost((void**)&b.host, 2 * sizeof(BatchState)));
  b.sched = make_schedule(g.row_ptr.get(), g.n_rows, g.m_unique, al, g.stream, kSpmmChunk);
  const size_t nc = (size_t)(b.sched.tiles > 0 ? b.sched.tiles : 1);
  b.carry_head.reset(al, nc * 32);
  b.carry_tail.reset(al, nc * 32);
  b.carry_head64.reset(al, nc * 32);
  b.carry_tail64.reset(al, nc * 32);
  int per_sm = 0;
  PSI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm_claims<EpiSeriesS>, 256, 0));
  b.grid = (int)num_sms() * (per_sm > 0 ? per_sm : 1);
  b.fgrid = (int)num_sms() * 2;

  b.gap_part.reset(al, (size_t)b.grid * 8 * kSp);
  b.gap_fix.reset(al, (size_t)b.fgrid * 8 * kSp);
  b.gap_chunk.reset(al, nc * kSp);
  b.chunk_ctr.reset(al, 2);
  PSI_CUDA(cudaMemsetAsync(b.chunk_ctr.get(), 0, 2 * sizeof(int32_t), g.stream));
}

SpmmArgs spmm_args(Batch& b) {
  Graph& g = b.g;
  SpmmArgs a{};
  a.row_ptr = g.row_ptr.get();
  a.col = g.col.get();  // padded to a multiple of kSpmvTileMax nonzeros, a multiple of the chunk
  a.chunk_row = b.sched.tile_row.get();
  a.num_chunks = b.sched.tiles;
  a.n_rows = g.n_rows;
  a.m = g.m_unique;
  a.S = kSp;
  a.active = b.active.get();
  a.done = reinterpret_cast<const int32_t*>(b.state.get());  // BatchState::done comes first
  a.gap_part = b.gap_part.get();
  a.carry_head = b.carry_head.get();
  a.carry_tail = b.carry_tail.get();
  a.carry_head64 = b.carry_head64.get();
  a.carry_tail64 = b.carry_tail64.get();
  return a;
}

// one step for every active scenario: product, fix-up, per-scenario stop tests.  The FP32
// product claims its chunks at run time; its gaps then reach k_b_finalize through the
// fix-up, which adds the per-chunk gaps in fixed slices and so runs on every such step.
template <typename V, typename Epi>
void batch_step(Batch& b, const V* u, const Epi& epi) {
  cudaStream_t s = b.g.stream;
  SpmmArgs a = spmm_args(b);
  constexpr bool claims = std::is_same<V, float2>::value;
  if (claims) {
    a.chunk_ctr = b.chunk_ctr.get();
    a.gap_chunk = b.gap_chunk.get();
  }
  int ngp = 0, ngf = 0;
  if (a.num_chunks > 0) {
    if constexpr (claims) k_spmm_claims<Epi><<<b.grid, 256, 0, s>>>(a, u, epi);
    else k_spmm<V, Epi><<<b.grid, 256, 0, s>>>(a, u, epi);
    PSI_LAUNCHED();
    ngp = claims ? 0 : b.grid * 8;
  }
  if (b.sched.num_fix > 0 || (claims && a.num_chunks > 0)) {
    k_spmm_fixup<V, Epi><<<b.fgrid, 256, 0, s>>>(a, b.sched.fix_tile.get(), b.sched.num_fix, b.gap_fix.get(), epi);
    PSI_LAUNCHED();
    ngf = b.fgrid * 8;
  }
  k_b_finalize<<<1, 1024, 0, s>>>(b.state.get(), b.active.get(), b.iters.get(), b.phase_it.get(), b.ok.get(),
                                  b.converged.get(),
                                  b.gap_last.get(), b.scale.get(), b.gap_part.get(), ngp, b.gap_fix.get(), ngf, kSp);
  PSI_LAUNCHED();
}

void set_state(Batch& b, int mode, int max_iter, double eps) {
  BatchState h{};
  h.done = 0;
  h.mode = mode;
  h.max_iter = max_iter;
  h.eps = eps;
  b.host[0] = h;
  PSI_CUDA(cudaMemcpyAsync(b.state.get(), b.host, sizeof(BatchState), cudaMemcpyHostToDevice, b.g.stream));
  PSI_CUDA(cudaStreamSynchronize(b.g.stream));
}

template <typename T>
void read_vec(std::vector<T>& h, const T* d, size_t k, cudaStream_t s) {
  h.resize(k);
  PSI_CUDA(cudaMemcpyAsync(h.data(), d, sizeof(T) * k, cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

psi_status batch_solve(Batch& b, double eps, int32_t max_iter, psi_solve_info* info) {
  NvtxRange nvtx_range("psi_batch_solve");
  PSI_REQUIRE(max_iter >= 0 && !std::isnan(eps), PSI_ERR_INVALID_ARG, "bad eps or max_iter");
  Graph& g = b.g;
  cudaStream_t s = g.stream;
  const int64_t n = g.n;
  const int32_t nX = g.nX, nR = g.nR;
  const int64_t nu = (int64_t)g.nX + g.nU;
  const int S = b.S;
  // float pairs in the confirming and final products when every scenario's tolerance is far
  // above their rounding (as in the single-graph path), FP64 otherwise
  bool pairs = true;
  {
    std::vector<double> sc;
    read_vec(sc, b.scale.get(), kSp, s);
    for (int q = 0; q < S; ++q) pairs = pairs && eps / sc[q] >= std::ldexp(1.0, -30) * (double)n;
  }
  auto to_u = [&](double* dst, const double* src, int64_t lo, int64_t hi) {
    if (hi <= lo) return;
    if (pairs)
      k_b_to_u_g<DF><<<bgrid((hi - lo) * kSp), 256, 0, s>>>(reinterpret_cast<DF*>(dst), src, b.isig64.get(), nX, nR,
                                                             lo, hi, kSp);
    else
      k_b_to_u_g<double><<<bgrid((hi - lo) * kSp), 256, 0, s>>>(dst, src, b.isig64.get(), nX, nR, lo, hi, kSp);
    PSI_LAUNCHED();
  };
  cudaEvent_t t0, t1;
  PSI_CUDA(cudaEventCreate(&t0));
  PSI_CUDA(cudaEventCreate(&t1));
  PSI_CUDA(cudaEventRecord(t0, s));
  // s_0 = c; v_0 = c / sigma; later series terms of U users are 0; U's FP64 u = c / sigma
  PSI_CUDA(cudaMemcpyAsync(b.s64.get(), b.c64.get(), sizeof(double) * n * kSp, cudaMemcpyDeviceToDevice, s));
  const int64_t nuS = (nu + 1) * kSp;
  k_b_fill<float><<<bgrid(nuS), 256, 0, s>>>(b.v0.get(), nuS, 0.f);
  k_b_fill<float><<<bgrid(nuS), 256, 0, s>>>(b.va.get(), nuS, 0.f);
  k_b_fill<float><<<bgrid(nuS), 256, 0, s>>>(b.vb.get(), nuS, 0.f);
  k_b_fill<double><<<bgrid(nuS), 256, 0, s>>>(b.u64a.get(), nuS, 0.0);
  k_b_fill<double><<<bgrid(nuS), 256, 0, s>>>(b.u64b.get(), nuS, 0.0);
  for (int t = 0; t < 4; ++t) count_launch();
  PSI_LAUNCHED();
  k_b_to_u<float, float><<<bgrid(nu * kSp), 256, 0, s>>>(b.v0.get(), b.c32.get(), b.isig32.get(), nX, nR, 0, nu, kSp);
  PSI_LAUNCHED();
  to_u(b.u64a.get(), b.c64.get(), nX, nu);
  to_u(b.u64b.get(), b.c64.get(), nX, nu);
  std::vector<int32_t> act(kSp, 0);
  for (int q = 0; q < S; ++q) act[q] = 1;
  PSI_CUDA(cudaMemcpyAsync(b.active.get(), act.data(), sizeof(int32_t) * kSp, cudaMemcpyHostToDevice, s));
  PSI_CUDA(cudaMemsetAsync(b.iters.get(), 0, sizeof(int32_t) * kSp, s));
  PSI_CUDA(cudaMemsetAsync(b.converged.get(), 0, sizeof(int32_t) * kSp, s));
  PSI_CUDA(cudaMemsetAsync(b.gap_last.get(), 0, sizeof(double) * kSp, s));
  const bool iterate = (1.0 > eps) && max_iter > 0;
  int cur_u = 0;
  bool u_current = false;
  bool v0_u_cleared = false;
  int refinements = 0;
  double* ub[2] = {b.u64a.get(), b.u64b.get()};
  float* vb[2] = {b.va.get(), b.vb.get()};
  std::vector<int32_t> h_conv, h_iters, h_ok;
  const int batch = 4;
  // profile: CUDA events around every FP32 series product; only the steps some scenario
  // executed are counted (launches queued past the stop test exit at once)
  const bool prof = g.opt.profile != 0;
  std::vector<cudaEvent_t> pev;
  double series_ms = 0.0;
  int32_t series_timed = 0;
  while (iterate) {
    // FP32 series for the scenarios still active (Eq. 13), terms summed into s64
    PSI_CUDA(cudaMemsetAsync(b.ok.get(), 0, sizeof(int32_t) * kSp, s));
    PSI_CUDA(cudaMemsetAsync(b.phase_it.get(), 0, sizeof(int32_t) * kSp, s));
    set_state(b, 0, max_iter, eps);
    int k = 0;
    for (;;) {
      for (int i = 0; i < batch; ++i, ++k) {
        EpiSeriesS e{reinterpret_cast<const float2*>(b.mu32.get()), reinterpret_cast<const float2*>(b.isig32.get()),
                     reinterpret_cast<double2*>(b.s64.get()), reinterpret_cast<float2*>(vb[k & 1]), nX};
        const float* vin = k == 0 ? b.v0.get() : vb[(k + 1) & 1];
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (prof) {
          PSI_CUDA(cudaEventCreate(&e0));
          PSI_CUDA(cudaEventCreate(&e1));
          PSI_CUDA(cudaEventRecord(e0, s));
        }
        batch_step<float2, EpiSeriesS>(b, reinterpret_cast<const float2*>(vin), e);
        if (prof) {
          PSI_CUDA(cudaEventRecord(e1, s));
          pev.push_back(e0);
          pev.push_back(e1);
        }
      }
      PSI_CUDA(cudaMemcpyAsync(b.host, b.state.get(), sizeof(BatchState), cudaMemcpyDeviceToHost, s));
      PSI_CUDA(cudaStreamSynchronize(s));
      if (b.host[0].done) break;
    }
    if (prof) {
      std::vector<int32_t> ph;
      read_vec(ph, b.phase_it.get(), kSp, s);
      int32_t ran = 0;
      for (int q = 0; q < S; ++q) ran = ph[q] > ran ? ph[q] : ran;
      for (size_t i = 0; i + 1 < pev.size(); i += 2) {
        if ((int32_t)(i / 2) < ran) {
          float e = 0.f;
          PSI_CUDA(cudaEventElapsedTime(&e, pev[i], pev[i + 1]));
          series_ms += e;
          ++series_timed;
        }
        cudaEventDestroy(pev[i]);
        cudaEventDestroy(pev[i + 1]);
      }
      pev.clear();
    }
    u_current = false;
    read_vec(h_ok, b.ok.get(), kSp, s);
    read_vec(h_iters, b.iters.get(), kSp, s);
    read_vec(h_conv, b.converged.get(), kSp, s);
    // one FP64 step for every scenario whose series met eps; its gap decides
    std::vector<int32_t> next(kSp, 0);
    bool any = false;
    for (int q = 0; q < S; ++q)
      if (h_ok[q] && !h_conv[q]) { next[q] = 1; any = true; }
    if (!any) break;
    to_u(ub[cur_u], b.s64.get(), 0, nX);
    if (!v0_u_cleared && g.nU > 0) {
      k_b_fill<float><<<bgrid((int64_t)g.nU * kSp), 256, 0, s>>>(b.v0.get() + (int64_t)nX * kSp, (int64_t)g.nU * kSp,
                                                                0.f);
      PSI_LAUNCHED();
      v0_u_cleared = true;
    }
    PSI_CUDA(cudaMemcpyAsync(b.active.get(), next.data(), sizeof(int32_t) * kSp, cudaMemcpyHostToDevice, s));
    set_state(b, 1, max_iter, eps);
    auto resid = [&](auto tag) {
      using V = decltype(tag);
      EpiResidS<V> e{reinterpret_cast<const double2*>(b.c64.get()), reinterpret_cast<const double2*>(b.mu64.get()),
                     reinterpret_cast<const double2*>(b.isig64.get()), reinterpret_cast<double2*>(b.s64.get()),
                     reinterpret_cast<V*>(ub[cur_u ^ 1]), reinterpret_cast<float2*>(b.v0.get()), nX};
      batch_step<V, EpiResidS<V>>(b, reinterpret_cast<const V*>(ub[cur_u]), e);
    };
    if (pairs) resid(DF2{});
    else resid(double2{});
    ++refinements;
    cur_u ^= 1;
    u_current = true;
    read_vec(h_conv, b.converged.get(), kSp, s);
    read_vec(h_iters, b.iters.get(), kSp, s);
    bool more = false;
    for (int q = 0; q < S; ++q) {
      next[q] = (!h_conv[q] && h_iters[q] < max_iter) ? 1 : 0;
      more = more || next[q];
    }
    if (!more) break;
    PSI_CUDA(cudaMemcpyAsync(b.active.get(), next.data(), sizeof(int32_t) * kSp, cudaMemcpyHostToDevice, s));
  }
  if (!u_current) {
    to_u(ub[cur_u], b.s64.get(), 0, nX);
  }
  // final step of Algorithm 2 for every scenario: psi = (s B + d) / N
  std::vector<int32_t> all(kSp, 1);
  PSI_CUDA(cudaMemcpyAsync(b.active.get(), all.data(), sizeof(int32_t) * kSp, cudaMemcpyHostToDevice, s));
  std::vector<int32_t> it_save;
  read_vec(it_save, b.iters.get(), kSp, s);
  std::vector<double> gap_save;
  read_vec(gap_save, b.gap_last.get(), kSp, s);
  set_state(b, 1, INT32_MAX, -1.0);
  auto final_step = [&](auto tag) {
    using V = decltype(tag);
    EpiFinalS<V> ef{reinterpret_cast<const double2*>(b.lam64.get()), reinterpret_cast<const double2*>(b.d64.get()),
                    reinterpret_cast<double2*>(b.psi.get()), (double)n};
    batch_step<V, EpiFinalS<V>>(b, reinterpret_cast<const V*>(ub[cur_u]), ef);
  };
  if (pairs) final_step(DF2{});
  else final_step(double2{});
  if (g.n_rows < n) {
    k_b_psi_nonrow<<<bgrid((n - g.n_rows) * kSp), 256, 0, s>>>(b.psi.get(), b.d64.get(), g.n_rows, n, kSp);
    PSI_LAUNCHED();
  }
  PSI_CUDA(cudaEventRecord(t1, s));
  // per-scenario sums of psi
  const int cs_blocks = 256;
  DBuf<double> part(g.al, (size_t)cs_blocks * kSp);
  k_b_colsum<<<cs_blocks, 256, 0, s>>>(b.psi.get(), n, kSp, part.get());
  PSI_LAUNCHED();
  std::vector<double> hp;
  read_vec(hp, part.get(), (size_t)cs_blocks * kSp, s);
  float ms = 0.f;
  PSI_CUDA(cudaEventElapsedTime(&ms, t0, t1));
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  read_vec(h_conv, b.converged.get(), kSp, s);
  std::vector<double> bn;
  read_vec(bn, b.bnorm.get(), kSp, s);
  b.solved = true;
  bool all_conv = true;
  for (int q = 0; q < S; ++q) {
    if (!iterate) h_conv[q] = 1;
    all_conv = all_conv && h_conv[q];
    if (info) {
      psi_solve_info& o = info[q];
      std::memset(&o, 0, sizeof(o));
      o.iters = it_save[q];
      o.converged = h_conv[q];
      o.refinements = refinements;
      o.spmv_launches = it_save[q] + 1;
      o.gap_s_l1 = gap_save[q];
      const double sc = (g.opt.bnorm_mode == PSI_BNORM_INF ? bn[q] : 1.0) *
                        (g.opt.tol_mode == PSI_TOL_PSI ? 1.0 / (double)n : 1.0);
      o.gap_scaled = gap_save[q] * sc;
      o.gap_psi_bound = gap_save[q] * bn[q] / (double)n;
      double ps = 0.0;
      for (int c = 0; c < cs_blocks; ++c) ps += hp[(size_t)c * kSp + q];
      o.psi_sum = ps;
      o.ms = ms;
      o.spmv_ms = series_ms;
      o.spmv_timed = series_timed;
    }
  }
  return all_conv ? PSI_OK : PSI_ERR_NOT_CONVERGED;
}

}  // namespace psi

namespace psi {
namespace {

__global__ void k_b_check_rates(const double* __restrict__ lam, const double* __restrict__ mu, int64_t n,
                                uint32_t* bad) {
  uint32_t b = 0;
  BGRID_STRIDE(i, n) {
    const double x = lam[i], y = mu[i];
    if (!(isfinite(x) && isfinite(y) && x >= 0.0 && y >= 0.0 && x + y > 0.0)) b = 1;
  }
  if (b) atomicOr(bad, 1u);
}

template <typename F>
psi_status batch_guard(F&& f) {
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

}  // namespace
}  // namespace psi

struct psi_batch {
  psi::Batch b;
};

extern "C" {

psi_status psi_batch_create(int64_t n, int64_t m, const int32_t* follower, const int32_t* leader, int32_t S,
                            const double* lambda, const double* mu, const psi_options* opt, psi_batch** out) {
  using namespace psi;
  if (out) *out = nullptr;
  psi_batch* h = nullptr;
  psi_status st = batch_guard([&] {
    PSI_REQUIRE(out, PSI_ERR_INVALID_ARG, "out is NULL");
    PSI_REQUIRE(n >= 1 && n < ((int64_t)1 << 31) - 1, PSI_ERR_INVALID_ARG, "n must be in [1, 2^31 - 2]");
    PSI_REQUIRE(m >= 0 && m < ((int64_t)1 << 31) - 1, PSI_ERR_INVALID_ARG, "m must be in [0, 2^31 - 2]");
    PSI_REQUIRE(S >= 1 && S <= kSp, PSI_ERR_INVALID_ARG, "S must be in [1, 64]");
    PSI_REQUIRE(lambda && mu, PSI_ERR_INVALID_ARG, "lambda and mu are required");
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
    h = new psi_batch();
    Graph& g = h->b.g;
    g.opt = o;
    g.stream = static_cast<cudaStream_t>(o.stream);
    g.al.stream = g.stream;
    if (o.allocator) {
      PSI_REQUIRE(o.allocator->alloc && o.allocator->free, PSI_ERR_INVALID_ARG, "allocator callbacks are NULL");
      g.al.user = *o.allocator;
      g.al.has_user = true;
    }
    h->b.S = S;
    // stage every scenario's rates and validate them all
    const size_t bytes = sizeof(double) * (size_t)S * (size_t)n;
    DBuf<double> lam_d, mu_d;
    const double* dl = lambda;
    const double* dm = mu;
    if (!is_device_pointer(lambda)) {
      lam_d.reset(g.al, (size_t)S * n);
      copy_in(lam_d.get(), lambda, bytes, g.stream);
      dl = lam_d.get();
    }
    if (!is_device_pointer(mu)) {
      mu_d.reset(g.al, (size_t)S * n);
      copy_in(mu_d.get(), mu, bytes, g.stream);
      dm = mu_d.get();
    }
    DBuf<uint32_t> bad(g.al, 1);
    PSI_CUDA(cudaMemsetAsync(bad.get(), 0, sizeof(uint32_t), g.stream));
    k_b_check_rates<<<bgrid((int64_t)S * n), 256, 0, g.stream>>>(dl, dm, (int64_t)S * n, bad.get());
    PSI_LAUNCHED();
    uint32_t hb = 0;
    PSI_CUDA(cudaMemcpyAsync(&hb, bad.get(), sizeof(hb), cudaMemcpyDeviceToHost, g.stream));
    PSI_CUDA(cudaStreamSynchronize(g.stream));
    PSI_REQUIRE(!hb, PSI_ERR_BAD_RATE, "lambda/mu must be finite, >= 0, with lambda + mu > 0 in every scenario");
    BatchHook hook(h->b, dl, dm);
    build_graph(g, n, m, follower, leader, dl, dm, &hook);
    if (!hook.formed) hook.form(g, nullptr);  // no edges: sigma = 0 everywhere
    batch_buffers(h->b);
  });
  if (st != PSI_OK) {
    if (h) {
      cudaStreamSynchronize(h->b.g.stream);
      cudaGetLastError();
      if (h->b.host) cudaFreeHost(h->b.host);
      delete h;
    }
    return st;
  }
  *out = h;
  return PSI_OK;
}

psi_status psi_batch_solve(psi_batch* h, double eps, int32_t max_iter, psi_solve_info* info) {
  using namespace psi;
  if (!h) {
    set_last_error("batch is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  psi_status result = PSI_OK;
  psi_status st = batch_guard([&] { result = batch_solve(h->b, eps, max_iter, info); });
  if (st != PSI_OK) return st;
  if (result == PSI_ERR_NOT_CONVERGED) set_last_error("max_iter reached before every scenario met its stop test");
  return result;
}

psi_status psi_batch_scores(const psi_batch* h, double* psi_out) {
  using namespace psi;
  if (!h || !psi_out) {
    set_last_error("batch or output is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  if (!h->b.solved) {
    set_last_error("psi_batch_solve has not produced scores yet");
    return PSI_ERR_NOT_SOLVED;
  }
  return batch_guard([&] {
    Batch& b = const_cast<Batch&>(h->b);
    Graph& g = b.g;
    const int64_t n = g.n;
    const bool dev = is_device_pointer(psi_out);
    DBuf<double> tmp;
    double* dst = psi_out;
    if (!dev) {
      tmp.reset(g.al, (size_t)b.S * n);
      dst = tmp.get();
    }
    k_b_scatter<<<bgrid(n * kSp), 256, 0, g.stream>>>(b.psi.get(), g.perm.get(), n, b.S, kSp, dst);
    PSI_LAUNCHED();
    if (!dev) copy_out(psi_out, dst, sizeof(double) * (size_t)b.S * n, g.stream);
    PSI_CUDA(cudaStreamSynchronize(g.stream));
  });
}

psi_status psi_batch_topk(const psi_batch* h, int32_t k, int32_t* ids_out, double* vals_out) {
  using namespace psi;
  if (!h || !ids_out) {
    set_last_error("batch or ids_out is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  if (!h->b.solved) {
    set_last_error("psi_batch_solve has not produced scores yet");
    return PSI_ERR_NOT_SOLVED;
  }
  if (k < 1 || (int64_t)k > h->b.g.n || k > 65536) {
    set_last_error("k must be in [1, min(n, 65536)]");
    return PSI_ERR_INVALID_ARG;
  }
  return batch_guard([&] {
    Batch& b = const_cast<Batch&>(h->b);
    Graph& g = b.g;
    const int64_t n = g.n;
    const int S = b.S;
    DBuf<double> col(g.al, (size_t)n);
    DBuf<int32_t> di(g.al, (size_t)S * k);
    DBuf<double> dv(g.al, (size_t)S * k);
    for (int q = 0; q < S; ++q) {
      k_b_column<<<bgrid(n), 256, 0, g.stream>>>(b.psi.get(), n, kSp, q, col.get());
      PSI_LAUNCHED();
      topk_raw(col.get(), g.perm.get(), n, k, di.get() + (int64_t)q * k, dv.get() + (int64_t)q * k, g.al, g.stream);
    }
    copy_out(ids_out, di.get(), sizeof(int32_t) * (size_t)S * k, g.stream);
    if (vals_out) copy_out(vals_out, dv.get(), sizeof(double) * (size_t)S * k, g.stream);
    PSI_CUDA(cudaStreamSynchronize(g.stream));
  });
}

psi_status psi_batch_get_stats(const psi_batch* h, psi_graph_stats* st) {
  if (!h || !st) {
    psi::set_last_error("batch or stats is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  psi::fill_graph_stats(h->b.g, st);
  return PSI_OK;
}

void psi_batch_destroy(psi_batch* h) {
  if (!h) return;
  cudaStreamSynchronize(h->b.g.stream);
  if (h->b.host) cudaFreeHost(h->b.host);
  h->b.host = nullptr;
  if (h->b.g.host_state) cudaFreeHost(h->b.g.host_state);
  h->b.g.host_state = nullptr;
  delete h;
  cudaGetLastError();
}

}  // extern "C"
