// powernf.cu -- Power-NF (Algorithm 1) on the GPU for small graphs: the method Power-psi
// replaces, with every origin's newsfeed vector stepped at once.
//
// For an origin i, the vector p_i over users j (the share of j's newsfeed that holds i's
// posts) solves p_i = A p_i + b_i (Eq. 8), with a_jk = mu_k / sigma_j and b_ji = lambda_i /
// sigma_j for leaders k, i of j (Sec. II).  Algorithm 1 iterates p_i <- A p_i + b_i from
// p_i = b_i until ||p_i^t - p_i^{t-1}||_1 <= eps (a gap of 1 before the first step), then
// q_i^(n) = c_n p_i^(n) + d_i 1{n = i} (Eq. 7) and psi_i = (1/N) sum_n q_i^(n) (Eq. 1).
//
// Here the N vectors are the columns of an N x N matrix P (row j = user, column i =
// origin), all stepped together: one block per user row j forms sum_k a_jk P[k][:] over j's
// leaders (whole rows of P, read contiguously) plus b_j, and leaves the entries' |change|;
// a column sum gives each origin's gap, and an origin that met its test (or the step cap)
// keeps its column from then on, as Algorithm 1 stops each origin on its own.  Every sum
// runs in a fixed order (leaders in the graph's order, rows in index order): results are
// bit-reproducible.  N up to kNfMaxUsers: the method costs N times Power-psi per step.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "solve.cuh"

namespace psi {

namespace {

constexpr int64_t kNfMaxUsers = 4096;

// P[j][i] = b_ji for every edge (j follows i), 0 elsewhere (P zeroed before)
__global__ void k_nf_init(const int32_t* __restrict__ fptr, const int32_t* __restrict__ lead,
                          const double* __restrict__ b, int64_t n, double* P) {
  const int64_t j = blockIdx.x;
  for (int32_t e = fptr[j] + threadIdx.x; e < fptr[j + 1]; e += blockDim.x) P[j * n + lead[e]] = b[e];
}

// one step of every active origin: Pn[j][i] = sum_{k in L(j)} a_jk P[k][i] + b_ji, and
// part[j][i] = |Pn[j][i] - P[j][i]|; frozen origins copy their column.  Block (j, column
// tile), one column per thread; the leaders' rows are loaded kNfUnroll at a time so that
// the loads overlap, and summed in the graph's order.
constexpr int kNfThreads = 256;
constexpr int kNfUnroll = 8;
__global__ void __launch_bounds__(kNfThreads) k_nf_step(const int32_t* __restrict__ fptr,
                                                        const int32_t* __restrict__ lead, const double* __restrict__ a,
                                                        const double* __restrict__ b,
                                                        const int32_t* __restrict__ active, int64_t n,
                                                        const double* __restrict__ P, double* __restrict__ Pn,
                                                        double* __restrict__ part) {
  const int64_t j = blockIdx.x;
  const int64_t i = (int64_t)blockIdx.y * kNfThreads + threadIdx.x;
  if (i >= n) return;
  const double old = P[j * n + i];
  if (!active[i]) {
    Pn[j * n + i] = old;
    part[j * n + i] = 0.0;
    return;
  }
  const int32_t e0 = fptr[j], e1 = fptr[j + 1];
  double acc = 0.0, bji = 0.0;
  for (int32_t e = e0; e < e1; e += kNfUnroll) {
    double x[kNfUnroll];
#pragma unroll
    for (int q = 0; q < kNfUnroll; ++q) x[q] = e + q < e1 ? P[(int64_t)lead[e + q] * n + i] : 0.0;
#pragma unroll
    for (int q = 0; q < kNfUnroll; ++q) {
      if (e + q < e1) {
        acc += a[e + q] * x[q];
        if (lead[e + q] == i) bji = b[e + q];
      }
    }
  }
  const double v = acc + bji;
  Pn[j * n + i] = v;
  part[j * n + i] = fabs(v - old);
}

// gap of every active origin (rows in order), its step count and stop test; active_count
// receives the origins still stepping
__global__ void k_nf_gap(const double* __restrict__ part, int64_t n, double eps, int32_t max_iter, int32_t* active,
                         int32_t* steps, double* gap, int32_t* converged, int32_t* active_count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!active[i]) continue;
    double g = 0.0;
    for (int64_t j = 0; j < n; ++j) g += part[j * n + i];
    gap[i] = g;
    steps[i] += 1;
    if (g <= eps) {
      active[i] = 0;
      converged[i] = 1;
    } else if (steps[i] >= max_iter) {
      active[i] = 0;
    } else {
      atomicAdd(active_count, 1);
    }
  }
}

// psi_i = (sum_n c_n P[n][i] + d_i) / N, rows in order, into input order
__global__ void k_nf_psi(const double* __restrict__ P, const double* __restrict__ c, const double* __restrict__ d,
                         const int32_t* __restrict__ perm, int64_t n, double* psi) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double q = 0.0;
    for (int64_t j = 0; j < n; ++j) q += c[j] * P[j * n + i];
    psi[perm[i]] = (q + d[i]) / (double)n;
  }
}

int nf_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), num_sms() * 4)); }

}  // namespace

psi_status power_nf(Graph& g, double eps, int32_t max_iter, double* psi_out, psi_solve_info* info) {
  const int64_t n = g.n;
  PSI_REQUIRE(n <= kNfMaxUsers, PSI_ERR_INVALID_ARG, "psi_power_nf: at most 4096 users (N x N state)");
  PSI_REQUIRE(max_iter >= 0 && !std::isnan(eps), PSI_ERR_INVALID_ARG, "bad eps or max_iter");
  if (n == 0) {
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->converged = 1;
    }
    return PSI_OK;
  }
  cudaStream_t s = g.stream;
  Allocator& al = g.al;
  // the follower-grouped edge list (leaders of each user, internal ids) from the transposed
  // CSR: row r = leader r, entries = its followers' gathered indices
  std::vector<int32_t> rp((size_t)g.n_rows + 1), col((size_t)std::max<int64_t>(g.m_unique, 1));
  std::vector<double> mu((size_t)n), lam((size_t)n), isig((size_t)n);
  if (g.n_rows > 0) {
    PSI_CUDA(cudaMemcpyAsync(rp.data(), g.row_ptr.get(), sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost, s));
    if (g.m_unique > 0)
      PSI_CUDA(cudaMemcpyAsync(col.data(), g.col.get(), sizeof(int32_t) * (size_t)g.m_unique, cudaMemcpyDeviceToHost,
                               s));
  }
  PSI_CUDA(cudaMemcpyAsync(mu.data(), g.mu64.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaMemcpyAsync(lam.data(), g.lam64.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaMemcpyAsync(isig.data(), g.isig64.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaStreamSynchronize(s));
  std::vector<int32_t> deg((size_t)n + 1, 0);
  for (int32_t r = 0; r < g.n_rows; ++r)
    for (int32_t e = rp[r]; e < rp[r + 1]; ++e) {
      const int32_t gi = col[e];
      ++deg[(size_t)(gi < g.nX ? gi : gi + g.nR) + 1];
    }
  std::vector<int32_t> fptr((size_t)n + 1, 0);
  for (int64_t j = 0; j < n; ++j) fptr[j + 1] = fptr[j] + deg[j + 1];
  std::vector<int32_t> lead((size_t)std::max<int64_t>(g.m_unique, 1)), fill(fptr.begin(), fptr.end() - 1);
  std::vector<double> a(lead.size()), b(lead.size());
  for (int32_t r = 0; r < g.n_rows; ++r)  // leaders in increasing internal id for every user
    for (int32_t e = rp[r]; e < rp[r + 1]; ++e) {
      const int32_t gi = col[e];
      const int32_t j = gi < g.nX ? gi : gi + g.nR;
      const int32_t o = fill[j]++;
      lead[o] = r;
      a[o] = mu[r] * isig[j];
      b[o] = lam[r] * isig[j];
    }
  DBuf<int32_t> dptr(al, (size_t)n + 1), dlead(al, lead.size()), active(al, (size_t)n), steps(al, (size_t)n),
      conv(al, (size_t)n), cnt(al, 1);
  DBuf<double> da(al, a.size()), db(al, b.size()), P(al, (size_t)(n * n)), Pn(al, (size_t)(n * n)),
      part(al, (size_t)(n * n)), gap(al, (size_t)n), psi(al, (size_t)n);
  PSI_CUDA(cudaMemcpyAsync(dptr.get(), fptr.data(), sizeof(int32_t) * fptr.size(), cudaMemcpyHostToDevice, s));
  PSI_CUDA(cudaMemcpyAsync(dlead.get(), lead.data(), sizeof(int32_t) * lead.size(), cudaMemcpyHostToDevice, s));
  PSI_CUDA(cudaMemcpyAsync(da.get(), a.data(), sizeof(double) * a.size(), cudaMemcpyHostToDevice, s));
  PSI_CUDA(cudaMemcpyAsync(db.get(), b.data(), sizeof(double) * b.size(), cudaMemcpyHostToDevice, s));
  PSI_CUDA(cudaMemsetAsync(P.get(), 0, sizeof(double) * (size_t)(n * n), s));
  PSI_CUDA(cudaMemsetAsync(steps.get(), 0, sizeof(int32_t) * n, s));
  PSI_CUDA(cudaMemsetAsync(conv.get(), 0, sizeof(int32_t) * n, s));
  // Algorithm 1 starts each origin with gap = 1: eps >= 1 (or max_iter = 0) takes no step
  const bool iterate = 1.0 > eps && max_iter > 0;
  std::vector<int32_t> on((size_t)n, iterate ? 1 : 0);
  PSI_CUDA(cudaMemcpyAsync(active.get(), on.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
  cudaEvent_t t0, t1;
  PSI_CUDA(cudaEventCreate(&t0));
  PSI_CUDA(cudaEventCreate(&t1));
  PSI_CUDA(cudaEventRecord(t0, s));
  k_nf_init<<<(unsigned)n, 128, 0, s>>>(dptr.get(), dlead.get(), db.get(), n, P.get());
  PSI_LAUNCHED();
  int32_t t = 0;
  double* cur = P.get();
  double* nxt = Pn.get();
  // every origin steps at most max_iter times, so max_iter launches end the loop
  while (iterate && t < max_iter) {
    PSI_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t), s));
    k_nf_step<<<dim3((unsigned)n, (unsigned)ceil_div(n, kNfThreads)), kNfThreads, 0, s>>>(
        dptr.get(), dlead.get(), da.get(), db.get(), active.get(), n, cur, nxt, part.get());
    PSI_LAUNCHED();
    k_nf_gap<<<nf_grid(n), 256, 0, s>>>(part.get(), n, eps, max_iter, active.get(), steps.get(), gap.get(),
                                        conv.get(), cnt.get());
    PSI_LAUNCHED();
    std::swap(cur, nxt);
    ++t;
    int32_t left = 0;
    PSI_CUDA(cudaMemcpyAsync(&left, cnt.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PSI_CUDA(cudaStreamSynchronize(s));
    if (left == 0) break;
  }
  k_nf_psi<<<nf_grid(n), 256, 0, s>>>(cur, g.c64.get(), g.d64.get(), g.perm.get(), n, psi.get());
  PSI_LAUNCHED();
  PSI_CUDA(cudaEventRecord(t1, s));
  if (psi_out) copy_out(psi_out, psi.get(), sizeof(double) * n, s);
  std::vector<int32_t> hs((size_t)n), hc((size_t)n);
  std::vector<double> hg((size_t)n);
  PSI_CUDA(cudaMemcpyAsync(hs.data(), steps.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaMemcpyAsync(hc.data(), conv.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaMemcpyAsync(hg.data(), gap.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaStreamSynchronize(s));
  float ms = 0.f;
  PSI_CUDA(cudaEventElapsedTime(&ms, t0, t1));
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  int64_t matvecs = 0;
  int32_t most = 0;
  bool all = true;
  double worst = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    matvecs += hs[i];
    most = std::max(most, hs[i]);
    all = all && (hc[i] || (hs[i] == 0 && 1.0 <= eps));  // no step: the starting gap of 1 decides
    if (hs[i] > 0) worst = std::max(worst, hg[i]);
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = most;
    info->converged = all ? 1 : 0;
    info->spmv_launches = (int32_t)std::min<int64_t>(matvecs, INT32_MAX);  // matrix-vector products
    info->gap_s_l1 = worst;
    info->gap_scaled = worst;
    info->ms = ms;
  }
  return all ? PSI_OK : PSI_ERR_NOT_CONVERGED;
}

}  // namespace psi
