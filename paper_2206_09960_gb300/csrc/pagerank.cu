// pagerank.cu -- the PageRank power method of Eq. 22 on the Power-psi kernels.
//
// pi_t^T = alpha pi_{t-1}^T W + (1 - alpha)/N 1^T, W = D_out^{-1} L with L_ji = 1 when j
// follows i and D_out the number of leaders (a user without leaders has a zero row, as in
// the paper: no dangling redistribution).  Entry by entry,
//     pi_t(i) = (1 - alpha)/N + alpha * sum_{j follows i} pi_{t-1}(j) / |L(j)|,
// which is the Power-psi iteration s_t = c + mu (.) G(s_{t-1}) with c = (1 - alpha)/N,
// mu = alpha and 1/sigma_j = 1/|L(j)|, and pi = s itself (no final product with B).  So the
// same solve runs with these constants, from pi_0 = 1/N, stopping on the pi-tolerance
// ||pi_t - pi_{t-1}||_1 <= eps, in the handle's precision mode.
#include <cmath>
#include <cstring>

#include "solve.cuh"

namespace psi {

namespace {

__global__ void k_pagerank_consts(const int32_t* __restrict__ n_leaders, int64_t n, double alpha, double c0,
                                  double* c64, double* mu64, double* isig64, float* c32, float* mu32, float* isig32) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = n_leaders[k];
    const double is = d > 0 ? 1.0 / (double)d : 0.0;
    c64[k] = c0;
    mu64[k] = alpha;
    isig64[k] = is;
    c32[k] = (float)c0;
    mu32[k] = (float)alpha;
    isig32[k] = (float)is;
  }
}

__global__ void k_pagerank_fill(double* x, int64_t n, double v) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) x[k] = v;
}

__global__ void k_pagerank_scatter(const double* __restrict__ in, const int32_t* __restrict__ perm, int64_t n,
                                   double* out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    out[perm[k]] = in[k];
}

int pr_grid(int64_t n) {
  int64_t g = ceil_div(n > 0 ? n : 1, 256);
  const int64_t cap = num_sms() * 8;
  return (int)(g < cap ? g : cap);
}

}  // namespace

psi_status pagerank(Graph& g, double alpha, double eps, int32_t max_iter, double* pi_out, psi_solve_info* info) {
  PSI_REQUIRE(alpha >= 0.0 && alpha < 1.0, PSI_ERR_INVALID_ARG, "alpha must be in [0, 1)");
  cudaStream_t s = g.stream;
  const int64_t n = g.n;
  Allocator& al = g.al;
  DBuf<double> c64(al, (size_t)n), mu64(al, (size_t)n), isig64(al, (size_t)n), pi(al, (size_t)n),
      pi0(al, (size_t)n);
  DBuf<float> c32(al, (size_t)n), mu32(al, (size_t)n), isig32(al, (size_t)n);
  const int grid = pr_grid(n);
  k_pagerank_consts<<<grid, 256, 0, s>>>(g.n_leaders.get(), n, alpha, (1.0 - alpha) / (double)n, c64.get(),
                                         mu64.get(), isig64.get(), c32.get(), mu32.get(), isig32.get());
  PSI_LAUNCHED();
  k_pagerank_fill<<<grid, 256, 0, s>>>(pi0.get(), n, 1.0 / (double)n);  // pi_0 = 1/N (any order)
  PSI_LAUNCHED();
  // lambda and d only enter the final product with B, which PageRank does not take
  const SolveConsts K{c64.get(), mu64.get(), isig64.get(), nullptr, nullptr, c32.get(), mu32.get(), isig32.get()};
  const SolveTarget T{1.0, pi.get(), false};
  const psi_status st = solve_with(g, K, T, eps, max_iter, pi0.get(), info);
  if (pi_out) {
    if (is_device_pointer(pi_out)) {
      k_pagerank_scatter<<<grid, 256, 0, s>>>(pi.get(), g.perm.get(), n, pi_out);
      PSI_LAUNCHED();
    } else {
      DBuf<double> tmp(al, (size_t)n);
      k_pagerank_scatter<<<grid, 256, 0, s>>>(pi.get(), g.perm.get(), n, tmp.get());
      PSI_LAUNCHED();
      copy_out(pi_out, tmp.get(), sizeof(double) * (size_t)n, s);
    }
  }
  PSI_CUDA(cudaStreamSynchronize(s));
  return st;
}

}  // namespace psi
