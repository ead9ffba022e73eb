// solve.cuh -- entry points of the Power-psi loop (solve.cu) and ranking (topk.cu).
#pragma once

#include "common.cuh"

namespace psi {

void ensure_iteration_buffers(Graph& g);
psi_status solve(Graph& g, double eps, int32_t max_iter, const double* init_s, psi_solve_info* info);

// The per-user constants one run of the iteration uses (internal order, device): c, mu,
// 1/sigma in FP64 and FP32, lambda and d for the final product.
struct SolveConsts {
  const double *c64, *mu64, *isig64, *lam64, *d64;
  const float *c32, *mu32, *isig32;
};
// scale: the stop test is scale * ||s_t - s_{t-1}||_1 <= eps.  final_psi: out = the final
// product of Algorithm 2 (and the handle's scores are replaced); otherwise out = s itself.
struct SolveTarget {
  double scale;
  double* out;  // internal order, n values
  bool final_psi;
};
SolveConsts graph_consts(const Graph& g);
// Power-NF (Algorithm 1) for every origin at once, small graphs (powernf.cu); psi_out in
// input order (host or device)
psi_status power_nf(Graph& g, double eps, int32_t max_iter, int32_t origins_per_pass, double* psi_out,
                    psi_solve_info* info);
// PageRank power method (Eq. 22) on the graph's follower structure (pagerank.cu)
psi_status pagerank(Graph& g, double alpha, double eps, int32_t max_iter, double* pi_out, psi_solve_info* info);
psi_status solve_with(Graph& g, const SolveConsts& K, const SolveTarget& T, double eps, int32_t max_iter,
                      const double* init_s, psi_solve_info* info);
// top k of psi64 by (psi desc, input id asc); ids/vals device buffers of k entries
void topk(const Graph& g, int32_t k, int32_t* d_ids, double* d_vals);
// the same ranking of any psi vector in internal order (ids reported through perm)
void topk_raw(const double* psi, const int32_t* perm, int64_t n, int32_t k, int32_t* d_ids, double* d_vals,
              Allocator& al, cudaStream_t s);
bool is_device_pointer(const void* p);
// the psi_graph_stats of a built graph (the single-graph, batch and multi-graph handles)
void fill_graph_stats(const Graph& g, psi_graph_stats* st);
// graph build (build.cu); hook (nullable) sees the follower-grouped CSR before it is freed
struct BuildHook;
void build_graph(Graph& g, int64_t n, int64_t m, const int32_t* follower, const int32_t* leader,
                 const double* lambda, const double* mu, BuildHook* hook = nullptr);

}  // namespace psi

// the C ABI's opaque graph handle
struct psi_graph {
  psi::Graph g;
};
