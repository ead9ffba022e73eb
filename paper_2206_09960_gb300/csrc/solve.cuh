// solve.cuh -- entry points of the Power-psi loop (solve.cu) and ranking (topk.cu).
#pragma once

#include "common.cuh"

namespace psi {

void ensure_iteration_buffers(Graph& g);
psi_status solve(Graph& g, double eps, int32_t max_iter, const double* init_s, psi_solve_info* info);
// top k of psi64 by (psi desc, input id asc); ids/vals device buffers of k entries
void topk(const Graph& g, int32_t k, int32_t* d_ids, double* d_vals);
// graph build (build.cu)
void build_graph(Graph& g, int64_t n, int64_t m, const int32_t* follower, const int32_t* leader,
                 const double* lambda, const double* mu);

}  // namespace psi
