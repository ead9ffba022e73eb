// solve.cuh -- entry points of the Power-psi loop (solve.cu) and ranking (topk.cu).
#pragma once

#include "common.cuh"

namespace psi {

void ensure_iteration_buffers(Graph& g);
psi_status solve(Graph& g, double eps, int32_t max_iter, const double* init_s, psi_solve_info* info);
// top k of psi64 by (psi desc, input id asc); ids/vals device buffers of k entries
void topk(const Graph& g, int32_t k, int32_t* d_ids, double* d_vals);
// the same ranking of any psi vector in internal order (ids reported through perm)
void topk_raw(const double* psi, const int32_t* perm, int64_t n, int32_t k, int32_t* d_ids, double* d_vals,
              Allocator& al, cudaStream_t s);
bool is_device_pointer(const void* p);
// graph build (build.cu); hook (nullable) sees the follower-grouped CSR before it is freed
struct BuildHook;
void build_graph(Graph& g, int64_t n, int64_t m, const int32_t* follower, const int32_t* leader,
                 const double* lambda, const double* mu, BuildHook* hook = nullptr);

}  // namespace psi

// the C ABI's opaque graph handle
struct psi_graph {
  psi::Graph g;
};
