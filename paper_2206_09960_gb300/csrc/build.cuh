// build.cuh -- pieces of the graph build shared with the scenario-batch path.
#pragma once

#include "common.cuh"
#include "spmv.cuh"

namespace psi {

// Merge-path schedule of a CSR with n_rows non-empty rows and m nonzeros cut in tiles of
// `tile` nonzeros.
struct Schedule {
  DBuf<int32_t> tile_row;  // [tiles + 1]: row holding the tile's first nonzero
  DBuf<int32_t> fix_tile;  // tiles whose first row began in an earlier tile
  int32_t tile = kSpmvTileMax;  // nonzeros per tile
  int32_t tiles = 0;
  int32_t num_fix = 0;
};

Schedule make_schedule(const int32_t* row_ptr, int32_t n_rows, int64_t m, Allocator& al, cudaStream_t s,
                       int32_t tile);

// Per-user pair of sums over a CSR (one load-balanced product and its fix-up), summed in
// FP64 (D2 weights) or as float pairs (DF2 weights).
template <typename W>
void run_store_product(const int32_t* row_ptr, const int32_t* col, const Schedule& sc, int32_t n_rows, int64_t m,
                       const W* w, const EpiStore2& epi, Allocator& al, cudaStream_t s);

// The follower-grouped CSR of a graph under construction: rows are the users with leaders
// (X then U, compact), columns the leaders (internal ids), padded with the id n.
struct FollowerCsr {
  const int32_t* row_ptr;
  const int32_t* col;
  const Schedule* sched;
  int32_t n_rows;
  int64_t m;
};

struct BuildHook {
  virtual ~BuildHook() = default;
  // whether on_follower_csr needs the follower-grouped CSR, which is then always built (the
  // exact leader sums of a single graph do without it)
  virtual bool follower_csr() const { return false; }
  virtual void on_follower_csr(Graph&, const FollowerCsr&) {}
  // sigma and beta of every user (internal order, device), once formed
  virtual void on_leader_sums(Graph&, const double* /*sigma*/, const double* /*beta*/) {}
  // device array of a group id (< 1024) per input user, or nullptr: users of one group stay
  // contiguous inside each class of the renumbering
  virtual const int32_t* user_group() const { return nullptr; }
};

}  // namespace psi
