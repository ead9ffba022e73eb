// common.cuh -- internals shared by the CUDA translation units of libpsi_gb300.so:
// error handling, the device allocator, cache-hinted loads, the graph handle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <stdexcept>
#include <string>
#include <vector>

#include "psi.h"

namespace psi {

// ---------------------------------------------------------------- errors
// Internal failures are raised as PsiError and turned into a psi_status at the C ABI.
struct PsiError : std::runtime_error {
  psi_status status;
  PsiError(psi_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

void set_last_error(const std::string& msg);

[[noreturn]] void throw_cuda(cudaError_t e, const char* what, const char* file, int line);

#define PSI_CUDA(call)                                                     \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) ::psi::throw_cuda(e_, #call, __FILE__, __LINE__); \
  } while (0)

// after every kernel launch: count it and surface launch errors
void count_launch();
void count_launches(int64_t k);  // k launches at once (a CUDA graph replay)
#define PSI_LAUNCHED()                                                     \
  do {                                                                     \
    ::psi::count_launch();                                                 \
    cudaError_t e_ = cudaGetLastError();                                   \
    if (e_ != cudaSuccess) ::psi::throw_cuda(e_, "kernel launch", __FILE__, __LINE__); \
  } while (0)

#define PSI_REQUIRE(cond, status, msg)                        \
  do {                                                        \
    if (!(cond)) throw ::psi::PsiError((status), (msg));      \
  } while (0)

// ---------------------------------------------------------------- allocation
// Every device buffer of the library goes through one Allocator (the caller's
// psi_allocator, or cudaMallocAsync on the caller's stream).
struct Allocator {
  psi_allocator user{};
  bool has_user = false;
  cudaStream_t stream = nullptr;
  int64_t live_bytes = 0;

  void* alloc(size_t bytes);
  void free(void* p, size_t bytes);
};

template <typename T>
struct DBuf {
  T* ptr = nullptr;
  size_t count = 0;
  Allocator* al = nullptr;

  DBuf() = default;
  DBuf(Allocator& a, size_t n) { reset(a, n); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : ptr(o.ptr), count(o.count), al(o.al) { o.ptr = nullptr; o.count = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      release();
      ptr = o.ptr; count = o.count; al = o.al;
      o.ptr = nullptr; o.count = 0;
    }
    return *this;
  }
  ~DBuf() { release(); }

  void reset(Allocator& a, size_t n) {
    release();
    al = &a;
    count = n;
    ptr = static_cast<T*>(a.alloc((n > 0 ? n : 1) * sizeof(T)));
  }
  void release() {
    if (ptr && al) al->free(ptr, (count > 0 ? count : 1) * sizeof(T));
    ptr = nullptr;
    count = 0;
  }
  T* get() const { return ptr; }
  size_t bytes() const { return count * sizeof(T); }
};

// ---------------------------------------------------------------- cache-hinted access
// Streams (column indices, per-user constants) are loaded evict-first so the gathered
// iterate, loaded evict-last, keeps its L2 lines.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ int4 ld_stream_v4(const int4* p, uint64_t pol) {
  int4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_gather(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_gather(const double* p, uint64_t pol) {
  double v;
  asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
template <typename T>
__device__ __forceinline__ T ld_stream(const T* p, uint64_t pol);
template <>
__device__ __forceinline__ float ld_stream<float>(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
template <>
__device__ __forceinline__ double ld_stream<double>(const double* p, uint64_t pol) {
  double v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
template <>
__device__ __forceinline__ int ld_stream<int>(const int* p, uint64_t pol) {
  int v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_keep(float* p, float v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_keep(double* p, double v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
}

// 8 column indices (32 bytes) in one 256-bit load, streamed past L1
__device__ __forceinline__ void ld_stream_v8(const int* p, uint64_t pol, int (&c)[8]) {
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
               : "=r"(c[0]), "=r"(c[1]), "=r"(c[2]), "=r"(c[3]), "=r"(c[4]), "=r"(c[5]), "=r"(c[6]), "=r"(c[7])
               : "l"(p), "l"(pol));
}

// ---------------------------------------------------------------- sizes
// One warp sums one tile of `tile` consecutive nonzeros (kSpmvTileMin .. kSpmvTileMax, a
// power of two chosen per graph), in steps of kSpmvStep nonzeros (kSpmvItems per lane: one
// 32-byte index load).  Column arrays are padded to a multiple of kSpmvTileMax.
constexpr int kSpmvThreads = 256;
constexpr int kSpmvWarps = kSpmvThreads / 32;
constexpr int kSpmvItems = 8;
constexpr int kSpmvStep = 32 * kSpmvItems;
constexpr int kSpmvTileMin = 512;
constexpr int kSpmvTileMax = 2048;
static_assert(kSpmvItems == 8, "a lane's row ends are one byte of the tile's bitmap");
static_assert(kSpmvTileMin >= 2 * kSpmvStep && kSpmvTileMax % kSpmvTileMin == 0, "whole steps per tile, two at least");

// ---------------------------------------------------------------- device-side loop state
struct DevState {
  int32_t done;          // the current phase met its stop test (or the step cap)
  int32_t phase_iters;   // steps executed in the current phase
  int32_t total_iters;   // power-iteration steps so far (t)
  int32_t max_iter;      // step cap
  int32_t converged;     // scaled gap <= eps at the last step (or predicted for the next one)
  int32_t predict;       // FP32 series phase: stop one step early when the next gap is predicted to pass
  double eps;            // stop threshold
  double scale;          // gap scale (B_norm, divided by N for the psi tolerance)
  double gap;            // last unscaled gap ||s_t - s_{t-1}||_1
  double gap_scaled;
  double extra_gap;      // added to the next step's gap (warm start: users without followers)
};

// ---------------------------------------------------------------- the graph handle
// Users are renumbered internally into four contiguous classes:
//   X = [0, nX)            users with followers and leaders   (rows, gathered)
//   R = [nX, nX+nR)        users with followers, no leaders   (rows)
//   U = [nX+nR, +nU)       users with leaders, no followers   (gathered, constant)
//   Z = the rest           isolated users                     (psi = d/N)
// Rows of the iteration are [0, n_rows = nX+nR); gathered entries are X and U.
struct Graph {
  Allocator al;
  psi_options opt{};
  cudaStream_t stream = nullptr;
  int64_t n = 0, m_input = 0, m_unique = 0;
  int32_t nX = 0, nR = 0, nU = 0, nZ = 0, n_rows = 0;
  int64_t max_followers = 0;
  double bnorm_inf = 0.0, rho_inf = 0.0, build_ms = 0.0;

  DBuf<int32_t> perm;       // internal -> input id [n]
  DBuf<int32_t> n_leaders;  // leaders of each user (internal order), for model features
  DBuf<int32_t> row_ptr;    // [n_rows + 1]
  DBuf<int32_t> col;        // [m padded to a multiple of kSpmvTileMax]: internal follower id, pad = n
  DBuf<int32_t> tile_row;   // [num_tiles + 1]: row holding the tile's first nnz
  DBuf<int32_t> fix_tile;   // tiles whose first row started in an earlier tile
  int32_t tile = kSpmvTileMax;  // nonzeros per tile of the product
  int32_t num_tiles = 0, num_fix = 0;
  int32_t series_hot = 0;       // gathered entries of the FP32 series product kept in shared memory
  bool tuned = false;           // the autotuner has chosen tile and series_hot
  double tune_ms = 0.0;

  // per-user constants, internal order
  DBuf<double> c64, d64, mu64, lam64, isig64;
  DBuf<float> c32, mu32, isig32;

  // iteration state
  DBuf<double> s64;            // FP64 iterate (REFINE, FP64)
  DBuf<double> s64b;           // second FP64 iterate buffer (FP64 mode)
  DBuf<float> s32a, s32b;      // FP32 iterate (FP32 mode)
  DBuf<double> u64a, u64b;     // gathered FP64 vector s*isig [n+1]
  DBuf<float> u32a, u32b, u32c;// gathered FP32 vectors [n+1]
  DBuf<double> psi64;          // psi, internal order
  DBuf<double> carry_head, carry_tail, gap_part, gap_fix;
  DBuf<double> gap_tile;       // per-tile gaps of the product ([num_tiles])
  DBuf<int32_t> tile_ctr;      // the product's tile claims {claimed, warps done}
  DBuf<DevState> state;
  DevState* host_state = nullptr;  // pinned mirror
  bool solved = false;
  bool allocated_iter = false;
  int last_s_kind = 0;             // 0: s64, 1: s64b, 2: s32a, 3: s32b
};

int64_t num_sms();
__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// copy n elements to device memory `dst` from a host or device pointer
void copy_in(void* dst, const void* src, size_t bytes, cudaStream_t s);
// copy to a host or device pointer
void copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s);

}  // namespace psi
