// topk.cu -- bit-exact ranking: the k largest psi, equal psi by ascending user id.
//
// Every user gets the unique 96-bit key K = (bits(psi) << 32) | (0xFFFFFFFF - id); psi >= 0,
// so the FP64 bit pattern orders like the value.  An MSB-first radix select (12 digits of
// 8 bits) finds the exact k-th largest key K*, the users with K >= K* (exactly k) are
// collected, and a stable LSD radix sort orders them.  After the first two digits the users
// at or above the prefix (typically a few hundred) are compacted into a candidate list, and
// the remaining digits and the collect step run over it.  All counts are integers, so the
// result does not depend on thread timing.
#include <algorithm>

#include "primitives.cuh"
#include "solve.cuh"

namespace psi {

namespace {

constexpr int64_t kTopkCandidates = 1 << 20;  // candidate list of the compacted select

struct SelectState {
  unsigned long long pref_p;  // known top digits of bits(psi)
  uint32_t pref_q;            // known top digits of the id part
  uint32_t k_rem;             // rank still to find among the matching users
  uint32_t count;             // collected users
  uint32_t pad_;
};

// Keys come from the whole ranking (psi and perm; the id part is read only when needed) or
// from a compacted candidate list (p, q).
struct FullSrc {
  const double* psi;
  const int32_t* perm;
  __device__ __forceinline__ void key(int64_t i, bool need_q, uint64_t& p, uint32_t& q) const {
    p = (uint64_t)__double_as_longlong(psi[i]);
    q = need_q ? 0xFFFFFFFFu - (uint32_t)perm[i] : 0u;
  }
};
struct CandSrc {
  const uint64_t* p_;
  const uint32_t* q_;
  __device__ __forceinline__ void key(int64_t i, bool, uint64_t& p, uint32_t& q) const {
    p = p_[i];
    q = q_[i];
  }
};

// does (p, q) match the first `level` digits of the prefix?
__device__ __forceinline__ bool matches(uint64_t p, uint32_t q, const SelectState& st, int level) {
  if (level == 0) return true;
  if (level <= 8) return (p >> (64 - 8 * level)) == (st.pref_p >> (64 - 8 * level));
  if (p != st.pref_p) return false;
  const int lq = level - 8;
  return (q >> (32 - 8 * lq)) == (st.pref_q >> (32 - 8 * lq));
}

__device__ __forceinline__ uint32_t digit_of(uint64_t p, uint32_t q, int level) {
  return level < 8 ? (uint32_t)(p >> (56 - 8 * level)) & 0xFFu : (q >> (24 - 8 * (level - 8))) & 0xFFu;
}

template <typename Src>
__global__ void k_select_histo(Src src, int64_t n, const SelectState* st_p, int level, uint32_t* hist) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const SelectState st = *st_p;
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    int d = 256;
    if (i < n) {
      uint64_t p;
      uint32_t q;
      src.key(i, level >= 8, p, q);
      if (matches(p, q, st, level)) d = (int)digit_of(p, q, level);
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    if (d < 256 && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// The users whose first `level` digits of bits(psi) are at least the prefix's: every user
// above the prefix (all of them rank among the k) and the ones still tied with it.  Appended
// in any order (the selection that follows counts, and the survivors are sorted by key);
// st->count receives how many there are, written only up to `cap`.
__global__ void k_select_compact(const double* __restrict__ psi, const int32_t* __restrict__ perm, int64_t n,
                                 SelectState* st, int level, uint32_t cap, uint64_t* cp, uint32_t* cq) {
  const int sh = 64 - 8 * level;
  const uint64_t pref = st->pref_p >> sh;
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    uint64_t p = 0;
    bool in = false;
    if (i < n) {
      p = (uint64_t)__double_as_longlong(psi[i]);
      in = (p >> sh) >= pref;
    }
    const uint32_t b = __ballot_sync(0xffffffffu, in);
    uint32_t slot0 = 0;
    if (lane == 0 && b) slot0 = atomicAdd(&st->count, (uint32_t)__popc(b));
    slot0 = __shfl_sync(0xffffffffu, slot0, 0);
    if (in) {
      const uint32_t slot = slot0 + __popc(b & ((1u << lane) - 1u));
      if (slot < cap) {
        cp[slot] = p;
        cq[slot] = 0xFFFFFFFFu - (uint32_t)perm[i];
      }
    }
  }
}

// picks the digit holding rank k_rem (counting from the largest) and extends the prefix
__global__ void k_select_choose(SelectState* st, uint32_t* hist, int level) {
  if (threadIdx.x != 0) return;
  uint32_t above = 0;
  int d = 255;
  for (; d > 0; --d) {
    if (above + hist[d] >= st->k_rem) break;
    above += hist[d];
  }
  st->k_rem -= above;
  if (level < 8) st->pref_p |= (unsigned long long)d << (56 - 8 * level);
  else st->pref_q |= (uint32_t)d << (24 - 8 * (level - 8));
  for (int i = 0; i < 256; ++i) hist[i] = 0;
}

template <typename Src>
__global__ void k_select_collect(Src src, int64_t n, SelectState* st, uint32_t k, uint64_t* out_p, uint32_t* out_q) {
  const uint64_t kp = st->pref_p;
  const uint32_t kq = st->pref_q;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t p;
    uint32_t q;
    src.key(i, true, p, q);
    if (p > kp || (p == kp && q >= kq)) {
      uint32_t slot = atomicAdd(&st->count, 1u);
      if (slot < k) {  // exactly k keys qualify; the bound only guards the buffers
        out_p[slot] = p;
        out_q[slot] = q;
      }
    }
  }
}

__global__ void k_iota(uint32_t* x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (uint32_t)i;
}

__global__ void k_gather_u32(const uint32_t* __restrict__ src, const uint32_t* __restrict__ idx, int64_t n,
                             uint32_t* dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}
__global__ void k_gather_u64(const uint64_t* __restrict__ src, const uint32_t* __restrict__ idx, int64_t n,
                             uint64_t* dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}

// ascending (p, q) order -> descending output
__global__ void k_emit(const uint64_t* __restrict__ p, const uint32_t* __restrict__ q, int32_t k, int32_t* ids,
                       double* vals) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
    const int32_t src = k - 1 - i;
    ids[i] = (int32_t)(0xFFFFFFFFu - q[src]);
    if (vals) vals[i] = __longlong_as_double((long long)p[src]);
  }
}

}  // namespace

void topk(const Graph& gc, int32_t k, int32_t* d_ids, double* d_vals) {
  Graph& g = const_cast<Graph&>(gc);
  topk_raw(g.psi64.get(), g.perm.get(), g.n, k, d_ids, d_vals, g.al, g.stream);
}

void topk_raw(const double* psi, const int32_t* perm, int64_t n, int32_t k, int32_t* d_ids, double* d_vals,
              Allocator& al, cudaStream_t s) {
  DBuf<SelectState> st(al, 1);
  DBuf<uint32_t> hist(al, 256);
  SelectState h{};
  h.k_rem = (uint32_t)k;
  PSI_CUDA(cudaMemcpyAsync(st.get(), &h, sizeof(h), cudaMemcpyHostToDevice, s));
  PSI_CUDA(cudaMemsetAsync(hist.get(), 0, 256 * sizeof(uint32_t), s));
  auto grid = [](int64_t len) {
    const int64_t b = ceil_div(len > 0 ? len : 1, 256), cap = num_sms() * 8;
    return (int)(b < cap ? b : cap);
  };
  const FullSrc full{psi, perm};
  DBuf<uint64_t> p0(al, (size_t)k), p1(al, (size_t)k);
  DBuf<uint32_t> q0(al, (size_t)k), q1(al, (size_t)k), i0(al, (size_t)k), i1(al, (size_t)k);
  // the first kFullLevels digits over every user; then, when few users remain tied with the
  // prefix, the rest of the select runs over a compacted candidate list
  constexpr int kFullLevels = 2;
  int level = 0;
  for (; level < kFullLevels; ++level) {
    k_select_histo<FullSrc><<<grid(n), 256, 0, s>>>(full, n, st.get(), level, hist.get());
    PSI_LAUNCHED();
    k_select_choose<<<1, 32, 0, s>>>(st.get(), hist.get(), level);
    PSI_LAUNCHED();
  }
  const uint32_t cand_cap = (uint32_t)std::min<int64_t>(n, std::max<int64_t>(kTopkCandidates, k));
  DBuf<uint64_t> cp(al, cand_cap);
  DBuf<uint32_t> cq(al, cand_cap);
  k_select_compact<<<grid(n), 256, 0, s>>>(psi, perm, n, st.get(), level, cand_cap, cp.get(), cq.get());
  PSI_LAUNCHED();
  SelectState hs{};
  PSI_CUDA(cudaMemcpyAsync(&hs, st.get(), sizeof(hs), cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaStreamSynchronize(s));
  const bool compact = hs.count <= cand_cap;
  const CandSrc cand{cp.get(), cq.get()};
  const int64_t nc = compact ? (int64_t)hs.count : n;
  hs.count = 0;  // the collect step counts again
  PSI_CUDA(cudaMemcpyAsync(st.get(), &hs, sizeof(hs), cudaMemcpyHostToDevice, s));
  for (; level < 12; ++level) {
    if (compact) k_select_histo<CandSrc><<<grid(nc), 256, 0, s>>>(cand, nc, st.get(), level, hist.get());
    else k_select_histo<FullSrc><<<grid(nc), 256, 0, s>>>(full, nc, st.get(), level, hist.get());
    PSI_LAUNCHED();
    k_select_choose<<<1, 32, 0, s>>>(st.get(), hist.get(), level);
    PSI_LAUNCHED();
  }
  if (compact) k_select_collect<CandSrc><<<grid(nc), 256, 0, s>>>(cand, nc, st.get(), (uint32_t)k, p0.get(), q0.get());
  else k_select_collect<FullSrc><<<grid(nc), 256, 0, s>>>(full, nc, st.get(), (uint32_t)k, p0.get(), q0.get());
  PSI_LAUNCHED();
  // stable LSD order: by q, then by p (payload = position)
  const int eb = (int)ceil_div(k, 256);
  k_iota<<<eb, 256, 0, s>>>(i0.get(), k);
  PSI_LAUNCHED();
  DBuf<uint32_t> qk0(al, (size_t)k), qk1(al, (size_t)k);
  PSI_CUDA(cudaMemcpyAsync(qk0.get(), q0.get(), sizeof(uint32_t) * k, cudaMemcpyDeviceToDevice, s));
  bool alt = radix_sort<uint32_t>(qk0.get(), qk1.get(), i0.get(), i1.get(), k, 32, al, s);
  const uint32_t* ord = alt ? i1.get() : i0.get();
  // p and q in q-order
  k_gather_u64<<<eb, 256, 0, s>>>(p0.get(), ord, k, p1.get());
  PSI_LAUNCHED();
  k_gather_u32<<<eb, 256, 0, s>>>(q0.get(), ord, k, q1.get());
  PSI_LAUNCHED();
  DBuf<uint32_t> j0(al, (size_t)k), j1(al, (size_t)k);
  k_iota<<<eb, 256, 0, s>>>(j0.get(), k);
  PSI_LAUNCHED();
  PSI_CUDA(cudaMemcpyAsync(p0.get(), p1.get(), sizeof(uint64_t) * k, cudaMemcpyDeviceToDevice, s));
  bool alt2 = radix_sort<uint64_t>(p0.get(), p1.get(), j0.get(), j1.get(), k, 64, al, s);
  const uint64_t* ps = alt2 ? p1.get() : p0.get();
  const uint32_t* ord2 = alt2 ? j1.get() : j0.get();
  // q1 is in q-order; reorder by ord2
  k_gather_u32<<<eb, 256, 0, s>>>(q1.get(), ord2, k, q0.get());
  PSI_LAUNCHED();
  k_emit<<<eb, 256, 0, s>>>(ps, q0.get(), k, d_ids, d_vals);
  PSI_LAUNCHED();
}

}  // namespace psi
