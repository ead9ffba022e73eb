// topk.cu -- bit-exact ranking: the k largest psi, equal psi by ascending user id.
//
// Every user gets the unique 96-bit key K = (bits(psi) << 32) | (0xFFFFFFFF - id); psi >= 0,
// so the FP64 bit pattern orders like the value.  An MSB-first radix select (12 digits of
// 8 bits) finds the exact k-th largest key K*, the users with K >= K* (exactly k) are
// collected, and a stable LSD radix sort orders them.  All counts are integers, so the
// result does not depend on thread timing.
#include "primitives.cuh"
#include "solve.cuh"

namespace psi {

namespace {

struct SelectState {
  unsigned long long pref_p;  // known top digits of bits(psi)
  uint32_t pref_q;            // known top digits of the id part
  uint32_t k_rem;             // rank still to find among the matching users
  uint32_t count;             // collected users
  uint32_t pad_;
};

__device__ __forceinline__ void key_of(const double* psi, const int32_t* perm, int64_t i, uint64_t& p, uint32_t& q) {
  p = (uint64_t)__double_as_longlong(psi[i]);
  q = 0xFFFFFFFFu - (uint32_t)perm[i];
}

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

__global__ void k_select_histo(const double* __restrict__ psi, const int32_t* __restrict__ perm, int64_t n,
                               const SelectState* st_p, int level, uint32_t* hist) {
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
      key_of(psi, perm, i, p, q);
      if (matches(p, q, st, level)) d = (int)digit_of(p, q, level);
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    if (d < 256 && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
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

__global__ void k_select_collect(const double* __restrict__ psi, const int32_t* __restrict__ perm, int64_t n,
                                 SelectState* st, uint32_t k, uint64_t* out_p, uint32_t* out_q) {
  const uint64_t kp = st->pref_p;
  const uint32_t kq = st->pref_q;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t p;
    uint32_t q;
    key_of(psi, perm, i, p, q);
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
  int64_t blocks = ceil_div(n, 256);
  const int64_t cap = num_sms() * 8;
  if (blocks > cap) blocks = cap;
  for (int level = 0; level < 12; ++level) {
    k_select_histo<<<(int)blocks, 256, 0, s>>>(psi, perm, n, st.get(), level, hist.get());
    PSI_LAUNCHED();
    k_select_choose<<<1, 32, 0, s>>>(st.get(), hist.get(), level);
    PSI_LAUNCHED();
  }
  DBuf<uint64_t> p0(al, (size_t)k), p1(al, (size_t)k);
  DBuf<uint32_t> q0(al, (size_t)k), q1(al, (size_t)k), i0(al, (size_t)k), i1(al, (size_t)k);
  k_select_collect<<<(int)blocks, 256, 0, s>>>(psi, perm, n, st.get(), (uint32_t)k, p0.get(), q0.get());
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
