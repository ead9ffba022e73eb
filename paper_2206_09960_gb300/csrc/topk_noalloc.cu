// topk_noalloc.cu -- psi_topk_noalloc: the ranking of psi_topk for a psi vector the caller
// owns, without allocating any device memory.
//
// Who needs it: a caller that cannot let a library call cudaMalloc -- for example a serving
// process that reserves all of its device memory up front in its own arena (a late
// cudaMalloc could fail or fragment that budget, and cudaMalloc/cudaFree may synchronise
// the device in the middle of latency-critical work), or a host framework whose allocator
// owns every device byte.  Such a caller already holds psi (e.g. written by psi_scores
// into its own buffer) and its output buffers; this entry point only needs a small, fixed
// working area, which lives in the file-scope device array below.
//
// The working area is shared by every call in the process on a given device and keeps
// the contents of the last call: each call clears what must start at zero.  Calls whose
// work overlaps on the GPU (two streams, or two host threads) race on it and must be
// serialised by the caller.
#include <mutex>

#include "common.cuh"

namespace psi {

namespace {

constexpr int kNoAllocMaxK = 4096;  // largest k accepted

struct NaState {
  unsigned long long pref_p;  // known top digits of bits(psi)
  uint32_t pref_q;            // known top digits of the id part
  uint32_t k_rem;             // rank still to find among the matching users
  uint32_t count;             // collected users
  uint32_t pad_;
};

// layout of the working area
constexpr size_t kOffState = 0;
constexpr size_t kOffHist = 256;
constexpr size_t kOffP = kOffHist + 256 * sizeof(uint32_t);
constexpr size_t kOffQ = kOffP + kNoAllocMaxK * sizeof(uint64_t);
constexpr size_t kScratchBytes = kOffQ + kNoAllocMaxK * sizeof(uint32_t);  // 50,432 bytes

// The working area (held by every device that loads the library, until exit).  Host code
// must not pass this symbol to a kernel: on the host it names a stand-in, not device memory.
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct Scratch {
  NaState* st;
  uint32_t* hist;
  uint64_t* p;
  uint32_t* q;
};

// Order key of psi[i]: unsigned comparison of p follows the numeric order of the values
// (sign bit flipped for values >= 0, all bits flipped for negative ones); -0.0 is ranked as
// +0.0 (adding +0.0 turns it into +0.0) and every NaN as the canonical positive NaN, above
// +infinity.  q = ~i ranks equal values by ascending id.
__device__ __forceinline__ void na_key(const double* psi, int64_t i, uint64_t& p, uint32_t& q) {
  const double v = psi[i] + 0.0;
  uint64_t b = v != v ? 0x7FF8000000000000ull : (uint64_t)__double_as_longlong(v);
  p = (b >> 63) ? ~b : (b | 0x8000000000000000ull);
  q = 0xFFFFFFFFu - (uint32_t)i;
}

__device__ __forceinline__ bool na_matches(uint64_t p, uint32_t q, const NaState& st, int level) {
  if (level == 0) return true;
  if (level <= 8) return (p >> (64 - 8 * level)) == (st.pref_p >> (64 - 8 * level));
  if (p != st.pref_p) return false;
  const int lq = level - 8;
  return (q >> (32 - 8 * lq)) == (st.pref_q >> (32 - 8 * lq));
}

__device__ __forceinline__ uint32_t na_digit(uint64_t p, uint32_t q, int level) {
  return level < 8 ? (uint32_t)(p >> (56 - 8 * level)) & 0xFFu : (q >> (24 - 8 * (level - 8))) & 0xFFu;
}

__global__ void k_na_reset(Scratch s, uint32_t k) {
  if (threadIdx.x == 0) {
    s.st->pref_p = 0ull;
    s.st->pref_q = 0u;
    s.st->k_rem = k;
    s.st->count = 0u;
    s.st->pad_ = 0u;
  }
  s.hist[threadIdx.x] = 0u;
}

__global__ void k_na_histo(const double* __restrict__ psi, int64_t n, Scratch s, int level) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const NaState st = *s.st;
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    int d = 256;
    if (i < n) {
      uint64_t p;
      uint32_t q;
      na_key(psi, i, p, q);
      if (na_matches(p, q, st, level)) d = (int)na_digit(p, q, level);
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    if (d < 256 && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&s.hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_na_choose(Scratch s, int level) {
  if (threadIdx.x != 0) return;
  uint32_t above = 0;
  int d = 255;
  for (; d > 0; --d) {
    if (above + s.hist[d] >= s.st->k_rem) break;
    above += s.hist[d];
  }
  s.st->k_rem -= above;
  if (level < 8) s.st->pref_p |= (unsigned long long)d << (56 - 8 * level);
  else s.st->pref_q |= (uint32_t)d << (24 - 8 * (level - 8));
  for (int i = 0; i < 256; ++i) s.hist[i] = 0;
}

__global__ void k_na_collect(const double* __restrict__ psi, int64_t n, Scratch s, uint32_t k) {
  const uint64_t kp = s.st->pref_p;
  const uint32_t kq = s.st->pref_q;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t p;
    uint32_t q;
    na_key(psi, i, p, q);
    if (p > kp || (p == kp && q >= kq)) {
      uint32_t slot = atomicAdd(&s.st->count, 1u);
      if (slot < k) {
        s.p[slot] = p;
        s.q[slot] = q;
      }
    }
  }
}

// one block: bitonic sort of the k collected keys (descending), then the output
__global__ void __launch_bounds__(1024) k_na_sort_emit(Scratch s, int32_t k, const double* __restrict__ psi,
                                                       int32_t* ids, double* vals) {
  __shared__ unsigned long long sp[kNoAllocMaxK];
  __shared__ uint32_t sq[kNoAllocMaxK];
  int m = 1;
  while (m < k) m <<= 1;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    sp[i] = i < k ? s.p[i] : 0ull;  // padding sorts last: no real key equals (0, 0) (p = 0
                                      // only for a negative NaN, which na_key replaces)
    sq[i] = i < k ? s.q[i] : 0u;
  }
  __syncthreads();
  for (int size = 2; size <= m; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool desc = (i & size) == 0;
          const bool i_less = sp[i] < sp[j] || (sp[i] == sp[j] && sq[i] < sq[j]);
          if (i_less == desc) {
            unsigned long long tp = sp[i];
            sp[i] = sp[j];
            sp[j] = tp;
            uint32_t tq = sq[i];
            sq[i] = sq[j];
            sq[j] = tq;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const int32_t id = (int32_t)(0xFFFFFFFFu - sq[i]);
    ids[i] = id;
    if (vals) vals[i] = psi[id];  // the caller's own value
  }
}

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_dev[kMaxDevices] = {};

// Device address of the working area on the current device, looked up once per device.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

// Device memory of the current device `dev`, or managed memory (reachable from every
// device).  Device memory of another GPU is refused: the kernels would read or write it
// through the peer mapping, or fault where there is none.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // the error this lookup itself raised
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

}  // namespace psi

extern "C" psi_status psi_topk_noalloc(const double* psi_in, int64_t n, int32_t k, int32_t* ids_out,
                                       double* vals_out, void* stream) {
  using namespace psi;
  if (!psi_in || !ids_out || n < 1 || n >= ((int64_t)1 << 31) - 1) {
    set_last_error("psi_topk_noalloc: psi and ids_out are required and 1 <= n < 2^31 - 1");
    return PSI_ERR_INVALID_ARG;
  }
  if (k < 1 || (int64_t)k > n || k > kNoAllocMaxK) {
    set_last_error("psi_topk_noalloc: k must be in [1, min(n, 4096)]");
    return PSI_ERR_INVALID_ARG;
  }
  // an error left pending by earlier work of the caller is not this call's: report it
  // without clearing it, before anything here could be blamed for it
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("psi_topk_noalloc: a CUDA error was pending before the call (left in place): ") +
                   cudaGetErrorString(e));
    return PSI_ERR_CUDA;
  }
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_last_error(std::string("psi_topk_noalloc: cudaGetDevice failed: ") + cudaGetErrorString(e));
    return PSI_ERR_CUDA;
  }
  if (!on_device(psi_in, dev) || !on_device(ids_out, dev) || (vals_out && !on_device(vals_out, dev))) {
    set_last_error("psi_topk_noalloc: psi, ids_out and vals_out must be device memory of the current device");
    return PSI_ERR_INVALID_ARG;
  }
  void* base = nullptr;
  e = scratch_address(&base);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_last_error(std::string("psi_topk_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    return PSI_ERR_CUDA;
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  Scratch s{reinterpret_cast<NaState*>(b + kOffState), reinterpret_cast<uint32_t*>(b + kOffHist),
            reinterpret_cast<uint64_t*>(b + kOffP), reinterpret_cast<uint32_t*>(b + kOffQ)};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = (n + 255) / 256;
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
  if (blocks > cap) blocks = cap;
  k_na_reset<<<1, 256, 0, st>>>(s, (uint32_t)k);
  for (int level = 0; level < 12; ++level) {
    k_na_histo<<<(int)blocks, 256, 0, st>>>(psi_in, n, s, level);
    k_na_choose<<<1, 32, 0, st>>>(s, level);
  }
  k_na_collect<<<(int)blocks, 256, 0, st>>>(psi_in, n, s, (uint32_t)k);
  k_na_sort_emit<<<1, 1024, 0, st>>>(s, k, psi_in, ids_out, vals_out);
  e = cudaGetLastError();  // nothing was pending on entry: only these launches can have failed
  if (e != cudaSuccess) {
    set_last_error(std::string("psi_topk_noalloc: launch failed: ") + cudaGetErrorString(e));
    return PSI_ERR_CUDA;
  }
  return PSI_OK;
}
