// primitives.cu -- exclusive scan, stable LSD radix sort, deterministic FP64 sum.
#include "primitives.cuh"

namespace psi {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// block-wide exclusive scan of one value per thread; returns the block total in *total
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* smem_warp, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = (lane < (int)(blockDim.x >> 5)) ? smem_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    smem_warp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  uint32_t warp_base = warp > 0 ? smem_warp[warp - 1] : 0u;
  *total = smem_warp[(blockDim.x >> 5) - 1];
  return warp_base + x - v;
}

__global__ void k_scan_reduce(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ sums) {
  __shared__ uint32_t sw[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) acc += in[base + i];
  uint32_t tot;
  block_exclusive_scan(acc, sw, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_down(const uint32_t* in, uint32_t* out, int64_t n,
                            const uint32_t* __restrict__ offsets, uint32_t* d_total) {
  __shared__ uint32_t sw[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0u;
    acc += v[i];
  }
  uint32_t tot;
  uint32_t run = block_exclusive_scan(acc, sw, &tot) + (offsets ? offsets[blockIdx.x] : 0u);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (d_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) *d_total = run;
}

// ---------------------------------------------------------------- radix sort
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsItems = 12;                    // measured: 12 beats 8 and 16 on the 537M-key edge sort
constexpr int kRsTile = kRsThreads * kRsItems;  // 3072 keys per tile
constexpr int kRsPerWarp = 32 * kRsItems;       // 384 consecutive keys per warp

// Lanes of the warp holding the same 8-bit digit.  Ballots (one per digit bit: the lanes
// that agree with this lane on every bit) run on the ALU pipe, the match instruction on the
// narrower ADU pipe; a pass that used only one of them kept that pipe ~90% busy, so the
// rounds of a tile share the work: every kRsMatchEvery-th round matches (measured on the
// scale-25 build: every 2nd / 3rd / 4th / 6th round 60.1 / 59.7 / 60.3 / 60.8 ms, ballots
// only 61.2 ms).
constexpr int kRsMatchEvery = 3;
__device__ __forceinline__ uint32_t digit_peers_ballot(int d) {
  uint32_t peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const bool bit = (d >> b) & 1;
    const uint32_t bal = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? bal : ~bal;
  }
  return peers;
}

// ---------------------------------------------------------------- onesweep passes
// One kernel per 8-bit digit pass, in the manner of the onesweep LSD sort (Adinets and
// Merrill, "Onesweep: A Faster Least Significant Digit Radix Sort for GPUs", 2022): the
// digit histograms of every pass come from one read of the input before the first pass;
// within a pass each block claims the next tile (3072 keys, in input order) from a
// counter, ranks the tile's keys by digit, publishes its digit counts, and finds the
// number of keys of each digit in all earlier tiles by looking back at the counts those
// tiles published (a tile whose own look-back is done publishes inclusive counts, which
// end a look-back).  The tile then writes each digit's run contiguously at
// base[digit] + (earlier keys of that digit).  Tiles are claimed in launch order, so a
// tile only ever waits on tiles whose blocks are already running.
constexpr uint64_t kOsAgg = 1ull << 62;   // status word: the tile's own digit count
constexpr uint64_t kOsIncl = 1ull << 63;  // status word: count of the tile and all before it
constexpr uint64_t kOsValue = kOsAgg - 1;
constexpr int kOsWindow = 4;               // predecessors read per look-back round
constexpr uint32_t kOsSpinLimit = 1u << 22;  // polls of a not-yet-published tile before giving up
constexpr int kOsMaxPasses = 8;

__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Digit histograms of every pass in one read: hist[p][d] = keys whose digit p is d.
template <typename K>
__global__ void __launch_bounds__(kRsThreads) k_os_histo(const K* __restrict__ keys, int64_t n, int passes,
                                                        uint32_t* __restrict__ hist) {
  extern __shared__ uint32_t oh[];  // [kRsWarps][passes][256]: one sub-histogram per warp
  for (int i = threadIdx.x; i < kRsWarps * passes * 256; i += kRsThreads) oh[i] = 0;
  __syncthreads();
  uint32_t* h = oh + (threadIdx.x >> 5) * passes * 256;
  const int64_t stride = (int64_t)gridDim.x * kRsThreads;
  int64_t i = (int64_t)blockIdx.x * kRsThreads + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {
    K k[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) k[q] = keys[i + q * stride];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      for (int p = 0; p < passes; ++p) atomicAdd(&h[p * 256 + ((uint32_t)(k[q] >> (8 * p)) & 0xFFu)], 1u);
  }
  for (; i < n; i += stride) {
    const K k = keys[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&h[p * 256 + ((uint32_t)(k >> (8 * p)) & 0xFFu)], 1u);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < passes * 256; j += kRsThreads) {
    uint32_t t = 0;
    for (int w = 0; w < kRsWarps; ++w) t += oh[w * passes * 256 + j];
    if (t) atomicAdd(&hist[j], t);
  }
}

// base[p][d] = keys of pass p whose digit is below d (one block per pass)
__global__ void k_os_bases(const uint32_t* __restrict__ hist, uint32_t* __restrict__ base) {
  __shared__ uint32_t sw[32];
  const uint32_t v = hist[blockIdx.x * 256 + threadIdx.x];
  uint32_t total;
  base[blockIdx.x * 256 + threadIdx.x] = block_exclusive_scan(v, sw, &total);
}

template <typename K, bool VALS>
__global__ void __launch_bounds__(kRsThreads) k_os_pass(const K* __restrict__ keys, const uint32_t* __restrict__ vals,
                                                       K* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                                                       int64_t n, int shift, uint64_t* __restrict__ status,
                                                       const uint32_t* __restrict__ base, uint32_t* counter,
                                                       uint32_t* err) {
  extern __shared__ __align__(16) unsigned char rs_dyn[];
  K* sk = reinterpret_cast<K*>(rs_dyn);
  uint32_t* sv = reinterpret_cast<uint32_t*>(rs_dyn + (size_t)kRsTile * sizeof(K));
  __shared__ uint32_t wh[kRsWarps][257];  // per-warp digit counts (padded row: fewer bank conflicts)
  __shared__ uint32_t gofs[256];          // output position of the tile's item i of digit d: gofs[d] + i
  __shared__ uint32_t dstart[256];
  __shared__ uint32_t wsum[kRsWarps];
  __shared__ int64_t tile_sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) tile_sh = (int64_t)atomicAdd(counter, 1u);
  for (int i = threadIdx.x; i < kRsWarps * 257; i += kRsThreads) (&wh[0][0])[i] = 0;
  __syncthreads();
  const int64_t tile = tile_sh;
  const int64_t tile0 = tile * kRsTile;
  const int64_t wbase = tile0 + (int64_t)warp * kRsPerWarp;
  const uint32_t lt_mask = (1u << lane) - 1u;
  K k[kRsItems];
  uint32_t v[kRsItems];
  uint32_t dp[kRsItems];  // digit << 16 | rank inside the warp's digit run
#pragma unroll
  for (int r = 0; r < kRsItems; ++r) {
    const int64_t idx = wbase + (int64_t)r * 32 + lane;
    const bool ok = idx < n;
    k[r] = ok ? keys[idx] : K(0);
    if (VALS) v[r] = ok ? vals[idx] : 0u;
    // a key past the end takes digit 255: such keys are a suffix of the tile in ranking
    // order, so they sort to the end of the tile's buffer and are never written out
    const int d = ok ? (int)((uint32_t)(k[r] >> shift) & 0xFFu) : 255;
    const uint32_t peers = (kRsMatchEvery > 0 && r % kRsMatchEvery == 0) ? __match_any_sync(0xffffffffu, d)
                                                                          : digit_peers_ballot(d);
    const uint32_t before = wh[warp][d];
    __syncwarp();
    if ((peers & lt_mask) == 0) wh[warp][d] = before + __popc(peers);
    __syncwarp();
    dp[r] = ((uint32_t)d << 16) | (before + __popc(peers & lt_mask));
  }
  __syncthreads();
  const int64_t rem = n - tile0;
  const int valid = rem < kRsTile ? (int)rem : kRsTile;
  // per digit (= thread): exclusive prefix over warps, the tile's count of the digit
  const int d = threadIdx.x;
  uint32_t total = 0;
#pragma unroll
  for (int w = 0; w < kRsWarps; ++w) {
    const uint32_t t = wh[w][d];
    wh[w][d] = total;
    total += t;
  }
  if (d == 255) total -= (uint32_t)(kRsTile - valid);  // the padding keys are not counted
  // publish the count, look back over the earlier tiles, publish the inclusive count
  uint64_t* mine = status + tile * 256 + d;
  uint64_t excl = 0;
  if (tile == 0) {
    st_relaxed_u64(mine, kOsIncl | (uint64_t)total);
  } else {
    st_relaxed_u64(mine, kOsAgg | (uint64_t)total);
    int64_t p = tile - 1;  // the nearest tile not yet added
    uint32_t polls = 0;
    for (;;) {
      uint64_t w[kOsWindow];
#pragma unroll
      for (int i = 0; i < kOsWindow; ++i) w[i] = p - i >= 0 ? ld_relaxed_u64(status + (p - i) * 256 + d) : kOsIncl;
      int used = 0;
      bool closed = false;
#pragma unroll
      for (int i = 0; i < kOsWindow; ++i) {
        if (closed || used < i) continue;  // stop at the first tile not yet published
        if (w[i] == 0) continue;
        excl += w[i] & kOsValue;
        ++used;
        if (w[i] & kOsIncl) closed = true;
      }
      if (closed) break;
      p -= used;
      if (used < kOsWindow) {
        if (++polls > kOsSpinLimit) {
          atomicOr(err, 1u);  // never expected: the tile's predecessors are all running
          break;
        }
        __nanosleep(64);
      }
    }
    st_relaxed_u64(mine, kOsIncl | (excl + total));
  }
  // tile-local start of every digit's run: exclusive scan of the counts over the digits
  uint32_t x = total;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  uint32_t wb = 0;
  for (int w = 0; w < warp; ++w) wb += wsum[w];
  const uint32_t ds = wb + x - total;
  dstart[d] = ds;
  gofs[d] = base[d] + (uint32_t)excl - ds;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRsItems; ++r) {
    const int dd = (int)(dp[r] >> 16);
    const uint32_t lp = dstart[dd] + wh[warp][dd] + (dp[r] & 0xFFFFu);
    sk[lp] = k[r];
    if (VALS) sv[lp] = v[r];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < valid; i += kRsThreads) {
    const K key = sk[i];
    const uint32_t o = gofs[(uint32_t)(key >> shift) & 0xFFu] + (uint32_t)i;
    keys_out[o] = key;
    if (VALS) vals_out[o] = sv[i];
  }
}

template <typename K, bool VALS>
void launch_pass(const K* src, const uint32_t* vsrc, K* dst, uint32_t* vdst, int64_t n, int shift, int64_t tiles,
                 uint64_t* status, const uint32_t* base, uint32_t* counter, uint32_t* err, cudaStream_t s) {
  const size_t dyn = (size_t)kRsTile * (sizeof(K) + (VALS ? sizeof(uint32_t) : 0));
  static bool configured = false;
  if (!configured) {
    PSI_CUDA(cudaFuncSetAttribute(k_os_pass<K, VALS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    configured = true;
  }
  PSI_CUDA(cudaMemsetAsync(status, 0, sizeof(uint64_t) * 256 * (size_t)tiles, s));
  k_os_pass<K, VALS><<<(unsigned)tiles, kRsThreads, dyn, s>>>(src, vsrc, dst, vdst, n, shift, status, base, counter,
                                                             err);
  PSI_LAUNCHED();
}

// ---------------------------------------------------------------- FP64 sum
constexpr int kSumThreads = 512;
constexpr int kSumBlocks = 512;

__global__ void k_sum_partial(const double* __restrict__ x, int64_t n, double* __restrict__ part) {
  __shared__ double sh[kSumThreads];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kSumThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kSumThreads)
    acc += x[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kSumThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

}  // namespace

void exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, Allocator& al, cudaStream_t s,
                        uint32_t* d_total) {
  if (n <= 0) {
    if (d_total) PSI_CUDA(cudaMemsetAsync(d_total, 0, sizeof(uint32_t), s));
    return;
  }
  const int64_t blocks = ceil_div(n, kScanTile);
  if (blocks == 1) {
    k_scan_down<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, d_total);
    PSI_LAUNCHED();
    return;
  }
  DBuf<uint32_t> sums(al, (size_t)blocks);
  k_scan_reduce<<<(unsigned)blocks, kScanThreads, 0, s>>>(in, n, sums.get());
  PSI_LAUNCHED();
  exclusive_scan_u32(sums.get(), sums.get(), blocks, al, s, nullptr);
  k_scan_down<<<(unsigned)blocks, kScanThreads, 0, s>>>(in, out, n, sums.get(), d_total);
  PSI_LAUNCHED();
}

template <typename K>
bool radix_sort(K* keys, K* keys_alt, uint32_t* vals, uint32_t* vals_alt, int64_t n, int bits, Allocator& al,
                cudaStream_t s, const K* keys_in, const uint32_t* vals_in) {
  if (n <= 1 || bits <= 0) {
    if (keys_in && n > 0) PSI_CUDA(cudaMemcpyAsync(keys, keys_in, sizeof(K) * n, cudaMemcpyDeviceToDevice, s));
    if (vals && vals_in && n > 0)
      PSI_CUDA(cudaMemcpyAsync(vals, vals_in, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    return false;
  }
  const int passes = (bits + 7) / 8;
  PSI_REQUIRE(passes <= kOsMaxPasses && passes * 8 <= (int)(8 * sizeof(K)), PSI_ERR_INVALID_ARG,
              "internal: radix sort wider than its key");
  const int64_t tiles = ceil_div(n, kRsTile);
  // the first pass reads the separate inputs when given (they are never written)
  K* src = keys_in ? const_cast<K*>(keys_in) : keys;
  K* dst = keys_alt;
  uint32_t* vsrc = vals_in ? const_cast<uint32_t*>(vals_in) : vals;
  uint32_t* vdst = vals_alt;
  // [0, 256 * passes): histograms, then bases; then a tile counter per pass and an error word
  DBuf<uint32_t> small(al, (size_t)2 * 256 * passes + passes + 1);
  uint32_t* hist = small.get();
  uint32_t* base = hist + 256 * passes;
  uint32_t* counters = base + 256 * passes;
  uint32_t* err = counters + passes;
  PSI_CUDA(cudaMemsetAsync(small.get(), 0, sizeof(uint32_t) * small.count, s));
  DBuf<uint64_t> status(al, (size_t)tiles * 256);
  {
    const size_t dyn = sizeof(uint32_t) * kRsWarps * passes * 256;
    static bool configured[2] = {false, false};
    if (!configured[sizeof(K) == 8]) {
      PSI_CUDA(cudaFuncSetAttribute(k_os_histo<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(sizeof(uint32_t) * kRsWarps * kOsMaxPasses * 256)));
      configured[sizeof(K) == 8] = true;
    }
    const int64_t want = ceil_div(n, (int64_t)kRsThreads * 16);
    const int64_t cap = num_sms() * 2;
    k_os_histo<K><<<(unsigned)(want < cap ? (want > 0 ? want : 1) : cap), kRsThreads, dyn, s>>>(src, n, passes, hist);
    PSI_LAUNCHED();
    k_os_bases<<<passes, 256, 0, s>>>(hist, base);
    PSI_LAUNCHED();
  }
  bool flipped = false;
  for (int p = 0; p < passes; ++p) {
    if (vals) launch_pass<K, true>(src, vsrc, dst, vdst, n, 8 * p, tiles, status.get(), base + 256 * p, counters + p,
                                   err, s);
    else launch_pass<K, false>(src, nullptr, dst, nullptr, n, 8 * p, tiles, status.get(), base + 256 * p,
                               counters + p, err, s);
    if (p == 0 && keys_in) {  // from now on the two buffers alternate
      src = keys;
      vsrc = vals;
    }
    std::swap(src, dst);
    std::swap(vsrc, vdst);
    flipped = !flipped;
  }
  uint32_t herr = 0;
  PSI_CUDA(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaStreamSynchronize(s));
  PSI_REQUIRE(herr == 0, PSI_ERR_TIMEOUT, "radix sort: a tile waited too long for an earlier tile's counts");
  return flipped;
}

template bool radix_sort<uint32_t>(uint32_t*, uint32_t*, uint32_t*, uint32_t*, int64_t, int, Allocator&, cudaStream_t,
                                   const uint32_t*, const uint32_t*);
template bool radix_sort<uint64_t>(uint64_t*, uint64_t*, uint32_t*, uint32_t*, int64_t, int, Allocator&, cudaStream_t,
                                   const uint64_t*, const uint32_t*);

void sum_f64(const double* x, int64_t n, double* d_out, Allocator& al, cudaStream_t s) {
  DBuf<double> part(al, kSumBlocks);
  k_sum_partial<<<kSumBlocks, kSumThreads, 0, s>>>(x, n, part.get());
  PSI_LAUNCHED();
  k_sum_partial<<<1, kSumThreads, 0, s>>>(part.get(), kSumBlocks, d_out);
  PSI_LAUNCHED();
}

}  // namespace psi
