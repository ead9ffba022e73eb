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
static_assert(kRsTile == kRadixTileKeys, "the tile of the published first-pass counts");
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

template <typename K>
__global__ void __launch_bounds__(kRsThreads) k_radix_histo(const K* __restrict__ keys, int64_t n, int shift,
                                                           uint32_t mask, int64_t num_tiles,
                                                           uint32_t* __restrict__ counts) {
  __shared__ uint32_t h[kRsWarps][256];  // one sub-histogram per warp: contention stays inside a warp
  for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&h[0][0])[i] = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll 4
  for (int i = 0; i < kRsItems; ++i) {
    int64_t idx = base + (int64_t)i * kRsThreads + threadIdx.x;
    if (idx < n) atomicAdd(&h[warp][(uint32_t)(keys[idx] >> shift) & mask], 1u);
  }
  __syncthreads();
  uint32_t t = 0;
#pragma unroll
  for (int w = 0; w < kRsWarps; ++w) t += h[w][threadIdx.x];
  counts[(int64_t)threadIdx.x * num_tiles + blockIdx.x] = t;
}

// Stable scatter of one tile: items are ranked per warp (warp-major, then round, then
// lane: the input order), placed in shared memory in digit order, and written out so that
// each digit's run of the tile lands contiguously (coalesced) at its global offset.
template <typename K, bool VALS>
__global__ void __launch_bounds__(kRsThreads) k_radix_scatter(const K* __restrict__ keys, const uint32_t* __restrict__ vals,
                                                             K* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                                                             int64_t n, int shift, uint32_t mask,
                                                             int64_t num_tiles,
                                                             const uint32_t* __restrict__ offsets) {
  extern __shared__ __align__(16) unsigned char rs_dyn[];
  K* sk = reinterpret_cast<K*>(rs_dyn);
  uint32_t* sv = reinterpret_cast<uint32_t*>(rs_dyn + (size_t)kRsTile * sizeof(K));
  __shared__ uint32_t wh[kRsWarps][257];  // per-warp digit counts (padded row: fewer bank conflicts)
  __shared__ uint32_t tile_base[256];
  __shared__ uint32_t dstart[256];
  __shared__ uint32_t wsum[kRsWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kRsWarps * 257; i += kRsThreads) (&wh[0][0])[i] = 0;
  tile_base[threadIdx.x] = offsets[(int64_t)threadIdx.x * num_tiles + blockIdx.x];
  __syncthreads();
  const int64_t tile0 = (int64_t)blockIdx.x * kRsTile;
  const int64_t wbase = tile0 + (int64_t)warp * kRsPerWarp;
  const uint32_t lt_mask = (1u << lane) - 1u;
  K k[kRsItems];
  uint32_t v[kRsItems];
  uint32_t dp[kRsItems];  // digit << 16 | rank inside the warp's digit run
#pragma unroll
  for (int r = 0; r < kRsItems; ++r) {
    int64_t idx = wbase + (int64_t)r * 32 + lane;
    bool ok = idx < n;
    k[r] = ok ? keys[idx] : K(0);
    if (VALS) v[r] = ok ? vals[idx] : 0u;
    // a key past the end takes digit 255 (above every digit of a pass, mask <= 255): such
    // keys are a suffix of the tile in ranking order, so they sort to the end of the tile's
    // buffer and are never written out
    const int d = ok ? (int)((uint32_t)(k[r] >> shift) & mask) : 255;
    const uint32_t peers = (kRsMatchEvery > 0 && r % kRsMatchEvery == 0) ? __match_any_sync(0xffffffffu, d)
                                                                          : digit_peers_ballot(d);
    uint32_t before = wh[warp][d];
    __syncwarp();
    if ((peers & lt_mask) == 0) wh[warp][d] = before + __popc(peers);
    __syncwarp();
    dp[r] = ((uint32_t)d << 16) | (before + __popc(peers & lt_mask));
  }
  __syncthreads();
  // per digit (= thread): exclusive prefix over warps, then exclusive scan over digits
  uint32_t total = 0;
  {
    const int d = threadIdx.x;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) {
      uint32_t t = wh[w][d];
      wh[w][d] = total;
      total += t;
    }
  }
  uint32_t x = total;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  uint32_t wb = 0;
  for (int w = 0; w < warp; ++w) wb += wsum[w];
  dstart[threadIdx.x] = wb + x - total;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRsItems; ++r) {
    const int d = (int)(dp[r] >> 16);
    const uint32_t lp = dstart[d] + wh[warp][d] + (dp[r] & 0xFFFFu);
    sk[lp] = k[r];
    if (VALS) sv[lp] = v[r];
  }
  __syncthreads();
  const int64_t rem = n - tile0;
  const int valid = rem < kRsTile ? (int)rem : kRsTile;
  for (int i = threadIdx.x; i < valid; i += kRsThreads) {
    const K key = sk[i];
    const int d = (int)((uint32_t)(key >> shift) & mask);
    const uint32_t o = tile_base[d] + (uint32_t)i - dstart[d];
    keys_out[o] = key;
    if (VALS) vals_out[o] = sv[i];
  }
}

template <typename K, bool VALS>
void launch_scatter(const K* src, const uint32_t* vsrc, K* dst, uint32_t* vdst, int64_t n, int shift, uint32_t mask,
                    int64_t tiles, const uint32_t* offsets, cudaStream_t s) {
  const size_t dyn = (size_t)kRsTile * (sizeof(K) + (VALS ? sizeof(uint32_t) : 0));
  static const bool configured = [dyn] {  // once, thread-safe (concurrent builds on several streams)
    PSI_CUDA(cudaFuncSetAttribute(k_radix_scatter<K, VALS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    return true;
  }();
  (void)configured;
  k_radix_scatter<K, VALS><<<(unsigned)tiles, kRsThreads, dyn, s>>>(src, vsrc, dst, vdst, n, shift, mask, tiles,
                                                                     offsets);
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
  return radix_sort_bits(keys, keys_alt, vals, vals_alt, n, 0, bits, al, s, keys_in, vals_in, nullptr);
}

template <typename K>
bool radix_sort_bits(K* keys, K* keys_alt, uint32_t* vals, uint32_t* vals_alt, int64_t n, int lo, int hi,
                     Allocator& al, cudaStream_t s, const K* keys_in, const uint32_t* vals_in,
                     uint32_t* first_counts) {
  if (n <= 1 || hi <= lo) {
    if (keys_in && n > 0) PSI_CUDA(cudaMemcpyAsync(keys, keys_in, sizeof(K) * n, cudaMemcpyDeviceToDevice, s));
    if (vals && vals_in && n > 0)
      PSI_CUDA(cudaMemcpyAsync(vals, vals_in, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    return false;
  }
  const int64_t tiles = ceil_div(n, kRsTile);
  DBuf<uint32_t> own;
  if (!first_counts) own.reset(al, (size_t)(tiles * 256));
  uint32_t* counts = first_counts ? first_counts : own.get();
  // the first pass reads the separate inputs when given (they are never written)
  K* src = keys_in ? const_cast<K*>(keys_in) : keys;
  K* dst = keys_alt;
  uint32_t* vsrc = vals_in ? const_cast<uint32_t*>(vals_in) : vals;
  uint32_t* vdst = vals_alt;
  bool flipped = false;
  for (int shift = lo; shift < hi; shift += 8) {
    const uint32_t mask = hi - shift >= 8 ? 0xFFu : (1u << (hi - shift)) - 1u;  // bits at or above hi stay out
    if (shift != lo || !first_counts) {
      k_radix_histo<K><<<(unsigned)tiles, kRsThreads, 0, s>>>(src, n, shift, mask, tiles, counts);
      PSI_LAUNCHED();
    }
    exclusive_scan_u32(counts, counts, tiles * 256, al, s, nullptr);
    if (vals) launch_scatter<K, true>(src, vsrc, dst, vdst, n, shift, mask, tiles, counts, s);
    else launch_scatter<K, false>(src, nullptr, dst, nullptr, n, shift, mask, tiles, counts, s);
    if (shift == lo && keys_in) {  // from now on the two buffers alternate
      src = keys;
      vsrc = vals;
    }
    std::swap(src, dst);
    std::swap(vsrc, vdst);
    flipped = !flipped;
  }
  return flipped;
}

template bool radix_sort<uint32_t>(uint32_t*, uint32_t*, uint32_t*, uint32_t*, int64_t, int, Allocator&, cudaStream_t,
                                   const uint32_t*, const uint32_t*);
template bool radix_sort<uint64_t>(uint64_t*, uint64_t*, uint32_t*, uint32_t*, int64_t, int, Allocator&, cudaStream_t,
                                   const uint64_t*, const uint32_t*);
template bool radix_sort_bits<uint64_t>(uint64_t*, uint64_t*, uint32_t*, uint32_t*, int64_t, int, int, Allocator&,
                                        cudaStream_t, const uint64_t*, const uint32_t*, uint32_t*);

void sum_f64(const double* x, int64_t n, double* d_out, Allocator& al, cudaStream_t s) {
  DBuf<double> part(al, kSumBlocks);
  k_sum_partial<<<kSumBlocks, kSumThreads, 0, s>>>(x, n, part.get());
  PSI_LAUNCHED();
  k_sum_partial<<<1, kSumThreads, 0, s>>>(part.get(), kSumBlocks, d_out);
  PSI_LAUNCHED();
}

}  // namespace psi
