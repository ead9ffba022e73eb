// primitives.cuh -- device-wide building blocks written for this library: exclusive
// scan, stable LSD radix sort, deterministic FP64 sum.
#pragma once

#include "common.cuh"

namespace psi {

// out[i] = in[0] + ... + in[i-1] (uint32).  in == out is allowed.  If d_total is not
// null it receives the sum of all n values (device memory).
void exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, Allocator& al,
                        cudaStream_t s, uint32_t* d_total = nullptr);

// Stable LSD radix sort of keys on bits [0, bits), 8 bits per pass, carrying an optional
// uint32 payload (vals may be null).  Sorts between (keys, vals) and (keys_alt,
// vals_alt); returns true when the sorted data ended up in the *_alt buffers.  When
// keys_in (and vals_in) are given, the data to sort is read from them, which are left
// untouched, and (keys, vals) only serve as buffers.
template <typename K>
bool radix_sort(K* keys, K* keys_alt, uint32_t* vals, uint32_t* vals_alt, int64_t n, int bits,
                Allocator& al, cudaStream_t s, const K* keys_in = nullptr, const uint32_t* vals_in = nullptr);

// The same sort on key bits [lo, hi) only (passes of 8 bits from lo, the last one
// narrower): sorting [0, b) and then [b, hi) gives the sort on [0, hi), and between the two
// calls the data is in the order of bits [0, b).  first_counts (nullable): a device buffer of
// 256 * ceil(n / kRadixTileKeys) counts holding, at [digit * tiles + tile], how many keys of
// each tile of kRadixTileKeys consecutive keys have each value of the first pass's digit
// ((key >> lo) & radix_first_mask(lo, hi)); the first histogram pass is then skipped, and
// the buffer is overwritten.
constexpr int kRadixTileKeys = 3072;
inline uint32_t radix_first_mask(int lo, int hi) { return hi - lo >= 8 ? 0xFFu : (1u << (hi - lo)) - 1u; }
template <typename K>
bool radix_sort_bits(K* keys, K* keys_alt, uint32_t* vals, uint32_t* vals_alt, int64_t n, int lo, int hi,
                     Allocator& al, cudaStream_t s, const K* keys_in = nullptr, const uint32_t* vals_in = nullptr,
                     uint32_t* first_counts = nullptr);

// Deterministic FP64 sum of n values (fixed order for a given n) into *d_out.
void sum_f64(const double* x, int64_t n, double* d_out, Allocator& al, cudaStream_t s);

// Number of bits needed to hold values in [0, v].
inline int bits_for(uint64_t v) {
  int b = 0;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

}  // namespace psi
