// df.cuh -- float pairs: a value carried as the unevaluated sum hi + lo of two floats.
#pragma once

#include "common.cuh"

namespace psi {

// A value carried as the unevaluated sum hi + lo of two floats (about 48 significant
// bits).  Sums of such pairs take a dozen FP32 instructions (Knuth's two-sum on the high
// parts, then the low parts and a renormalisation), several times cheaper than FP64 adds
// on a part whose FP64 rate is a small fraction of its FP32 rate.  Used for the FP64
// confirming step and the final product of the FP32-series mode (8-byte gathers, as FP64),
// and as pairs of pairs (DF2, two scenarios per lane) in the scenario batches.
struct DF {
  float hi, lo;
  DF() = default;
  __device__ __forceinline__ DF(int z) : hi((float)z), lo(0.f) {}
  __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
};
__device__ __forceinline__ DF operator+(DF a, DF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  const float h = s + e;
  return DF(h, e - (h - s));
}
__device__ __forceinline__ DF& operator+=(DF& x, DF y) {
  x = x + y;
  return x;
}
__device__ __forceinline__ DF df_from(double x) {
  const float h = (float)x;
  return DF(h, (float)(x - (double)h));
}
__device__ __forceinline__ double df_value(DF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ void st_keep(DF* p, DF v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1,%2}, %3;" ::"l"(p), "f"(v.hi), "f"(v.lo), "l"(pol)
               : "memory");
}
__device__ __forceinline__ DF ld_gather(const DF* p, uint64_t pol) {
  float x, y;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0,%1}, [%2], %3;" : "=f"(x), "=f"(y) : "l"(p), "l"(pol));
  return DF(x, y);
}

// two float pairs: the two scenarios of one lane in the batched product, or the two sums
// (sigma, beta) of the build's leader product
struct DF2 {
  DF a, b;
  DF2() = default;
  __device__ __forceinline__ DF2(int z) : a(z), b(z) {}
  __device__ __forceinline__ DF2(DF x, DF y) : a(x), b(y) {}
};
__device__ __forceinline__ DF2 operator+(DF2 x, DF2 y) { return DF2(x.a + y.a, x.b + y.b); }
__device__ __forceinline__ DF2& operator+=(DF2& x, DF2 y) {
  x = x + y;
  return x;
}
__device__ __forceinline__ DF2 ld_gather(const DF2* p, uint64_t pol) {
  float a, b, c, d;
  asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
               : "=f"(a), "=f"(b), "=f"(c), "=f"(d)
               : "l"(p), "l"(pol));
  return DF2(DF(a, b), DF(c, d));
}

}  // namespace psi
