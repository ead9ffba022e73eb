// warmstart.cu -- a learned start vector for Power-psi.
//
// Per-user features (8): log(1 + followers), log(1 + leaders), log lambda, log mu, and the
// mean of each of these over the user's followers (one pull product over the followers).
// A small network, 8 -> 64 -> 64 -> 1 with GELU, BF16 weights and BF16 (rounded) inputs,
// FP32 accumulation, predicts log s_i of the converged iterate; s_0 = exp(prediction) replaces
// s_0 = c.  Algorithm 2 then runs unchanged from that start, so only the step count can
// change, never the fixed point.  The network is trained on the GPU by the kernels below
// (forward, backward with per-block gradient partials summed in a fixed order, Adam).
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "build.cuh"
#include "solve.cuh"
#include "spmv.cuh"

namespace psi {

// parameter layout (FP32 master copy and BF16 working copy)
constexpr int kIn = 8, kH = 64;
constexpr int kOffW1 = 0;                      // [kIn][kH]
constexpr int kOffB1 = kOffW1 + kIn * kH;      // [kH]
constexpr int kOffW2 = kOffB1 + kH;            // [kH][kH], W2[j][k]
constexpr int kOffB2 = kOffW2 + kH * kH;       // [kH]
constexpr int kOffW3 = kOffB2 + kH;            // [kH]
constexpr int kOffB3 = kOffW3 + kH;            // [1]
constexpr int kParams = kOffB3 + 1;            // 4801
constexpr int kNorm = 2 * kIn + 2;             // x mean, x std, target mean, target std

namespace {

#define WGRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

int wgrid(int64_t n) {
  int64_t g = ceil_div(n > 0 ? n : 1, 256);
  int64_t cap = num_sms() * 16;
  return (int)(g < cap ? g : cap);
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ---------------------------------------------------------------- features

// base features of every user (internal order): log(1+followers), log(1+leaders), log lambda,
// log mu; the gathered-space copy feeds the follower means
__global__ void k_base_features(const int32_t* __restrict__ row_ptr, int32_t n_rows,
                                const int32_t* __restrict__ n_leaders, const double* __restrict__ lam,
                                const double* __restrict__ mu, int64_t n, float* x) {
  WGRID_STRIDE(k, n) {
    const int32_t fol = k < n_rows ? row_ptr[k + 1] - row_ptr[k] : 0;
    float* o = x + k * kIn;
    o[0] = logf(1.f + (float)fol);
    o[1] = logf(1.f + (float)n_leaders[k]);
    o[2] = (float)log(fmax(lam[k], 1e-12));
    o[3] = (float)log(fmax(mu[k], 1e-12));
    o[4] = o[5] = o[6] = o[7] = 0.f;
  }
}

// the four base features of every gathered user (X then U), zero at the pad entry
__global__ void k_features_to_u(const float* __restrict__ x, int32_t nX, int32_t nR, int64_t nu, F4* f) {
  WGRID_STRIDE(i, nu + 1) {
    if (i == nu) {
      f[i] = F4(0);
    } else {
      const int64_t user = i < nX ? i : i + nR;
      const float4 o = *reinterpret_cast<const float4*>(x + user * kIn);
      f[i] = F4(o.x, o.y, o.z, o.w);
    }
  }
}


// mean over the followers of row r of the four base features, into columns 4..7
struct EpiMean4 {
  const int32_t* row_ptr;
  float* x;
  __device__ __forceinline__ void row(int32_t r, F4 y, double&, uint64_t, uint64_t) const {
    const float inv = 1.f / (float)(row_ptr[r + 1] - row_ptr[r]);
    *reinterpret_cast<float4*>(x + (int64_t)r * kIn + 4) = make_float4(y.x * inv, y.y * inv, y.z * inv, y.w * inv);
  }
};

__global__ void k_scatter_rows8(const float* __restrict__ in, const int32_t* __restrict__ perm, int64_t n, float* out) {
  WGRID_STRIDE(idx, n * kIn) {
    const int64_t k = idx / kIn;
    out[(int64_t)perm[k] * kIn + idx % kIn] = in[idx];
  }
}

// ---------------------------------------------------------------- the network

__global__ void k_to_bf16(const float* __restrict__ w, int n, __nv_bfloat16* b) {
  WGRID_STRIDE(i, n) b[i] = __float2bfloat16_rn(w[i]);
}

// ---- tensor-core tiles (mma.sync m16n8k16, BF16 operands, FP32 accumulation)
// Fragment layout (PTX ISA, mma.m16n8k16 with .bf16): lane = 4 g + t (g = lane / 4, t = lane % 4);
//   A (16x16, row major): a0 = A[g][2t..2t+1], a1 = A[g+8][2t..], a2 = A[g][2t+8..], a3 = A[g+8][2t+8..]
//   B (16x8):             b0 = B[2t..2t+1][g], b1 = B[2t+8..2t+9][g]
//   C (16x8, FP32):       c0, c1 = C[g][2t..2t+1], c2, c3 = C[g+8][2t..2t+1]
// Two adjacent C tiles of a layer's output therefore form one A fragment of the next layer.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // lo in the low half
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t pack_raw(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The network's weights as B fragments of one warp (registers): W1 (K = 8 inputs padded to
// 16, 8 column tiles), W2 (4 K steps x 8 column tiles), W3 (4 K steps, column 0 of a tile).
struct MlpFrags {
  uint32_t w1[8];
  uint32_t w2[4][8][2];
  uint32_t w3[4][2];
};

__device__ __forceinline__ void load_frags(const __nv_bfloat16* __restrict__ wb, int lane, MlpFrags& f) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
    f.w1[nt] = pack_raw(wb[kOffW1 + (2 * t) * kH + 8 * nt + g], wb[kOffW1 + (2 * t + 1) * kH + 8 * nt + g]);
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int k0 = 16 * kk + 2 * t, n = 8 * nt + g;
      f.w2[kk][nt][0] = pack_raw(wb[kOffW2 + k0 * kH + n], wb[kOffW2 + (k0 + 1) * kH + n]);
      f.w2[kk][nt][1] = pack_raw(wb[kOffW2 + (k0 + 8) * kH + n], wb[kOffW2 + (k0 + 9) * kH + n]);
    }
    const int k0 = 16 * kk + 2 * t;
    f.w3[kk][0] = g == 0 ? pack_raw(wb[kOffW3 + k0], wb[kOffW3 + k0 + 1]) : 0u;
    f.w3[kk][1] = g == 0 ? pack_raw(wb[kOffW3 + k0 + 8], wb[kOffW3 + k0 + 9]) : 0u;
  }
}

// Forward pass of 16 rows [r0, r0 + 16) by one warp.  Outputs the normalised prediction of
// rows r0 + g (y_lo) and r0 + g + 8 (y_hi) in lanes with t == 0; optionally keeps z1, z2
// (pre-activations) and the BF16 A fragments of h1, h2 for the backward pass.
struct MlpTile {
  float z1[8][4], z2[8][4];
  uint32_t h1[4][4], h2[4][4];
  uint32_t x[4];
};

template <typename W2Frag>
__device__ __forceinline__ void mlp_tile_forward(const MlpFrags& f, W2Frag&& w2frag, const float* __restrict__ bias1,
                                                 const float* __restrict__ bias2, float bias3,
                                                 const float* __restrict__ nm, const float* __restrict__ x,
                                                 int64_t rows, int64_t r0, int lane, MlpTile& T, float& y_lo,
                                                 float& y_hi) {
  const int g = lane >> 2, t = lane & 3;
  // inputs: normalised, rounded to BF16; features 2t, 2t+1 of rows r0+g and r0+g+8
  float xv[2][2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t r = r0 + g + 8 * h;
    const bool ok = r < rows;
    const float2 v = ok ? *reinterpret_cast<const float2*>(x + r * kIn + 2 * t) : make_float2(0.f, 0.f);
    xv[h][0] = ok ? (v.x - nm[2 * t]) / nm[kIn + 2 * t] : 0.f;
    xv[h][1] = ok ? (v.y - nm[2 * t + 1]) / nm[kIn + 2 * t + 1] : 0.f;
  }
  T.x[0] = pack_bf16(xv[0][0], xv[0][1]);
  T.x[1] = pack_bf16(xv[1][0], xv[1][1]);
  T.x[2] = 0u;  // input columns 8..15 are padding
  T.x[3] = 0u;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float b0 = bias1[8 * nt + 2 * t], b1 = bias1[8 * nt + 2 * t + 1];
    T.z1[nt][0] = b0;
    T.z1[nt][1] = b1;
    T.z1[nt][2] = b0;
    T.z1[nt][3] = b1;
    mma_bf16(T.z1[nt], T.x, f.w1[nt], 0u);
  }
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    T.h1[kk][0] = pack_bf16(gelu(T.z1[2 * kk][0]), gelu(T.z1[2 * kk][1]));
    T.h1[kk][1] = pack_bf16(gelu(T.z1[2 * kk][2]), gelu(T.z1[2 * kk][3]));
    T.h1[kk][2] = pack_bf16(gelu(T.z1[2 * kk + 1][0]), gelu(T.z1[2 * kk + 1][1]));
    T.h1[kk][3] = pack_bf16(gelu(T.z1[2 * kk + 1][2]), gelu(T.z1[2 * kk + 1][3]));
  }
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float b0 = bias2[8 * nt + 2 * t], b1 = bias2[8 * nt + 2 * t + 1];
    T.z2[nt][0] = b0;
    T.z2[nt][1] = b1;
    T.z2[nt][2] = b0;
    T.z2[nt][3] = b1;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      uint32_t b0, b1;
      w2frag(kk, nt, b0, b1);
      mma_bf16(T.z2[nt], T.h1[kk], b0, b1);
    }
  }
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    T.h2[kk][0] = pack_bf16(gelu(T.z2[2 * kk][0]), gelu(T.z2[2 * kk][1]));
    T.h2[kk][1] = pack_bf16(gelu(T.z2[2 * kk][2]), gelu(T.z2[2 * kk][3]));
    T.h2[kk][2] = pack_bf16(gelu(T.z2[2 * kk + 1][0]), gelu(T.z2[2 * kk + 1][1]));
    T.h2[kk][3] = pack_bf16(gelu(T.z2[2 * kk + 1][2]), gelu(T.z2[2 * kk + 1][3]));
  }
  float o[4] = {bias3, 0.f, bias3, 0.f};
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) mma_bf16(o, T.h2[kk], f.w3[kk][0], f.w3[kk][1]);
  y_lo = o[0];  // column 0 (lanes with t == 0)
  y_hi = o[2];
}

// y[r] = prediction of log s for row r (de-normalised); one warp per 16-row tile
__global__ void __launch_bounds__(256) k_mlp_forward(const __nv_bfloat16* __restrict__ wb, const float* __restrict__ norm,
                                                    int64_t rows, const float* __restrict__ x, float* y) {
  __shared__ float bias[2 * kH + 1];
  __shared__ float nm[kNorm];
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    bias[i] = __bfloat162float(wb[kOffB1 + i]);
    bias[kH + i] = __bfloat162float(wb[kOffB2 + i]);
  }
  if (threadIdx.x == 0) bias[2 * kH] = __bfloat162float(wb[kOffB3]);
  if (threadIdx.x < kNorm) nm[threadIdx.x] = norm[threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  MlpFrags f;
  load_frags(wb, lane, f);
  const int64_t tiles = ceil_div(rows, 16);
  const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t tl = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tl < tiles; tl += wstride) {
    MlpTile T;
    float ylo, yhi;
    const int64_t r0 = tl * 16;
    mlp_tile_forward(
        f, [&](int kk, int nt, uint32_t& b0, uint32_t& b1) { b0 = f.w2[kk][nt][0]; b1 = f.w2[kk][nt][1]; }, bias,
        bias + kH, bias[2 * kH], nm, x, rows, r0, lane, T, ylo, yhi);
    if ((lane & 3) == 0) {
      const int64_t ra = r0 + (lane >> 2), rb = ra + 8;
      if (ra < rows) y[ra] = ylo * nm[2 * kIn + 1] + nm[2 * kIn];
      if (rb < rows) y[rb] = yhi * nm[2 * kIn + 1] + nm[2 * kIn];
    }
  }
}

// ---- training: loss gradient on tensor cores
// A block takes 128 rows at a time (16 per warp).  Each warp runs the forward pass of its
// rows, then the backward pass through the output layer and GELU (dz2 = dy W3 * gelu'(z2))
// and through W2 (dz1 = (dz2 W2^T) * gelu'(z1), an MMA with W2 as the B operand), and
// leaves x, h1, dz2 and dz1 as BF16 rows in shared memory.  The block then forms
// dW2 += h1^T dz2 and dW1 += x^T dz1 as MMAs over the 128 rows (K = rows), each warp owning
// a fixed set of output tiles whose accumulators stay in registers across iterations; the
// bias and W3 gradients are column sums in FP32.  Every sum runs in an order fixed by the
// row count and the grid: the gradient is bit-reproducible.  BF16 operands of every
// product (x, weights, h1, h2, dz2, dz1), FP32 accumulation.
constexpr int kGradRows = 128;   // rows per block iteration
constexpr int kActStride = 72;   // BF16 per shared-memory row of h1, dz2, dz1 (64 + 8 padding)
constexpr int kXStride = 24;     // BF16 per shared-memory row of x (16 + 8 padding)

struct GradSmem {
  __nv_bfloat16 w2t[kH * kActStride];  // W2^T[n][k]: B fragments of the forward layer 2
  __nv_bfloat16 w2[kH * kActStride];   // W2[n][k]: B fragments of dz2 W2^T
  __nv_bfloat16 h1[kGradRows * kActStride];
  __nv_bfloat16 d2[kGradRows * kActStride];
  __nv_bfloat16 d1[kGradRows * kActStride];
  __nv_bfloat16 xs[kGradRows * kXStride];
  float colsum[kSpmvWarps][3][kH];  // per warp: sum dz1, sum dz2, sum h2 dy
  float bias[2 * kH + 1];
  float w3[kH];
  float nm[kNorm];
  double loss[kSpmvWarps];
  float db3[kSpmvWarps];
};

__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_trans(uint32_t (&r)[2], const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}
__device__ __forceinline__ void st_pair(__nv_bfloat16* base, int row, int col, int stride, uint32_t v) {
  *reinterpret_cast<uint32_t*>(base + row * stride + col) = v;
}

__global__ void __launch_bounds__(256) k_mlp_grad(const __nv_bfloat16* __restrict__ wb, const float* __restrict__ norm,
                                                 int64_t rows, const float* __restrict__ x,
                                                 const float* __restrict__ target, float* part, double* loss_part) {
  extern __shared__ __align__(16) unsigned char grad_dyn[];
  GradSmem& S = *reinterpret_cast<GradSmem*>(grad_dyn);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) {
    const int n = i / kH, k = i % kH;
    S.w2[n * kActStride + k] = wb[kOffW2 + n * kH + k];
    S.w2t[k * kActStride + n] = wb[kOffW2 + n * kH + k];
  }
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    S.bias[i] = __bfloat162float(wb[kOffB1 + i]);
    S.bias[kH + i] = __bfloat162float(wb[kOffB2 + i]);
    S.w3[i] = __bfloat162float(wb[kOffW3 + i]);
  }
  if (threadIdx.x == 0) S.bias[2 * kH] = __bfloat162float(wb[kOffB3]);
  if (threadIdx.x < kNorm) S.nm[threadIdx.x] = norm[threadIdx.x];
  for (int i = threadIdx.x; i < kSpmvWarps * 3 * kH; i += blockDim.x) (&S.colsum[0][0][0])[i] = 0.f;
  __syncthreads();
  MlpFrags f;  // W1 and W3 fragments (W2 comes from shared memory)
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
    f.w1[nt] = pack_raw(wb[kOffW1 + (2 * t) * kH + 8 * nt + g], wb[kOffW1 + (2 * t + 1) * kH + 8 * nt + g]);
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const int k0 = 16 * kk + 2 * t;
    f.w3[kk][0] = g == 0 ? pack_raw(wb[kOffW3 + k0], wb[kOffW3 + k0 + 1]) : 0u;
    f.w3[kk][1] = g == 0 ? pack_raw(wb[kOffW3 + k0 + 8], wb[kOffW3 + k0 + 9]) : 0u;
  }
  auto w2t_frag = [&](int kk, int nt, uint32_t& b0, uint32_t& b1) {
    const __nv_bfloat16* p = S.w2t + (8 * nt + g) * kActStride + 16 * kk + 2 * t;
    b0 = *reinterpret_cast<const uint32_t*>(p);
    b1 = *reinterpret_cast<const uint32_t*>(p + 8);
  };
  // output tiles owned by this warp: dW2 rows (h1 units) 16*(warp/2).., columns 32*(warp%2)..
  // (four 8-column tiles); dW1 columns 8*warp..
  const int mt2 = warp >> 1, nt2 = (warp & 1) * 4;
  float acc2[4][4], acc1[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    acc1[q] = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) acc2[q][c] = 0.f;
  }
  double loss = 0.0;
  float db3 = 0.f;
  const float inv_b = 1.f / (float)rows;
  const float tmean = S.nm[2 * kIn], tstd = S.nm[2 * kIn + 1];
  const int64_t iters = ceil_div(rows, kGradRows);
  for (int64_t it = blockIdx.x; it < iters; it += gridDim.x) {
    const int64_t r0 = it * kGradRows + warp * 16;
    MlpTile T;
    float ylo, yhi;
    mlp_tile_forward(f, w2t_frag, S.bias, S.bias + kH, S.bias[2 * kH], S.nm, x, rows, r0, lane, T, ylo, yhi);
    // dy of rows g and g + 8 (computed in the lane holding the prediction, t == 0)
    float dya = 0.f, dyb = 0.f;
    if (t == 0) {
      const int64_t ra = r0 + g, rb = ra + 8;
      if (ra < rows) {
        const float e = ylo - (target[ra] - tmean) / tstd;
        dya = 2.f * e * inv_b;
        loss += (double)e * (double)e;
      }
      if (rb < rows) {
        const float e = yhi - (target[rb] - tmean) / tstd;
        dyb = 2.f * e * inv_b;
        loss += (double)e * (double)e;
      }
      db3 += dya + dyb;
    }
    dya = __shfl_sync(0xffffffffu, dya, lane & ~3);
    dyb = __shfl_sync(0xffffffffu, dyb, lane & ~3);
    // dz2 = dy W3 gelu'(z2) (FP32, C layout), then its BF16 A fragments
    float dz2[8][4];
    float* cs = &S.colsum[warp][0][0];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int c0 = 8 * nt + 2 * t;
      const float wa = S.w3[c0], wbv = S.w3[c0 + 1];
      dz2[nt][0] = dya * wa * gelu_grad(T.z2[nt][0]);
      dz2[nt][1] = dya * wbv * gelu_grad(T.z2[nt][1]);
      dz2[nt][2] = dyb * wa * gelu_grad(T.z2[nt][2]);
      dz2[nt][3] = dyb * wbv * gelu_grad(T.z2[nt][3]);
    }
    uint32_t D2[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      D2[kk][0] = pack_bf16(dz2[2 * kk][0], dz2[2 * kk][1]);
      D2[kk][1] = pack_bf16(dz2[2 * kk][2], dz2[2 * kk][3]);
      D2[kk][2] = pack_bf16(dz2[2 * kk + 1][0], dz2[2 * kk + 1][1]);
      D2[kk][3] = pack_bf16(dz2[2 * kk + 1][2], dz2[2 * kk + 1][3]);
    }
    // dz1 = (dz2 W2^T) gelu'(z1): B[k][n] = W2[n][k]
    float dz1[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      dz1[nt][0] = dz1[nt][1] = dz1[nt][2] = dz1[nt][3] = 0.f;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const __nv_bfloat16* p = S.w2 + (8 * nt + g) * kActStride + 16 * kk + 2 * t;
        mma_bf16(dz1[nt], D2[kk], *reinterpret_cast<const uint32_t*>(p), *reinterpret_cast<const uint32_t*>(p + 8));
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) dz1[nt][c] *= gelu_grad(T.z1[nt][c]);
    }
    // column sums of this warp's 16 rows: dz1, dz2 (FP32) and h2 dy (h2 as the BF16 operand)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const uint32_t hp0 = T.h2[nt >> 1][(nt & 1) * 2], hp1 = T.h2[nt >> 1][(nt & 1) * 2 + 1];
      const float h2a0 = __uint_as_float(hp0 << 16), h2a1 = __uint_as_float(hp0 & 0xFFFF0000u);
      const float h2b0 = __uint_as_float(hp1 << 16), h2b1 = __uint_as_float(hp1 & 0xFFFF0000u);
      float v[3][2] = {{dz1[nt][0] + dz1[nt][2], dz1[nt][1] + dz1[nt][3]},
                       {dz2[nt][0] + dz2[nt][2], dz2[nt][1] + dz2[nt][3]},
                       {h2a0 * dya + h2b0 * dyb, h2a1 * dya + h2b1 * dyb}};
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int o = 4; o < 32; o <<= 1) v[q][c] += __shfl_xor_sync(0xffffffffu, v[q][c], o);
      if (g == 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          cs[q * kH + 8 * nt + 2 * t] += v[q][0];
          cs[q * kH + 8 * nt + 2 * t + 1] += v[q][1];
        }
      }
    }
    // BF16 rows of x, h1, dz2, dz1 for the block's weight-gradient products
    const int rw = warp * 16;
    st_pair(S.xs, rw + g, 2 * t, kXStride, T.x[0]);
    st_pair(S.xs, rw + g + 8, 2 * t, kXStride, T.x[1]);
    st_pair(S.xs, rw + g, 8 + 2 * t, kXStride, 0u);
    st_pair(S.xs, rw + g + 8, 8 + 2 * t, kXStride, 0u);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      st_pair(S.h1, rw + g, 16 * kk + 2 * t, kActStride, T.h1[kk][0]);
      st_pair(S.h1, rw + g + 8, 16 * kk + 2 * t, kActStride, T.h1[kk][1]);
      st_pair(S.h1, rw + g, 16 * kk + 8 + 2 * t, kActStride, T.h1[kk][2]);
      st_pair(S.h1, rw + g + 8, 16 * kk + 8 + 2 * t, kActStride, T.h1[kk][3]);
      st_pair(S.d2, rw + g, 16 * kk + 2 * t, kActStride, D2[kk][0]);
      st_pair(S.d2, rw + g + 8, 16 * kk + 2 * t, kActStride, D2[kk][1]);
      st_pair(S.d2, rw + g, 16 * kk + 8 + 2 * t, kActStride, D2[kk][2]);
      st_pair(S.d2, rw + g + 8, 16 * kk + 8 + 2 * t, kActStride, D2[kk][3]);
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      st_pair(S.d1, rw + g, 8 * nt + 2 * t, kActStride, pack_bf16(dz1[nt][0], dz1[nt][1]));
      st_pair(S.d1, rw + g + 8, 8 * nt + 2 * t, kActStride, pack_bf16(dz1[nt][2], dz1[nt][3]));
    }
    __syncthreads();
    // dW2 += h1^T dz2 and dW1 += x^T dz1 over the block's 128 rows (K = rows, 8 steps of 16)
    const int q = lane >> 3, i8 = lane & 7;  // ldmatrix: matrix q, row i8 of it
#pragma unroll 2
    for (int ks = 0; ks < kGradRows / 16; ++ks) {
      const int rA = 16 * ks + ((q & 2) ? 8 : 0) + i8;  // A = h1^T: matrices (rows, cols) of h1
      uint32_t a[4];
      ldsm_x4_trans(a, S.h1 + rA * kActStride + 16 * mt2 + ((q & 1) ? 8 : 0));
      // B = dz2 rows 16ks.., two column tiles per x4
#pragma unroll
      for (int p2 = 0; p2 < 2; ++p2) {
        uint32_t b[4];
        const int rB = 16 * ks + ((q & 1) ? 8 : 0) + i8;
        ldsm_x4_trans(b, S.d2 + rB * kActStride + 8 * (nt2 + 2 * p2 + (q >> 1)));
        mma_bf16(acc2[2 * p2], a, b[0], b[1]);
        mma_bf16(acc2[2 * p2 + 1], a, b[2], b[3]);
      }
      uint32_t ax[4];
      ldsm_x4_trans(ax, S.xs + rA * kXStride + ((q & 1) ? 8 : 0));
      uint32_t bx[2];
      const int rX = 16 * ks + ((lane >> 3) & 1 ? 8 : 0) + i8;
      ldsm_x2_trans(bx, S.d1 + rX * kActStride + 8 * warp);
      mma_bf16(acc1, ax, bx[0], bx[1]);
    }
    __syncthreads();  // the rows are rewritten by the next iteration
  }
  // this block's partial gradient
  float* o = part + (int64_t)blockIdx.x * kParams;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int col = 8 * (nt2 + p) + 2 * t, row = 16 * mt2 + g;
    o[kOffW2 + row * kH + col] = acc2[p][0];
    o[kOffW2 + row * kH + col + 1] = acc2[p][1];
    o[kOffW2 + (row + 8) * kH + col] = acc2[p][2];
    o[kOffW2 + (row + 8) * kH + col + 1] = acc2[p][3];
  }
  {
    const int col = 8 * warp + 2 * t;  // dW1 rows g < 8 are the inputs; rows 8..15 are padding
    o[kOffW1 + g * kH + col] = acc1[0];
    o[kOffW1 + g * kH + col + 1] = acc1[1];
  }
  if (t == 0) {
    S.loss[warp] = loss;  // lanes with t == 0 hold partial losses; sum them in lane order
  }
  __syncwarp();
  double lw = loss;
  for (int o2 = 16; o2 > 0; o2 >>= 1) lw += __shfl_xor_sync(0xffffffffu, lw, o2);
  float dw = db3;
  for (int o2 = 16; o2 > 0; o2 >>= 1) dw += __shfl_xor_sync(0xffffffffu, dw, o2);
  if (lane == 0) {
    S.loss[warp] = lw;
    S.db3[warp] = dw;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < 3 * kH; j += blockDim.x) {
    float a = 0.f;
    for (int w = 0; w < kSpmvWarps; ++w) a += (&S.colsum[w][0][0])[j];
    const int qq = j / kH, c = j % kH;
    o[(qq == 0 ? kOffB1 : (qq == 1 ? kOffB2 : kOffW3)) + c] = a;
  }
  if (threadIdx.x == 0) {
    double l = 0.0;
    float b3 = 0.f;
    for (int w = 0; w < kSpmvWarps; ++w) {
      l += S.loss[w];
      b3 += S.db3[w];
    }
    o[kOffB3] = b3;
    loss_part[blockIdx.x] = l;
  }
}

__global__ void k_mlp_reduce(const float* __restrict__ part, int blocks, float* grad, const double* __restrict__ lp,
                             double* loss, int64_t rows) {
  WGRID_STRIDE(i, kParams) {
    float a = 0.f;
    for (int b = 0; b < blocks; ++b) a += part[(int64_t)b * kParams + i];
    grad[i] = a;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < blocks; ++b) s += lp[b];
    *loss = s / (double)rows;
  }
}

// Adam (Kingma & Ba, 2015) on the FP32 master weights; refreshes the BF16 copy
__global__ void k_mlp_adam(float* w, float* m, float* v, const float* __restrict__ g, __nv_bfloat16* wb, float lr,
                           float b1, float b2, float eps, float c1, float c2) {
  WGRID_STRIDE(i, kParams) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void k_scatter_f64_w(const double* __restrict__ in, const int32_t* __restrict__ perm, int64_t n,
                                double* out) {
  WGRID_STRIDE(k, n) out[perm[k]] = in[k];
}

// s_0 from the prediction: exp(yhat) for users with followers, c for the others (exact)
__global__ void k_warm_s0(const float* __restrict__ yhat, const float* __restrict__ x, const double* __restrict__ lam,
                          const double* __restrict__ mu, int64_t n, double* s0) {
  WGRID_STRIDE(i, n) {
    const double c = mu[i] * (1.0 / (lam[i] + mu[i]));  // as the build forms c
    const bool has_followers = x[i * kIn] > 0.f;
    double v = has_followers ? exp((double)yhat[i]) : c;
    s0[i] = v < c ? c : v;  // s_i >= c_i always holds at the fixed point
  }
}

}  // namespace

// ---------------------------------------------------------------- host side

// [n][8] features, internal order, into x (device): the four base features, then their
// means over each user's followers in one load-balanced product with four FP32 sums
void compute_features(Graph& g, float* x) {
  cudaStream_t s = g.stream;
  Allocator& al = g.al;
  const int64_t n = g.n;
  const int64_t nu = (int64_t)g.nX + g.nU;
  k_base_features<<<wgrid(n), 256, 0, s>>>(g.row_ptr.get(), g.n_rows, g.n_leaders.get(), g.lam64.get(), g.mu64.get(),
                                           n, x);
  PSI_LAUNCHED();
  if (g.num_tiles == 0) return;
  DBuf<F4> f(al, (size_t)nu + 1);
  k_features_to_u<<<wgrid(nu + 1), 256, 0, s>>>(x, g.nX, g.nR, nu, f.get());
  PSI_LAUNCHED();
  DBuf<DevState> st(al, 1);
  PSI_CUDA(cudaMemsetAsync(st.get(), 0, sizeof(DevState), s));
  int per_sm = 0;
  PSI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmv<F4, EpiMean4>, kSpmvThreads, 0));
  const int grid = spmv_blocks(per_sm, g.num_tiles);
  DBuf<double> gap_part(al, (size_t)grid);
  DBuf<F4> ch(al, (size_t)g.num_tiles), ct(al, (size_t)g.num_tiles);
  EpiMean4 epi{g.row_ptr.get(), x};
  SpmvArgs a{};
  a.row_ptr = g.row_ptr.get();
  a.col = g.col.get();
  a.tile_row = g.tile_row.get();
  a.tile = g.tile;
  a.num_tiles = g.num_tiles;
  a.n_rows = g.n_rows;
  a.m = g.m_unique;
  a.state = st.get();
  a.gap_part = gap_part.get();
  a.carry_head = ch.get();
  a.carry_tail = ct.get();
  k_spmv<F4, EpiMean4><<<grid, kSpmvThreads, 0, s>>>(a, f.get(), epi);
  PSI_LAUNCHED();
  if (g.num_fix > 0) {
    int fgrid = fix_blocks(g.num_fix);
    DBuf<double> gap_fix(al, (size_t)fgrid);
    FixArgs fa{};
    fa.row_ptr = g.row_ptr.get();
    fa.tile_row = g.tile_row.get();
    fa.tile = g.tile;
    fa.fix_tile = g.fix_tile.get();
    fa.num_fix = g.num_fix;
    fa.state = st.get();
    fa.gap_fix = gap_fix.get();
    fa.carry_head = ch.get();
    fa.carry_tail = ct.get();
    k_fixup<F4, EpiMean4><<<fgrid, kFixThreads, 0, s>>>(fa, epi);
    PSI_LAUNCHED();
  }
}

struct Mlp {
  Allocator al;
  cudaStream_t stream = nullptr;
  DBuf<float> w, m, v, grad, norm;
  DBuf<__nv_bfloat16> wb;
  DBuf<float> part;
  DBuf<double> loss_part, loss;
  int grid = 0;
  int64_t step = 0;
};

// deterministic initialisation: W ~ U(-a, a), a = sqrt(6 / fan_in) (He et al. 2015, uniform
// form), biases 0, from SplitMix64 counters
void mlp_init_host(uint64_t seed, std::vector<float>& w) {
  w.assign(kParams, 0.f);
  auto draw = [&](uint64_t i) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ULL * (i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-53;
  };
  const double a1 = std::sqrt(6.0 / kIn), a2 = std::sqrt(6.0 / kH), a3 = std::sqrt(6.0 / kH);
  for (int i = 0; i < kIn * kH; ++i) w[kOffW1 + i] = (float)((2 * draw(i) - 1) * a1);
  for (int i = 0; i < kH * kH; ++i) w[kOffW2 + i] = (float)((2 * draw(10000 + i) - 1) * a2);
  for (int i = 0; i < kH; ++i) w[kOffW3 + i] = (float)((2 * draw(20000 + i) - 1) * a3);
}

}  // namespace psi

struct psi_mlp {
  psi::Mlp m;
};

extern "C" {

psi_status psi_features(const psi_graph* g, float* out) {
  using namespace psi;
  if (!g || !out) {
    set_last_error("graph or output is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  try {
    Graph& gg = const_cast<Graph&>(g->g);
    const int64_t n = gg.n;
    DBuf<float> xi(gg.al, (size_t)n * kIn);
    compute_features(gg, xi.get());
    const bool dev = is_device_pointer(out);
    DBuf<float> tmp;
    float* dst = out;
    if (!dev) {
      tmp.reset(gg.al, (size_t)n * kIn);
      dst = tmp.get();
    }
    k_scatter_rows8<<<wgrid(n * kIn), 256, 0, gg.stream>>>(xi.get(), gg.perm.get(), n, dst);
    PSI_LAUNCHED();
    if (!dev) copy_out(out, dst, sizeof(float) * n * kIn, gg.stream);
    PSI_CUDA(cudaStreamSynchronize(gg.stream));
    return PSI_OK;
  } catch (const PsiError& e) {
    set_last_error(e.what());
    return e.status;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return PSI_ERR_CUDA;
  }
}

psi_status psi_mlp_create(uint64_t seed, void* stream, psi_mlp** out) {
  using namespace psi;
  if (!out) {
    set_last_error("out is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  *out = nullptr;
  psi_mlp* h = new psi_mlp();
  try {
    Mlp& m = h->m;
    m.stream = static_cast<cudaStream_t>(stream);
    m.al.stream = m.stream;
    m.w.reset(m.al, kParams);
    m.m.reset(m.al, kParams);
    m.v.reset(m.al, kParams);
    m.grad.reset(m.al, kParams);
    m.norm.reset(m.al, kNorm);
    m.wb.reset(m.al, kParams);
    m.grid = (int)num_sms() * 4;
    m.part.reset(m.al, (size_t)m.grid * kParams);
    m.loss_part.reset(m.al, (size_t)m.grid);
    m.loss.reset(m.al, 1);
    std::vector<float> w;
    mlp_init_host(seed, w);
    float nm[kNorm];
    for (int i = 0; i < kIn; ++i) {
      nm[i] = 0.f;
      nm[kIn + i] = 1.f;
    }
    nm[2 * kIn] = 0.f;
    nm[2 * kIn + 1] = 1.f;
    PSI_CUDA(cudaMemcpyAsync(m.w.get(), w.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice, m.stream));
    PSI_CUDA(cudaMemcpyAsync(m.norm.get(), nm, sizeof(nm), cudaMemcpyHostToDevice, m.stream));
    PSI_CUDA(cudaMemsetAsync(m.m.get(), 0, sizeof(float) * kParams, m.stream));
    PSI_CUDA(cudaMemsetAsync(m.v.get(), 0, sizeof(float) * kParams, m.stream));
    k_to_bf16<<<wgrid(kParams), 256, 0, m.stream>>>(m.w.get(), kParams, m.wb.get());
    PSI_LAUNCHED();
    PSI_CUDA(cudaStreamSynchronize(m.stream));
  } catch (const PsiError& e) {
    set_last_error(e.what());
    delete h;
    return e.status;
  }
  *out = h;
  return PSI_OK;
}

psi_status psi_mlp_set_params(psi_mlp* h, const float* params, const float* norm) {
  using namespace psi;
  if (!h) {
    set_last_error("model is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  try {
    Mlp& m = h->m;
    if (params) {
      copy_in(m.w.get(), params, sizeof(float) * kParams, m.stream);
      k_to_bf16<<<wgrid(kParams), 256, 0, m.stream>>>(m.w.get(), kParams, m.wb.get());
      PSI_LAUNCHED();
      PSI_CUDA(cudaMemsetAsync(m.m.get(), 0, sizeof(float) * kParams, m.stream));
      PSI_CUDA(cudaMemsetAsync(m.v.get(), 0, sizeof(float) * kParams, m.stream));
      m.step = 0;
    }
    if (norm) copy_in(m.norm.get(), norm, sizeof(float) * kNorm, m.stream);
    PSI_CUDA(cudaStreamSynchronize(m.stream));
    return PSI_OK;
  } catch (const PsiError& e) {
    set_last_error(e.what());
    return e.status;
  }
}

psi_status psi_mlp_get_params(const psi_mlp* h, float* params, float* norm) {
  using namespace psi;
  if (!h) {
    set_last_error("model is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  try {
    const Mlp& m = h->m;
    if (params) copy_out(params, m.w.get(), sizeof(float) * kParams, m.stream);
    if (norm) copy_out(norm, m.norm.get(), sizeof(float) * kNorm, m.stream);
    PSI_CUDA(cudaStreamSynchronize(m.stream));
    return PSI_OK;
  } catch (const PsiError& e) {
    set_last_error(e.what());
    return e.status;
  }
}

psi_status psi_mlp_forward(const psi_mlp* h, int64_t rows, const float* x, float* y) {
  using namespace psi;
  if (!h || !x || !y || rows < 0) {
    set_last_error("model, x or y is NULL, or rows < 0");
    return PSI_ERR_INVALID_ARG;
  }
  if (!is_device_pointer(x) || !is_device_pointer(y)) {
    set_last_error("x and y must be device memory");
    return PSI_ERR_INVALID_ARG;
  }
  try {
    const Mlp& m = h->m;
    if (rows > 0) {
      k_mlp_forward<<<wgrid(rows), 256, 0, m.stream>>>(m.wb.get(), m.norm.get(), rows, x, y);
      PSI_LAUNCHED();
    }
    PSI_CUDA(cudaStreamSynchronize(m.stream));
    return PSI_OK;
  } catch (const PsiError& e) {
    set_last_error(e.what());
    return e.status;
  }
}

psi_status psi_mlp_grad(psi_mlp* h, int64_t rows, const float* x, const float* target, float* grad_out,
                        double* loss_out) {
  using namespace psi;
  if (!h || !x || !target || rows < 1) {
    set_last_error("model, x or target is NULL, or rows < 1");
    return PSI_ERR_INVALID_ARG;
  }
  if (!is_device_pointer(x) || !is_device_pointer(target)) {
    set_last_error("x and target must be device memory");
    return PSI_ERR_INVALID_ARG;
  }
  try {
    Mlp& m = h->m;
    static const bool configured = [] {  // once, thread-safe
      PSI_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GradSmem)));
      return true;
    }();
    (void)configured;
    k_mlp_grad<<<m.grid, 256, sizeof(GradSmem), m.stream>>>(m.wb.get(), m.norm.get(), rows, x, target, m.part.get(),
                                                            m.loss_part.get());
    PSI_LAUNCHED();
    k_mlp_reduce<<<wgrid(kParams), 256, 0, m.stream>>>(m.part.get(), m.grid, m.grad.get(), m.loss_part.get(),
                                                       m.loss.get(), rows);
    PSI_LAUNCHED();
    if (grad_out) copy_out(grad_out, m.grad.get(), sizeof(float) * kParams, m.stream);
    double l = 0.0;
    PSI_CUDA(cudaMemcpyAsync(&l, m.loss.get(), sizeof(double), cudaMemcpyDeviceToHost, m.stream));
    PSI_CUDA(cudaStreamSynchronize(m.stream));
    if (loss_out) *loss_out = l;
    return PSI_OK;
  } catch (const PsiError& e) {
    set_last_error(e.what());
    return e.status;
  }
}

psi_status psi_mlp_adam_step(psi_mlp* h, float lr) {
  using namespace psi;
  if (!h || !(lr > 0.f)) {
    set_last_error("model is NULL or lr <= 0");
    return PSI_ERR_INVALID_ARG;
  }
  try {
    Mlp& m = h->m;
    m.step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - (float)std::pow(b1, (double)m.step), c2 = 1.f - (float)std::pow(b2, (double)m.step);
    k_mlp_adam<<<wgrid(kParams), 256, 0, m.stream>>>(m.w.get(), m.m.get(), m.v.get(), m.grad.get(), m.wb.get(), lr, b1,
                                                     b2, 1e-8f, c1, c2);
    PSI_LAUNCHED();
    return PSI_OK;
  } catch (const PsiError& e) {
    set_last_error(e.what());
    return e.status;
  }
}

// psi_solve from the network's start vector
psi_status psi_solve_warm(psi_graph* g, const psi_mlp* h, double eps, int32_t max_iter, psi_solve_info* info) {
  using namespace psi;
  if (!g || !h) {
    set_last_error("graph or model is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  psi_status result = PSI_OK;
  try {
    Graph& gg = g->g;
    const int64_t n = gg.n;
    DBuf<float> xi(gg.al, (size_t)n * kIn), yhat(gg.al, (size_t)n);
    compute_features(gg, xi.get());
    const Mlp& m = h->m;
    // only users with followers need a prediction (rows [0, n_rows)); the others have s = c
    if (gg.n_rows > 0) {
      k_mlp_forward<<<wgrid(gg.n_rows), 256, 0, gg.stream>>>(m.wb.get(), m.norm.get(), gg.n_rows, xi.get(),
                                                            yhat.get());
      PSI_LAUNCHED();
    }
    DBuf<double> s0i(gg.al, (size_t)n), s0(gg.al, (size_t)n);
    k_warm_s0<<<wgrid(n), 256, 0, gg.stream>>>(yhat.get(), xi.get(), gg.lam64.get(), gg.mu64.get(), n, s0i.get());
    PSI_LAUNCHED();
    // the solver takes s_0 in input order
    k_scatter_f64_w<<<wgrid(n), 256, 0, gg.stream>>>(s0i.get(), gg.perm.get(), n, s0.get());
    PSI_LAUNCHED();
    result = solve(gg, eps, max_iter, s0.get(), info);
  } catch (const PsiError& e) {
    set_last_error(e.what());
    return e.status;
  }
  return result;
}

void psi_mlp_destroy(psi_mlp* h) {
  if (!h) return;
  cudaStreamSynchronize(h->m.stream);
  delete h;
}

}  // extern "C"
