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

__global__ void k_features_to_u(const float* __restrict__ x, int32_t nX, int32_t nR, int64_t nu, D2* f01, D2* f23) {
  WGRID_STRIDE(i, nu + 1) {
    if (i == nu) {
      f01[i] = D2(0.0, 0.0);
      f23[i] = D2(0.0, 0.0);
    } else {
      const int64_t user = i < nX ? i : i + nR;
      const float* o = x + user * kIn;
      f01[i] = D2((double)o[0], (double)o[1]);
      f23[i] = D2((double)o[2], (double)o[3]);
    }
  }
}

// mean over the followers of row r of a pair of base features, into columns c0, c0 + 1
struct EpiMean2 {
  const int32_t* row_ptr;
  float* x;
  int c0;
  __device__ __forceinline__ void row(int32_t r, D2 y, double&, uint64_t, uint64_t) const {
    const double len = (double)(row_ptr[r + 1] - row_ptr[r]);
    x[(int64_t)r * kIn + c0] = (float)(y.a / len);
    x[(int64_t)r * kIn + c0 + 1] = (float)(y.b / len);
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

// y[r] = prediction of log s for row r (de-normalised)
__global__ void __launch_bounds__(256) k_mlp_forward(const __nv_bfloat16* __restrict__ wb, const float* __restrict__ norm,
                                                    int64_t rows, const float* __restrict__ x, float* y) {
  __shared__ float w[kParams];
  __shared__ float nm[kNorm];
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) w[i] = __bfloat162float(wb[i]);
  if (threadIdx.x < kNorm) nm[threadIdx.x] = norm[threadIdx.x];
  __syncthreads();
  WGRID_STRIDE(r, rows) {
    float xi[kIn];
#pragma unroll
    for (int i = 0; i < kIn; ++i) xi[i] = bf16r((x[r * kIn + i] - nm[i]) / nm[kIn + i]);
    float h1[kH];
#pragma unroll
    for (int j = 0; j < kH; ++j) {
      float z = w[kOffB1 + j];
#pragma unroll
      for (int i = 0; i < kIn; ++i) z = fmaf(w[kOffW1 + i * kH + j], xi[i], z);
      h1[j] = gelu(z);
    }
    float out = w[kOffB3];
    for (int k = 0; k < kH; ++k) {
      float z = w[kOffB2 + k];
#pragma unroll
      for (int j = 0; j < kH; ++j) z = fmaf(w[kOffW2 + j * kH + k], h1[j], z);
      out = fmaf(w[kOffW3 + k], gelu(z), out);
    }
    y[r] = out * nm[2 * kIn + 1] + nm[2 * kIn];
  }
}

constexpr int kRowsPerGroup = 16;  // rows per block iteration in training (16 threads per row)

// Gradient of L = (1/B) sum_r (yhat_r - t_r)^2 over normalised targets, per block over a fixed
// set of row groups; part[block][kParams] and loss_part[block].
__global__ void __launch_bounds__(256) k_mlp_grad(const __nv_bfloat16* __restrict__ wb, const float* __restrict__ norm,
                                                 int64_t rows, const float* __restrict__ x,
                                                 const float* __restrict__ target, float* part, double* loss_part) {
  __shared__ float w[kParams];
  __shared__ float nm[kNorm];
  __shared__ float X[kRowsPerGroup][kIn];
  __shared__ float H1[kRowsPerGroup][kH], G1[kRowsPerGroup][kH];
  __shared__ float H2[kRowsPerGroup][kH], G2[kRowsPerGroup][kH];
  __shared__ float DY[kRowsPerGroup];
  __shared__ double lsh[256];
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) w[i] = __bfloat162float(wb[i]);
  if (threadIdx.x < kNorm) nm[threadIdx.x] = norm[threadIdx.x];
  const int t = threadIdx.x;
  const int r = t / 16, p = t % 16;  // row in the group, part of the row
  // thread-owned gradient entries: dW2 entries t, t + 256, ... (16), dW1 entries t, t + 256,
  // b1/b2/W3 entry t (t < 64), b3 (t == 0)
  float gW2[16], gW1[2], gB1 = 0.f, gB2 = 0.f, gW3 = 0.f, gB3 = 0.f;
#pragma unroll
  for (int q = 0; q < 16; ++q) gW2[q] = 0.f;
  gW1[0] = gW1[1] = 0.f;
  double loss = 0.0;
  const float inv_b = 1.f / (float)rows;
  __syncthreads();
  const int64_t groups = ceil_div(rows, kRowsPerGroup);
  for (int64_t gidx = blockIdx.x; gidx < groups; gidx += gridDim.x) {
    const int64_t row = gidx * kRowsPerGroup + r;
    const bool valid = row < rows;
    if (p < kIn) X[r][p] = valid ? bf16r((x[row * kIn + p] - nm[p]) / nm[kIn + p]) : 0.f;
    __syncthreads();
    for (int j = p * 4; j < p * 4 + 4; ++j) {
      float z = w[kOffB1 + j];
#pragma unroll
      for (int i = 0; i < kIn; ++i) z = fmaf(w[kOffW1 + i * kH + j], X[r][i], z);
      H1[r][j] = gelu(z);
      G1[r][j] = gelu_grad(z);
    }
    __syncthreads();
    float ypart = 0.f;
    for (int k = p * 4; k < p * 4 + 4; ++k) {
      float z = w[kOffB2 + k];
      for (int j = 0; j < kH; ++j) z = fmaf(w[kOffW2 + j * kH + k], H1[r][j], z);
      const float h = gelu(z);
      H2[r][k] = h;
      G2[r][k] = gelu_grad(z);
      ypart = fmaf(w[kOffW3 + k], h, ypart);
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) ypart += __shfl_xor_sync(0xffffffffu, ypart, o);  // 16 threads of the row
    if (p == 0) {
      const float yhat = ypart + w[kOffB3];
      const float tn = valid ? (target[row] - nm[2 * kIn]) / nm[2 * kIn + 1] : yhat;
      const float e = yhat - tn;
      DY[r] = valid ? 2.f * e * inv_b : 0.f;
      loss += valid ? (double)e * (double)e : 0.0;
    }
    __syncthreads();
    for (int k = p * 4; k < p * 4 + 4; ++k) G2[r][k] *= w[kOffW3 + k] * DY[r];  // -> dL/dz2
    __syncthreads();
    for (int j = p * 4; j < p * 4 + 4; ++j) {
      float acc = 0.f;
      for (int k = 0; k < kH; ++k) acc = fmaf(w[kOffW2 + j * kH + k], G2[r][k], acc);
      G1[r][j] *= acc;  // -> dL/dz1
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {  // dW2[j][k] = sum_r h1[r][j] dz2[r][k]
      const int e = t + 256 * q, j = e / kH, k = e % kH;
      float acc = 0.f;
#pragma unroll
      for (int rr = 0; rr < kRowsPerGroup; ++rr) acc = fmaf(H1[rr][j], G2[rr][k], acc);
      gW2[q] += acc;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {  // dW1[i][j] = sum_r x[r][i] dz1[r][j]
      const int e = t + 256 * q, i = e / kH, j = e % kH;
      float acc = 0.f;
#pragma unroll
      for (int rr = 0; rr < kRowsPerGroup; ++rr) acc = fmaf(X[rr][i], G1[rr][j], acc);
      gW1[q] += acc;
    }
    if (t < kH) {
      float a1 = 0.f, a2 = 0.f, a3 = 0.f;
      for (int rr = 0; rr < kRowsPerGroup; ++rr) {
        a1 += G1[rr][t];
        a2 += G2[rr][t];
        a3 = fmaf(H2[rr][t], DY[rr], a3);
      }
      gB1 += a1;
      gB2 += a2;
      gW3 += a3;
    }
    if (t == 0) {
      float a = 0.f;
      for (int rr = 0; rr < kRowsPerGroup; ++rr) a += DY[rr];
      gB3 += a;
    }
    __syncthreads();
  }
  float* o = part + (int64_t)blockIdx.x * kParams;
#pragma unroll
  for (int q = 0; q < 16; ++q) o[kOffW2 + t + 256 * q] = gW2[q];
  o[kOffW1 + t] = gW1[0];
  o[kOffW1 + t + 256] = gW1[1];
  if (t < kH) {
    o[kOffB1 + t] = gB1;
    o[kOffB2 + t] = gB2;
    o[kOffW3 + t] = gW3;
  }
  if (t == 0) o[kOffB3] = gB3;
  lsh[t] = loss;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int i = 0; i < 256; ++i) s += lsh[i];
    loss_part[blockIdx.x] = s;
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

// [n][8] features, internal order, into x (device)
void compute_features(Graph& g, float* x) {
  cudaStream_t s = g.stream;
  Allocator& al = g.al;
  const int64_t n = g.n;
  const int64_t nu = (int64_t)g.nX + g.nU;
  k_base_features<<<wgrid(n), 256, 0, s>>>(g.row_ptr.get(), g.n_rows, g.n_leaders.get(), g.lam64.get(), g.mu64.get(),
                                           n, x);
  PSI_LAUNCHED();
  if (g.num_tiles == 0) return;
  DBuf<D2> f01(al, (size_t)nu + 1), f23(al, (size_t)nu + 1);
  k_features_to_u<<<wgrid(nu + 1), 256, 0, s>>>(x, g.nX, g.nR, nu, f01.get(), f23.get());
  PSI_LAUNCHED();
  Schedule sc;  // view of the graph's own schedule
  sc.tiles = g.num_tiles;
  sc.num_fix = g.num_fix;
  DBuf<DevState> st(al, 1);
  PSI_CUDA(cudaMemsetAsync(st.get(), 0, sizeof(DevState), s));
  int per_sm = 0;
  PSI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmv<D2, EpiMean2>, kSpmvThreads, 0));
  const int grid = spmv_blocks(per_sm, g.num_tiles);
  DBuf<double> gap_part(al, (size_t)grid);
  DBuf<D2> ch(al, (size_t)g.num_tiles), ct(al, (size_t)g.num_tiles);
  for (int c0 = 4; c0 <= 6; c0 += 2) {
    const D2* u = c0 == 4 ? f01.get() : f23.get();
    EpiMean2 epi{g.row_ptr.get(), x, c0};
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
    k_spmv<D2, EpiMean2><<<grid, kSpmvThreads, 0, s>>>(a, u, epi);
    PSI_LAUNCHED();
    if (g.num_fix > 0) {
      int fgrid = fix_blocks(g.num_fix);
      DBuf<double> gap_fix(al, (size_t)fgrid);
      FixArgs f{};
      f.row_ptr = g.row_ptr.get();
      f.tile_row = g.tile_row.get();
      f.tile = g.tile;
      f.fix_tile = g.fix_tile.get();
      f.num_fix = g.num_fix;
      f.state = st.get();
      f.gap_fix = gap_fix.get();
      f.carry_head = ch.get();
      f.carry_tail = ct.get();
      k_fixup<D2, EpiMean2><<<fgrid, kFixThreads, 0, s>>>(f, epi);
      PSI_LAUNCHED();
    }
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
    k_mlp_grad<<<m.grid, 256, 0, m.stream>>>(m.wb.get(), m.norm.get(), rows, x, target, m.part.get(),
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
