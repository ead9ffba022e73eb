// api.cu -- the C ABI declared in include/psi.h.  Every entry point converts internal
// failures (PsiError, CUDA errors, allocation failures) into a psi_status and a
// thread-local message; nothing aborts or traps.
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "solve.cuh"
#include "trace.cuh"

namespace psi {

namespace {
thread_local std::string g_last_error;
std::atomic<int64_t> g_launches{0};
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void set_last_error(const std::string& msg) { g_last_error = msg; }

void throw_cuda(cudaError_t e, const char* what, const char* file, int line) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" + std::to_string(line) + ")";
  if (e == cudaErrorMemoryAllocation) throw PsiError(PSI_ERR_OOM, m);
  throw PsiError(PSI_ERR_CUDA, m);
}

// The library's own stream-ordered pool on each device (used when the caller gives no
// allocator).  It keeps freed memory for reuse instead of returning it at every
// synchronisation, as the device's default pool does with its default settings; the
// default pool itself is left untouched.  psi_trim_memory() gives the cached memory back.
namespace {
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[64] = {};
}  // namespace

cudaMemPool_t library_pool() {
  int dev = 0;
  PSI_CUDA(cudaGetDevice(&dev));
  PSI_REQUIRE(dev >= 0 && dev < 64, PSI_ERR_CUDA, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  if (!g_pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    PSI_CUDA(cudaMemPoolCreate(&pool, &props));
    uint64_t keep = UINT64_MAX;
    PSI_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    g_pools[dev] = pool;
  }
  return g_pools[dev];
}

void* Allocator::alloc(size_t bytes) {
  void* p = nullptr;
  if (has_user) {
    p = user.alloc(bytes, (void*)stream, user.ctx);
    if (!p) throw PsiError(PSI_ERR_OOM, "allocator returned NULL for " + std::to_string(bytes) + " bytes");
  } else {
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, library_pool(), stream);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      throw PsiError(PSI_ERR_OOM, "cudaMallocAsync of " + std::to_string(bytes) + " bytes failed: " +
                                      cudaGetErrorString(e));
    }
  }
  live_bytes += (int64_t)bytes;
  return p;
}

void Allocator::free(void* p, size_t bytes) {
  if (!p) return;
  if (has_user) user.free(p, bytes, (void*)stream, user.ctx);
  else cudaFreeAsync(p, stream);
  live_bytes -= (int64_t)bytes;
}

int64_t num_sms() {
  static const int cached = [] {  // once, thread-safe
    int dev = 0;
    PSI_CUDA(cudaGetDevice(&dev));
    int v = 0;
    PSI_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    return v > 0 ? v : 1;
  }();
  return cached;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a{};
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void copy_in(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return;
  PSI_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
}

void copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return;
  PSI_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
}

namespace {

__global__ void k_scatter_f64(const double* __restrict__ in, const int32_t* __restrict__ perm, int64_t n, double* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[perm[i]] = in[i];
}
__global__ void k_scatter_f32(const float* __restrict__ in, const int32_t* __restrict__ perm, int64_t n, double* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[perm[i]] = (double)in[i];
}

int grid_n(int64_t n) {
  int64_t g = ceil_div(n > 0 ? n : 1, 256);
  int64_t cap = num_sms() * 8;
  return (int)(g < cap ? g : cap);
}

// write n doubles in input order (psi or s) to a host or device pointer
void scatter_out(Graph& g, const void* internal, bool is_f32, double* out) {
  cudaStream_t s = g.stream;
  const int64_t n = g.n;
  const bool dev = is_device_pointer(out);
  DBuf<double> tmp;
  double* dst = out;
  if (!dev) {
    tmp.reset(g.al, (size_t)n);
    dst = tmp.get();
  }
  if (is_f32) k_scatter_f32<<<grid_n(n), 256, 0, s>>>(static_cast<const float*>(internal), g.perm.get(), n, dst);
  else k_scatter_f64<<<grid_n(n), 256, 0, s>>>(static_cast<const double*>(internal), g.perm.get(), n, dst);
  PSI_LAUNCHED();
  if (!dev) copy_out(out, dst, sizeof(double) * n, s);
  PSI_CUDA(cudaStreamSynchronize(s));
}

template <typename F>
psi_status guarded(F&& f) {
  try {
    f();
    return PSI_OK;
  } catch (const PsiError& e) {
    set_last_error(e.what());
    return e.status;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return PSI_ERR_OOM;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return PSI_ERR_CUDA;
  } catch (...) {
    set_last_error("unknown failure");
    return PSI_ERR_CUDA;
  }
}

}  // namespace

void fill_graph_stats(const Graph& g, psi_graph_stats* st) {
  st->n = g.n;
  st->m_input = g.m_input;
  st->m_unique = g.m_unique;
  st->n_rows = g.n_rows;
  st->n_gathered = (int64_t)g.nX + g.nU;
  st->max_followers = g.max_followers;
  st->bnorm_inf = g.bnorm_inf;
  st->rho_inf = g.rho_inf;
  st->build_ms = g.build_ms;
  st->device_bytes = g.al.live_bytes;
  st->spmv_tile = g.tile;
  st->spmv_hot = g.series_hot;
  st->tune_ms = g.tune_ms;
}

}  // namespace psi

using psi::Graph;
using psi::PsiError;

extern "C" {

void psi_options_default(psi_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = PSI_FP32_REFINE;
  opt->tol_mode = PSI_TOL_PSI;
  opt->bnorm_mode = PSI_BNORM_NONE;
  opt->self_loops = PSI_REJECT;
  opt->reorder = 1;
  opt->profile = 0;
  opt->spmv_tile = 0;
  opt->stream = nullptr;
  opt->allocator = nullptr;
  opt->autotune = 1;
  opt->spmv_hot = -1;
}

psi_status psi_graph_create(int64_t n, int64_t m, const int32_t* follower, const int32_t* leader,
                            const double* lambda, const double* mu, const psi_options* opt, psi_graph** out) {
  psi::NvtxRange nvtx_range("psi_graph_create");
  if (out) *out = nullptr;
  psi_graph* h = nullptr;
  psi_status st = psi::guarded([&] {
    PSI_REQUIRE(out, PSI_ERR_INVALID_ARG, "out is NULL");
    PSI_REQUIRE(n >= 1 && n < ((int64_t)1 << 31) - 1, PSI_ERR_INVALID_ARG, "n must be in [1, 2^31 - 2]");
    PSI_REQUIRE(m >= 0 && m < ((int64_t)1 << 31) - 1, PSI_ERR_INVALID_ARG, "m must be in [0, 2^31 - 2]");
    PSI_REQUIRE(lambda && mu, PSI_ERR_INVALID_ARG, "lambda and mu are required");
    PSI_REQUIRE(m == 0 || (follower && leader), PSI_ERR_INVALID_ARG, "follower/leader are NULL");
    psi_options o;
    psi_options_default(&o);
    if (opt) o = *opt;
    PSI_REQUIRE(o.precision >= PSI_FP32 && o.precision <= PSI_FP64, PSI_ERR_INVALID_ARG, "unknown precision");
    PSI_REQUIRE(o.tol_mode == PSI_TOL_PSI || o.tol_mode == PSI_TOL_S_ABS, PSI_ERR_INVALID_ARG, "unknown tol_mode");
    PSI_REQUIRE(o.bnorm_mode == PSI_BNORM_NONE || o.bnorm_mode == PSI_BNORM_INF, PSI_ERR_INVALID_ARG,
                "unknown bnorm_mode");
    PSI_REQUIRE(o.self_loops == PSI_REJECT || o.self_loops == PSI_DROP, PSI_ERR_INVALID_ARG, "unknown self_loops");
    PSI_REQUIRE(o.spmv_tile == 0 || o.spmv_tile == 512 || o.spmv_tile == 1024 || o.spmv_tile == 2048,
                PSI_ERR_INVALID_ARG, "spmv_tile must be 0, 512, 1024 or 2048");
    PSI_REQUIRE(o.autotune == 0 || o.autotune == 1, PSI_ERR_INVALID_ARG, "autotune must be 0 or 1");
    PSI_REQUIRE(o.spmv_hot == -1 || o.spmv_hot == 0 || o.spmv_hot == 24576 || o.spmv_hot == 28672 ||
                    o.spmv_hot == 32768,
                PSI_ERR_INVALID_ARG, "spmv_hot must be -1, 0, 24576, 28672 or 32768");
    h = new psi_graph();
    h->g.opt = o;
    h->g.stream = static_cast<cudaStream_t>(o.stream);
    h->g.al.stream = h->g.stream;
    if (o.allocator) {
      PSI_REQUIRE(o.allocator->alloc && o.allocator->free, PSI_ERR_INVALID_ARG, "allocator callbacks are NULL");
      h->g.al.user = *o.allocator;
      h->g.al.has_user = true;
    }
    psi::build_graph(h->g, n, m, follower, leader, lambda, mu);
    psi::ensure_iteration_buffers(h->g);
  });
  if (st != PSI_OK) {
    if (h) {
      cudaStreamSynchronize(h->g.stream);
      cudaGetLastError();
      if (h->g.host_state) cudaFreeHost(h->g.host_state);
      delete h;
    }
    return st;
  }
  *out = h;
  return PSI_OK;
}

psi_status psi_solve(psi_graph* g, double eps, int32_t max_iter, const double* init_s, psi_solve_info* info) {
  psi::NvtxRange nvtx_range("psi_solve");
  if (!g) {
    psi::set_last_error("graph is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  psi_status result = PSI_OK;
  psi_status st = psi::guarded([&] { result = psi::solve(g->g, eps, max_iter, init_s, info); });
  if (st != PSI_OK) return st;
  if (result == PSI_ERR_NOT_CONVERGED) psi::set_last_error("max_iter reached before the stop test held");
  return result;
}

psi_status psi_pagerank(psi_graph* g, double alpha, double eps, int32_t max_iter, double* pi_out,
                        psi_solve_info* info) {
  psi::NvtxRange nvtx_range("psi_pagerank");
  if (!g) {
    psi::set_last_error("graph is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  psi_status result = PSI_OK;
  psi_status st = psi::guarded([&] { result = psi::pagerank(g->g, alpha, eps, max_iter, pi_out, info); });
  if (st != PSI_OK) return st;
  if (result == PSI_ERR_NOT_CONVERGED) psi::set_last_error("max_iter reached before the pi-tolerance was met");
  return result;
}

psi_status psi_power_nf(psi_graph* g, double eps, int32_t max_iter, int32_t origins_per_pass, double* psi_out,
                        psi_solve_info* info) {
  psi::NvtxRange nvtx_range("psi_power_nf");
  if (!g) {
    psi::set_last_error("graph is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  psi_status result = PSI_OK;
  psi_status st = psi::guarded([&] { result = psi::power_nf(g->g, eps, max_iter, origins_per_pass, psi_out, info); });
  if (st != PSI_OK) return st;
  if (result == PSI_ERR_NOT_CONVERGED) psi::set_last_error("max_iter reached before every origin met its test");
  return result;
}

psi_status psi_scores(const psi_graph* g, double* psi_out) {
  psi::NvtxRange nvtx_range("psi_scores");
  if (!g || !psi_out) {
    psi::set_last_error("graph or output is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  if (!g->g.solved) {
    psi::set_last_error("psi_solve has not produced scores yet");
    return PSI_ERR_NOT_SOLVED;
  }
  return psi::guarded([&] {
    Graph& gg = const_cast<Graph&>(g->g);
    psi::scatter_out(gg, gg.psi64.get(), false, psi_out);
  });
}

psi_status psi_topk(const psi_graph* g, int32_t k, int32_t* ids_out, double* vals_out) {
  psi::NvtxRange nvtx_range("psi_topk");
  if (!g || !ids_out) {
    psi::set_last_error("graph or ids_out is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  if (!g->g.solved) {
    psi::set_last_error("psi_solve has not produced scores yet");
    return PSI_ERR_NOT_SOLVED;
  }
  if (k < 1 || (int64_t)k > g->g.n || k > 65536) {
    psi::set_last_error("k must be in [1, min(n, 65536)]");
    return PSI_ERR_INVALID_ARG;
  }
  return psi::guarded([&] {
    Graph& gg = const_cast<Graph&>(g->g);
    cudaStream_t s = gg.stream;
    const bool dev_ids = psi::is_device_pointer(ids_out);
    const bool dev_vals = vals_out ? psi::is_device_pointer(vals_out) : true;
    psi::DBuf<int32_t> ti;
    psi::DBuf<double> tv;
    int32_t* di = ids_out;
    double* dv = vals_out;
    if (!dev_ids) {
      ti.reset(gg.al, (size_t)k);
      di = ti.get();
    }
    if (vals_out && !dev_vals) {
      tv.reset(gg.al, (size_t)k);
      dv = tv.get();
    }
    psi::topk(gg, k, di, dv);
    if (!dev_ids) psi::copy_out(ids_out, di, sizeof(int32_t) * k, s);
    if (vals_out && !dev_vals) psi::copy_out(vals_out, dv, sizeof(double) * k, s);
    PSI_CUDA(cudaStreamSynchronize(s));
  });
}

psi_status psi_get_iterate(const psi_graph* g, double* s_out) {
  if (!g || !s_out) {
    psi::set_last_error("graph or output is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  if (!g->g.solved) {
    psi::set_last_error("psi_solve has not produced an iterate yet");
    return PSI_ERR_NOT_SOLVED;
  }
  return psi::guarded([&] {
    Graph& gg = const_cast<Graph&>(g->g);
    switch (gg.last_s_kind) {
      case 0: psi::scatter_out(gg, gg.s64.get(), false, s_out); break;
      case 1: psi::scatter_out(gg, gg.s64b.get(), false, s_out); break;
      case 2: psi::scatter_out(gg, gg.s32a.get(), true, s_out); break;
      default: psi::scatter_out(gg, gg.s32b.get(), true, s_out); break;
    }
  });
}

psi_status psi_graph_get_stats(const psi_graph* g, psi_graph_stats* st) {
  if (!g || !st) {
    psi::set_last_error("graph or stats is NULL");
    return PSI_ERR_INVALID_ARG;
  }
  psi::fill_graph_stats(g->g, st);
  return PSI_OK;
}

void psi_graph_destroy(psi_graph* g) {
  if (!g) return;
  cudaStream_t s = g->g.stream;
  try {
    cudaStreamSynchronize(s);
    if (g->g.host_state) cudaFreeHost(g->g.host_state);
    g->g.host_state = nullptr;
    delete g;  // DBuf destructors free device memory on the stream
    cudaGetLastError();
  } catch (...) {
  }
}

const char* psi_status_string(psi_status s) {
  switch (s) {
    case PSI_OK: return "PSI_OK";
    case PSI_ERR_INVALID_ARG: return "PSI_ERR_INVALID_ARG";
    case PSI_ERR_OUT_OF_RANGE_ID: return "PSI_ERR_OUT_OF_RANGE_ID";
    case PSI_ERR_SELF_LOOP: return "PSI_ERR_SELF_LOOP";
    case PSI_ERR_BAD_RATE: return "PSI_ERR_BAD_RATE";
    case PSI_ERR_OOM: return "PSI_ERR_OOM";
    case PSI_ERR_CUDA: return "PSI_ERR_CUDA";
    case PSI_ERR_NOT_CONVERGED: return "PSI_ERR_NOT_CONVERGED";
    case PSI_ERR_TIMEOUT: return "PSI_ERR_TIMEOUT";
    case PSI_ERR_NOT_SOLVED: return "PSI_ERR_NOT_SOLVED";
  }
  return "PSI_UNKNOWN_STATUS";
}

const char* psi_last_error(void) { return psi::g_last_error.c_str(); }

int64_t psi_kernel_launches(void) { return psi::g_launches.load(); }

psi_status psi_trim_memory(void) {
  return psi::guarded([&] {
    cudaMemPool_t pool = psi::library_pool();
    PSI_CUDA(cudaDeviceSynchronize());
    PSI_CUDA(cudaMemPoolTrimTo(pool, 0));
  });
}

int32_t psi_version(void) { return 100; }

}  // extern "C"
