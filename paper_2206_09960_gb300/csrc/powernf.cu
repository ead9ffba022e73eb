// powernf.cu -- Power-NF (Algorithm 1) on the GPU: the method Power-psi replaces, with the
// newsfeed vectors of many origins stepped at once.
//
// For an origin i, the vector p_i over users j (the share of j's newsfeed that holds i's
// posts) solves p_i = A p_i + b_i (Eq. 8), with a_jk = mu_k / sigma_j and b_ji = lambda_i /
// sigma_j for leaders k, i of j (Sec. II).  Algorithm 1 iterates p_i <- A p_i + b_i from
// p_i = b_i until ||p_i^t - p_i^{t-1}||_1 <= eps (a gap of 1 before the first step), then
// q_i^(n) = c_n p_i^(n) + d_i 1{n = i} (Eq. 7) and psi_i = (1/N) sum_n q_i^(n) (Eq. 1).
//
// Only users with leaders have a nonzero entry in any p_i (the others have an empty
// newsfeed), and only origins with followers have a nonzero p_i (b_i = 0 otherwise, so
// p_i = 0 and psi_i = d_i / N).  In the internal numbering the first are the gathered index
// space [0, nG) and the second the rows [0, n_rows).  The vectors of a pass of C origins
// are the columns of an nG x C matrix P (row g = user, column = origin), all stepped
// together: a block takes a fixed range of rows and 256 origins, forms sum_k a_jk P[k][:]
// over each row's leaders (whole rows of P, read contiguously) plus b_j, and keeps the sum
// of the |change| over its rows; a fixed-order sum of those partials gives each origin's
// gap, and an origin that met its test (or the step cap) is not touched again, as
// Algorithm 1 stops each origin on its own (its last vector is in the buffer its step
// count's parity names); each step runs only over the list of origins still stepping.  A
// user with more than kNfLongRow leaders has its leader list summed in segments of that
// many by a kernel of its own (a hub would otherwise hold one thread per origin for the
// whole list at every step), and the row ranges of the blocks are cut by work (leaders,
// segments and rows), not by row count.  Passes run one after another; C is set so that
// the pass state fits a quarter of the free device memory (6 to 32 GiB).  Every sum runs in an order fixed by the
// graph: results are bit-reproducible and do not depend on C.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "solve.cuh"

namespace psi {

namespace {

constexpr int64_t kNfMaxRows = int64_t(1) << 20;          // users with leaders
constexpr int64_t kNfStateMin = int64_t(6) << 30;         // pass state (both P buffers and the
constexpr int64_t kNfStateMax = int64_t(32) << 30;        // partials): a quarter of the free
                                                          // device memory within these bounds
constexpr int kNfThreads = 256;                           // origins per block
constexpr int kNfUnroll = 8;                              // leader rows loaded at a time
constexpr int64_t kNfRowBlocks = 2048;                    // row ranges (fixed by the graph)
constexpr int kNfGroups = kNfThreads / 32;                // row-block groups in the reductions
constexpr int32_t kNfLongRow = 256;                       // leaders per segment of a long row

// origin (column of the pass) handled by list entry idx: the list of origins still stepping,
// or every column of the pass (list == nullptr, the first step)
__device__ __forceinline__ int32_t nf_column(const int32_t* __restrict__ list, int32_t idx) {
  return list ? list[idx] : idx;
}

// sum_{e in [e0, e1)} a_e src[lead_e][c] in the graph's order, kNfUnroll leader rows loaded
// at a time (a leader without leaders of its own has p = 0 and contributes nothing)
__device__ __forceinline__ double nf_leader_sum(const int32_t* __restrict__ lead, const double* __restrict__ a,
                                                int32_t e0, int32_t e1, int32_t nX, int32_t C, int32_t c,
                                                const double* __restrict__ src) {
  double acc = 0.0;
  for (int32_t e = e0; e < e1; e += kNfUnroll) {
    double x[kNfUnroll];
#pragma unroll
    for (int q = 0; q < kNfUnroll; ++q) {
      const int32_t k = e + q < e1 ? lead[e + q] : nX;
      x[q] = k < nX ? src[(int64_t)k * C + c] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < kNfUnroll; ++q)
      if (e + q < e1) acc += a[e + q] * x[q];
  }
  return acc;
}

// P[g][c] = b_ji for every leader i = i0 + c of user j (gathered index g) in the pass;
// P zeroed before
__global__ void k_nf_init(const int32_t* __restrict__ fptr, const int32_t* __restrict__ lead,
                          const double* __restrict__ b, int32_t i0, int32_t C, double* P) {
  const int64_t g = blockIdx.x;
  for (int32_t e = fptr[g] + threadIdx.x; e < fptr[g + 1]; e += blockDim.x) {
    const int32_t c = lead[e] - i0;
    if (c >= 0 && c < C) P[g * C + c] = b[e];
  }
}

// Partial sums of the long rows: segment s (leaders [seg_lo[s], seg_hi[s]) of one user)
// for every origin still stepping, into seg_acc[s][c].
__global__ void __launch_bounds__(kNfThreads) k_nf_segments(const int32_t* __restrict__ seg_lo,
                                                            const int32_t* __restrict__ seg_hi,
                                                            const int32_t* __restrict__ lead,
                                                            const double* __restrict__ a,
                                                            const int32_t* __restrict__ list, int32_t nact,
                                                            int32_t nX, int32_t C, const double* __restrict__ src,
                                                            double* __restrict__ seg_acc) {
  const int32_t idx = (int32_t)blockIdx.y * kNfThreads + threadIdx.x;
  if (idx >= nact) return;
  const int32_t c = nf_column(list, idx);
  const int32_t sg = blockIdx.x;
  seg_acc[(int64_t)sg * C + c] = nf_leader_sum(lead, a, seg_lo[sg], seg_hi[sg], nX, C, c, src);
}

// One step of every origin still stepping: for the rows g of this block's range, in order,
// dst[g][c] = sum_{k in L(j)} a_jk src[k][c] + b_ji -- the leader sum taken here, or for a
// long row the sum of its segments in order and b_ji found by a binary search of its
// leaders (kept in increasing id) -- and the block's sum of |dst - src| per origin goes to
// part[block][c].
__global__ void __launch_bounds__(kNfThreads) k_nf_step(const int32_t* __restrict__ fptr,
                                                        const int32_t* __restrict__ lead,
                                                        const double* __restrict__ a, const double* __restrict__ b,
                                                        const int32_t* __restrict__ long_first,
                                                        const double* __restrict__ seg_acc,
                                                        const int32_t* __restrict__ row_start,
                                                        const int32_t* __restrict__ list, int32_t nact, int32_t nX,
                                                        int32_t i0, int32_t C, const double* __restrict__ src,
                                                        double* __restrict__ dst, double* __restrict__ part) {
  const int32_t idx = (int32_t)blockIdx.y * kNfThreads + threadIdx.x;
  if (idx >= nact) return;
  const int32_t c = nf_column(list, idx);
  const int32_t i = i0 + c;
  const int32_t g0 = row_start[blockIdx.x], g1 = row_start[blockIdx.x + 1];
  double moved = 0.0;
  for (int32_t g = g0; g < g1; ++g) {
    const int32_t e0 = fptr[g], e1 = fptr[g + 1];
    const int32_t ls = long_first[g];
    double acc = 0.0, bji = 0.0;
    if (ls < 0) {
      acc = nf_leader_sum(lead, a, e0, e1, nX, C, c, src);
      for (int32_t e = e0; e < e1; ++e)
        if (lead[e] == i) bji = b[e];
    } else {
      const int32_t ns = (e1 - e0 + kNfLongRow - 1) / kNfLongRow;
      for (int32_t q = 0; q < ns; ++q) acc += seg_acc[(int64_t)(ls + q) * C + c];
      int32_t lo = e0, hi = e1;  // first leader id >= i
      while (lo < hi) {
        const int32_t mid = lo + (hi - lo) / 2;
        if (lead[mid] < i) lo = mid + 1;
        else hi = mid;
      }
      if (lo < e1 && lead[lo] == i) bji = b[lo];
    }
    const double v = acc + bji;
    const int64_t o = (int64_t)g * C + c;
    moved += fabs(v - src[o]);
    dst[o] = v;
  }
  part[(int64_t)blockIdx.x * C + c] = moved;
}

// Fixed-order sum over the row blocks of part[.][c] for the 32 origins of this block: group
// q of 8 sums blocks q, q + 8, ..., then the 8 group sums are added in group order.
__device__ __forceinline__ double nf_column_sum(const double* __restrict__ part, int32_t nb, int32_t C, int32_t c,
                                                bool on, double (*sh)[32]) {
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  double s = 0.0;
  if (on)
    for (int32_t k = grp; k < nb; k += kNfGroups) s += part[(int64_t)k * C + c];
  sh[grp][lane] = s;
  __syncthreads();
  double t = 0.0;
  if (grp == 0)
    for (int q = 0; q < kNfGroups; ++q) t += sh[q][lane];
  return t;
}

// gap of every active origin of the pass, its step count and stop test; active_count and
// list[0, active_count) receive the origins still stepping
__global__ void __launch_bounds__(kNfThreads) k_nf_gap(const double* __restrict__ part, int32_t nb, int32_t i0,
                                                       int32_t C, double eps, int32_t max_iter, int32_t* active,
                                                       int32_t* steps, double* gap, int32_t* converged,
                                                       int32_t* active_count, int32_t* list) {
  __shared__ double sh[kNfGroups][32];
  const int32_t c = (int32_t)blockIdx.x * 32 + (threadIdx.x & 31);
  const bool on = c < C && active[i0 + c];
  const double g = nf_column_sum(part, nb, C, c, on, sh);
  if (threadIdx.x >= 32 || !on) return;
  const int32_t i = i0 + c;
  gap[i] = g;
  const int32_t t = steps[i] + 1;
  steps[i] = t;
  if (g <= eps) {
    active[i] = 0;
    converged[i] = 1;
  } else if (t >= max_iter) {
    active[i] = 0;
  } else {
    list[atomicAdd(active_count, 1)] = c;  // any order: each origin's arithmetic is its own
  }
}

// part[block][c] = sum over the block's rows g, in order, of c_j P[g][c], P the buffer that
// holds origin c's last vector (step count even: P0, odd: P1)
__global__ void __launch_bounds__(kNfThreads) k_nf_dot(const double* __restrict__ P0, const double* __restrict__ P1,
                                                       const int32_t* __restrict__ steps,
                                                       const double* __restrict__ cvec, int32_t nX, int32_t nR,
                                                       const int32_t* __restrict__ row_start, int32_t i0, int32_t C,
                                                       double* __restrict__ part) {
  const int32_t c = (int32_t)blockIdx.y * kNfThreads + threadIdx.x;
  if (c >= C) return;
  const double* P = (steps[i0 + c] & 1) ? P1 : P0;
  const int32_t g0 = row_start[blockIdx.x], g1 = row_start[blockIdx.x + 1];
  double q = 0.0;
  for (int32_t g = g0; g < g1; ++g) q += cvec[g < nX ? g : g + nR] * P[(int64_t)g * C + c];
  part[(int64_t)blockIdx.x * C + c] = q;
}

// psi_i = (sum_n c_n p_i^(n) + d_i) / N for the origins of the pass, into input order
__global__ void __launch_bounds__(kNfThreads) k_nf_psi(const double* __restrict__ part, int32_t nb, int32_t i0,
                                                       int32_t C, const double* __restrict__ d,
                                                       const int32_t* __restrict__ perm, int64_t n, double* psi) {
  __shared__ double sh[kNfGroups][32];
  const int32_t c = (int32_t)blockIdx.x * 32 + (threadIdx.x & 31);
  const double q = nf_column_sum(part, nb, C, c, c < C, sh);
  if (threadIdx.x >= 32 || c >= C) return;
  const int32_t i = i0 + c;
  psi[perm[i]] = (q + d[i]) / (double)n;
}

// origins without followers: p_i = 0, psi_i = d_i / N
__global__ void k_nf_rest(const double* __restrict__ d, const int32_t* __restrict__ perm, int64_t lo, int64_t n,
                          double* psi) {
  for (int64_t i = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    psi[perm[i]] = d[i] / (double)n;
}

}  // namespace

psi_status power_nf(Graph& g, double eps, int32_t max_iter, int32_t origins_per_pass, double* psi_out,
                    psi_solve_info* info) {
  const int64_t n = g.n;
  const int64_t nG = (int64_t)g.nX + g.nU;  // users with leaders
  const int64_t nr = g.n_rows;              // origins with followers
  PSI_REQUIRE(nG <= kNfMaxRows, PSI_ERR_INVALID_ARG, "psi_power_nf: at most 2^20 users with leaders");
  PSI_REQUIRE(max_iter >= 0 && !std::isnan(eps) && origins_per_pass >= 0, PSI_ERR_INVALID_ARG,
              "bad eps, max_iter or origins_per_pass");
  if (n == 0) {
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->converged = 1;
    }
    return PSI_OK;
  }
  cudaStream_t s = g.stream;
  Allocator& al = g.al;
  // Algorithm 1 starts each origin with gap = 1: eps >= 1 (or max_iter = 0) takes no step
  const bool iterate = 1.0 > eps && max_iter > 0;

  // the leaders of each user with leaders (gathered index g), in increasing internal id,
  // with a_jk and b_jk, from the transposed CSR (row r = leader r, entries = its followers'
  // gathered indices)
  std::vector<int32_t> rp((size_t)nr + 1, 0), col((size_t)std::max<int64_t>(g.m_unique, 1));
  std::vector<double> mu((size_t)n), lam((size_t)n), isig((size_t)n);
  if (nr > 0) {
    PSI_CUDA(cudaMemcpyAsync(rp.data(), g.row_ptr.get(), sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost, s));
    if (g.m_unique > 0)
      PSI_CUDA(cudaMemcpyAsync(col.data(), g.col.get(), sizeof(int32_t) * (size_t)g.m_unique, cudaMemcpyDeviceToHost,
                               s));
  }
  PSI_CUDA(cudaMemcpyAsync(mu.data(), g.mu64.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaMemcpyAsync(lam.data(), g.lam64.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaMemcpyAsync(isig.data(), g.isig64.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaStreamSynchronize(s));
  std::vector<int32_t> fptr((size_t)nG + 1, 0);
  for (int64_t r = 0; r < nr; ++r)
    for (int32_t e = rp[r]; e < rp[r + 1]; ++e) ++fptr[(size_t)col[e] + 1];
  for (int64_t q = 0; q < nG; ++q) fptr[q + 1] += fptr[q];
  const size_t me = (size_t)std::max<int64_t>(g.m_unique, 1);
  std::vector<int32_t> lead(me), fill(fptr.begin(), fptr.end() - 1);
  std::vector<double> a(me), b(me);
  for (int64_t r = 0; r < nr; ++r)  // leaders in increasing internal id for every user
    for (int32_t e = rp[r]; e < rp[r + 1]; ++e) {
      const int32_t q = col[e];
      const int64_t j = q < g.nX ? q : (int64_t)q + g.nR;
      const int32_t o = fill[q]++;
      lead[o] = (int32_t)r;
      a[o] = mu[r] * isig[j];
      b[o] = lam[r] * isig[j];
    }
  // segments of the long rows, and the row ranges of the blocks cut by work (a function of
  // the graph only: the sums' order is fixed)
  std::vector<int32_t> long_first((size_t)std::max<int64_t>(nG, 1), -1), seg_lo, seg_hi;
  std::vector<int64_t> work((size_t)std::max<int64_t>(nG, 1));
  int64_t total = 0;
  for (int64_t q = 0; q < nG; ++q) {
    const int32_t e0 = fptr[q], e1 = fptr[q + 1];
    if (e1 - e0 > kNfLongRow) {
      long_first[q] = (int32_t)seg_lo.size();
      for (int32_t e = e0; e < e1; e += kNfLongRow) {
        seg_lo.push_back(e);
        seg_hi.push_back(std::min(e1, e + kNfLongRow));
      }
      work[q] = 2 + ceil_div(e1 - e0, kNfLongRow) + 32;  // segment sums and the binary search
    } else {
      work[q] = 2 + (e1 - e0);
    }
    total += work[q];
  }
  const int32_t nb = (int32_t)std::max<int64_t>(1, std::min<int64_t>(nG, kNfRowBlocks));
  std::vector<int32_t> row_start((size_t)nb + 1, (int32_t)nG);
  row_start[0] = 0;
  {
    int64_t acc = 0;
    int32_t blk = 1;
    for (int64_t q = 0; q < nG && blk < nb; ++q) {
      acc += work[q];
      if (acc * nb >= total * blk) row_start[blk++] = (int32_t)(q + 1);
    }
  }
  const int64_t nseg = (int64_t)seg_lo.size();
  int64_t C = nr;
  if (origins_per_pass > 0) {
    C = std::min<int64_t>(C, origins_per_pass);
  } else {
    size_t free_b = 0, total_b = 0;
    PSI_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const int64_t budget = std::min(kNfStateMax, std::max(kNfStateMin, (int64_t)(free_b / 4)));
    const int64_t fit = budget / (int64_t)(sizeof(double) * (2 * std::max<int64_t>(nG, 1) + nb + nseg));
    C = std::min<int64_t>(C, std::max<int64_t>(kNfThreads, fit / kNfThreads * kNfThreads));
  }
  // the step and product grids take a pass's origins in their y dimension (at most 65535
  // blocks of kNfThreads)
  C = std::max<int64_t>(std::min<int64_t>(C, int64_t(65535) * kNfThreads), 1);

  const size_t state = (size_t)(std::max<int64_t>(nG, 1) * C);
  const size_t hn = (size_t)std::max<int64_t>(nr, 1);
  DBuf<int32_t> dptr(al, fptr.size()), dlead(al, me), dfirst(al, long_first.size()), drows(al, row_start.size()),
      dseg_lo(al, (size_t)std::max<int64_t>(nseg, 1)), dseg_hi(al, (size_t)std::max<int64_t>(nseg, 1)),
      active(al, hn), steps(al, hn), conv(al, hn), list(al, (size_t)C), cnt(al, 1);
  DBuf<double> da(al, me), db(al, me), P0(al, state), P1(al, state), part(al, (size_t)nb * C),
      seg_acc(al, (size_t)(std::max<int64_t>(nseg, 1) * C)), gap(al, hn), psi(al, (size_t)n);
  PSI_CUDA(cudaMemcpyAsync(dptr.get(), fptr.data(), sizeof(int32_t) * fptr.size(), cudaMemcpyHostToDevice, s));
  PSI_CUDA(cudaMemcpyAsync(dlead.get(), lead.data(), sizeof(int32_t) * me, cudaMemcpyHostToDevice, s));
  PSI_CUDA(cudaMemcpyAsync(dfirst.get(), long_first.data(), sizeof(int32_t) * long_first.size(),
                           cudaMemcpyHostToDevice, s));
  PSI_CUDA(cudaMemcpyAsync(drows.get(), row_start.data(), sizeof(int32_t) * row_start.size(), cudaMemcpyHostToDevice,
                           s));
  if (nseg > 0) {
    PSI_CUDA(cudaMemcpyAsync(dseg_lo.get(), seg_lo.data(), sizeof(int32_t) * nseg, cudaMemcpyHostToDevice, s));
    PSI_CUDA(cudaMemcpyAsync(dseg_hi.get(), seg_hi.data(), sizeof(int32_t) * nseg, cudaMemcpyHostToDevice, s));
  }
  PSI_CUDA(cudaMemcpyAsync(da.get(), a.data(), sizeof(double) * me, cudaMemcpyHostToDevice, s));
  PSI_CUDA(cudaMemcpyAsync(db.get(), b.data(), sizeof(double) * me, cudaMemcpyHostToDevice, s));
  PSI_CUDA(cudaMemsetAsync(steps.get(), 0, sizeof(int32_t) * hn, s));
  PSI_CUDA(cudaMemsetAsync(conv.get(), 0, sizeof(int32_t) * hn, s));
  PSI_CUDA(cudaMemsetAsync(gap.get(), 0, sizeof(double) * hn, s));
  if (nr > 0) {
    std::vector<int32_t> on((size_t)nr, iterate ? 1 : 0);
    PSI_CUDA(cudaMemcpyAsync(active.get(), on.data(), sizeof(int32_t) * nr, cudaMemcpyHostToDevice, s));
  }
  cudaEvent_t t0, t1;
  PSI_CUDA(cudaEventCreate(&t0));
  PSI_CUDA(cudaEventCreate(&t1));
  PSI_CUDA(cudaEventRecord(t0, s));
  for (int64_t i0 = 0; i0 < nr; i0 += C) {
    const int32_t cc = (int32_t)std::min<int64_t>(C, nr - i0);
    const unsigned ctiles = (unsigned)ceil_div(cc, 32);
    if (nG > 0) {
      PSI_CUDA(cudaMemsetAsync(P0.get(), 0, sizeof(double) * (size_t)(nG * cc), s));
      k_nf_init<<<(unsigned)nG, 128, 0, s>>>(dptr.get(), dlead.get(), db.get(), (int32_t)i0, cc, P0.get());
      PSI_LAUNCHED();
    }
    int32_t t = 0;
    double* cur = P0.get();
    double* nxt = P1.get();
    int32_t nact = cc;                // origins stepping: every column at the first step
    const int32_t* alist = nullptr;   // then the list the gap kernel leaves
    // every origin steps at most max_iter times, so max_iter launches end the pass
    while (iterate && t < max_iter) {
      PSI_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t), s));
      const unsigned ytiles = (unsigned)ceil_div(nact, kNfThreads);
      if (nG > 0) {
        if (nseg > 0) {
          k_nf_segments<<<dim3((unsigned)nseg, ytiles), kNfThreads, 0, s>>>(
              dseg_lo.get(), dseg_hi.get(), dlead.get(), da.get(), alist, nact, g.nX, cc, cur, seg_acc.get());
          PSI_LAUNCHED();
        }
        k_nf_step<<<dim3((unsigned)nb, ytiles), kNfThreads, 0, s>>>(dptr.get(), dlead.get(), da.get(), db.get(),
                                                                     dfirst.get(), seg_acc.get(), drows.get(),
                                                                     alist, nact, g.nX, (int32_t)i0, cc, cur, nxt,
                                                                     part.get());
        PSI_LAUNCHED();
      } else {
        PSI_CUDA(cudaMemsetAsync(part.get(), 0, sizeof(double) * (size_t)cc, s));
      }
      k_nf_gap<<<ctiles, kNfThreads, 0, s>>>(part.get(), nG > 0 ? nb : 1, (int32_t)i0, cc, eps, max_iter,
                                             active.get(), steps.get(), gap.get(), conv.get(), cnt.get(), list.get());
      PSI_LAUNCHED();
      std::swap(cur, nxt);
      ++t;
      int32_t left = 0;
      PSI_CUDA(cudaMemcpyAsync(&left, cnt.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      PSI_CUDA(cudaStreamSynchronize(s));
      if (left == 0) break;
      nact = left;
      alist = list.get();
    }
    if (nG > 0) {
      k_nf_dot<<<dim3((unsigned)nb, (unsigned)ceil_div(cc, kNfThreads)), kNfThreads, 0, s>>>(
          P0.get(), P1.get(), steps.get(), g.c64.get(), g.nX, g.nR, drows.get(), (int32_t)i0, cc, part.get());
      PSI_LAUNCHED();
    } else {
      PSI_CUDA(cudaMemsetAsync(part.get(), 0, sizeof(double) * (size_t)cc, s));
    }
    k_nf_psi<<<ctiles, kNfThreads, 0, s>>>(part.get(), nG > 0 ? nb : 1, (int32_t)i0, cc, g.d64.get(),
                                           g.perm.get(), n, psi.get());
    PSI_LAUNCHED();
  }
  if (nr < n) {
    k_nf_rest<<<(unsigned)std::min<int64_t>(ceil_div(n - nr, 256), num_sms() * 4), 256, 0, s>>>(
        g.d64.get(), g.perm.get(), nr, n, psi.get());
    PSI_LAUNCHED();
  }
  PSI_CUDA(cudaEventRecord(t1, s));
  if (psi_out) copy_out(psi_out, psi.get(), sizeof(double) * n, s);
  std::vector<int32_t> hs(hn), hc(hn);
  std::vector<double> hg(hn);
  PSI_CUDA(cudaMemcpyAsync(hs.data(), steps.get(), sizeof(int32_t) * hn, cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaMemcpyAsync(hc.data(), conv.get(), sizeof(int32_t) * hn, cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaMemcpyAsync(hg.data(), gap.get(), sizeof(double) * hn, cudaMemcpyDeviceToHost, s));
  PSI_CUDA(cudaStreamSynchronize(s));
  float ms = 0.f;
  PSI_CUDA(cudaEventElapsedTime(&ms, t0, t1));
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  int64_t matvecs = 0;
  int32_t most = 0;
  bool all = true;
  double worst = 0.0;
  for (int64_t i = 0; i < nr; ++i) {
    matvecs += hs[i];
    most = std::max(most, hs[i]);
    all = all && (hc[i] || (hs[i] == 0 && 1.0 <= eps));  // no step: the starting gap of 1 decides
    if (hs[i] > 0) worst = std::max(worst, hg[i]);
  }
  if (nr < n) {
    // an origin without followers has b_i = 0: every step leaves p_i = 0 with gap 0, so it
    // stops after one step when 0 <= eps and runs to max_iter otherwise
    const int32_t k = !iterate ? 0 : (0.0 <= eps ? 1 : max_iter);
    matvecs += (n - nr) * (int64_t)k;
    most = std::max(most, k);
    all = all && (iterate ? 0.0 <= eps : 1.0 <= eps);
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = most;
    info->converged = all ? 1 : 0;
    info->spmv_launches = (int32_t)std::min<int64_t>(matvecs, INT32_MAX);  // matrix-vector products
    info->gap_s_l1 = worst;
    info->gap_scaled = worst;
    info->ms = ms;
  }
  return all ? PSI_OK : PSI_ERR_NOT_CONVERGED;
}

}  // namespace psi
