// Workspace-free plan pass: the column sums c = P^T a of the plan P^k(gamma)
// and the gradient norm ||c - b||, for callers that cannot allocate device
// memory at all.
//
// Some callers cannot call cudaMalloc or hand over a workspace: code that runs
// inside a host callback or another library's allocator-free section, code
// whose memory pool is owned by a runtime that forbids foreign allocations,
// or a process that must not grow its device footprint after start-up.  For
// them this entry point keeps its scratch in one fixed array compiled into
// the library (below), so a call allocates nothing.
//
// Costs of that choice, which every user of this entry point must accept:
//  * the array (kScratchDoubles doubles, about 4.1 MiB) is reserved on
//    every GPU that loads the library, for as long as the process lives;
//  * every call shares the array, so calls whose kernels overlap on the GPU
//    (different streams, or different host threads on the same device) race
//    and corrupt each other's results: serialise them on one stream;
//  * the first call on each device looks the array's device address up
//    (cudaGetSymbolAddress with that device current); make that first call
//    before any CUDA stream capture begins.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>

#include "../../include/ibsn.h"
#include "common.cuh"
#include "internal.h"

namespace {

constexpr int kNoAllocMaxN = 4096;       // widest problem (columns) accepted
constexpr int kNoAllocBlocks = 128;      // row blocks, one column partial each
constexpr int kNoAllocThreads = 256;
// Gamma + gamma and log b (2 x kNoAllocMaxN), column partials
// (kNoAllocBlocks x kNoAllocMaxN), and a slot for ||g||^2 at the end
constexpr size_t kScratchDoubles = (size_t)(kNoAllocBlocks + 2) * kNoAllocMaxN + 32;

// The scratch.  In host code this name is only a host-side handle: host code
// must use the address returned by cudaGetSymbolAddress, never the name.
static __device__ __align__(256) double g_plan_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_dev_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device (set-up on first use).
int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return IBSN_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_dev_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_plan_scratch) != cudaSuccess || p == nullptr) return IBSN_ERR_CUDA;
    g_dev_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_dev_ptr[dev];
  return IBSN_OK;
}

__device__ __forceinline__ double cost_entry(const ibsn::CostRef& c, int i, int j) {
  if (c.kind == 0) return static_cast<const double*>(c.C)[(int64_t)i * c.ldc + j];
  if (c.kind == 1) return (double)static_cast<const float*>(c.C)[(int64_t)i * c.ldc + j];
  const int ri = i / c.gw, ci = i - ri * c.gw, rj = j / c.gw, cj = j - rj * c.gw;
  return c.scale * (double)((ri - rj) * (ri - rj) + (ci - cj) * (ci - cj));
}

// Block b owns rows [b*rpb, (b+1)*rpb) and column partial b of the scratch.
// Exponent of entry (i, j): log b_j + (Gamma_j + gamma_j - (k+1) C_ij) / eta.
__global__ void __launch_bounds__(kNoAllocThreads)
k_plan_noalloc(ibsn::CostRef cost, int m, int n, int rpb, const double* __restrict__ logb,
               const double* __restrict__ G, double lam, double inv_eta, const double* __restrict__ a,
               double* __restrict__ part) {
  __shared__ double sh[kNoAllocThreads / 32];
  double* mine = part + (size_t)blockIdx.x * n;
  for (int j = threadIdx.x; j < n; j += kNoAllocThreads) mine[j] = 0.0;  // partials start at zero
  const int r0 = blockIdx.x * rpb, r1 = min(m, r0 + rpb);
  for (int i = r0; i < r1; ++i) {
    double mx = -ibsn::kInf;
    for (int j = threadIdx.x; j < n; j += kNoAllocThreads)
      mx = fmax(mx, logb[j] + G[j] * inv_eta - lam * cost_entry(cost, i, j));
    mx = ibsn::block_max<kNoAllocThreads>(mx, sh);
    double s[1] = {0.0};
    for (int j = threadIdx.x; j < n; j += kNoAllocThreads)
      s[0] += exp(logb[j] + G[j] * inv_eta - lam * cost_entry(cost, i, j) - mx);
    ibsn::block_sum<kNoAllocThreads, 1>(s, sh);
    const double w = a[i] / s[0];
    for (int j = threadIdx.x; j < n; j += kNoAllocThreads)
      mine[j] += w * exp(logb[j] + G[j] * inv_eta - lam * cost_entry(cost, i, j) - mx);
  }
}

// c_j = sum of the block partials; ||c - b||^2 into the last scratch slot.
__global__ void __launch_bounds__(1024) k_plan_noalloc_finish(int n, int nb, const double* __restrict__ part,
                                                              const double* __restrict__ b, double* colsum,
                                                              double* g2_out) {
  __shared__ double sh[32];
  double g2[1] = {0.0};
  for (int j = threadIdx.x; j < n; j += 1024) {
    double c = 0.0;
    for (int q = 0; q < nb; ++q) c += part[(size_t)q * n + j];
    colsum[j] = c;
    const double g = c - b[j];
    g2[0] += g * g;
  }
  ibsn::block_sum<1024, 1>(g2, sh);
  if (threadIdx.x == 0) *g2_out = g2[0];
}

__global__ void k_sum_vectors(int n, const double* x, const double* y, double* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = (x ? x[j] : 0.0) + (y ? y[j] : 0.0);
}

__global__ void k_log_vec(int n, const double* x, double* y) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) y[j] = log(x[j]);
}

}  // namespace

extern "C" int ibsn_plan_pass_noalloc(const ibsn_problem* prob, int64_t k, const double* Gamma,
                                      const double* gamma, double* colsum, double* grad_norm, void* stream) {
  if (!prob || !colsum || k < 0) return IBSN_ERR_INVALID_ARG;
  if (prob->m < 1 || prob->n < 1 || !prob->a || !prob->b || !(prob->eta > 0.0)) return IBSN_ERR_INVALID_ARG;
  if (prob->n > kNoAllocMaxN || prob->m > (int64_t)0x7fffffff) return IBSN_ERR_UNSUPPORTED;
  if ((prob->cost_kind == IBSN_COST_DENSE_F64 || prob->cost_kind == IBSN_COST_DENSE_F32) &&
      (!prob->C || prob->ldc < prob->n))
    return IBSN_ERR_INVALID_ARG;
  if (prob->cost_kind == IBSN_COST_GRID2D &&
      ((int64_t)prob->grid_h * prob->grid_w != prob->m || prob->m != prob->n))
    return IBSN_ERR_INVALID_ARG;
  if (prob->cost_kind < 0 || prob->cost_kind > 2) return IBSN_ERR_INVALID_ARG;
  double* scratch = nullptr;
  const int r = scratch_for_current_device(&scratch);
  if (r != IBSN_OK) return r;
  const int m = (int)prob->m, n = (int)prob->n;
  cudaStream_t st = (cudaStream_t)stream;
  // scratch layout: [G = Gamma + gamma (n)] [log b (n)] [partials (nb x n)] [||g||^2]
  const int nb = m < kNoAllocBlocks ? m : kNoAllocBlocks;
  const int rpb = (m + nb - 1) / nb;
  const int nbl = (m + rpb - 1) / rpb;
  double* G = scratch;
  double* logb = scratch + n;
  double* part = scratch + 2 * (size_t)n;
  double* g2 = scratch + kScratchDoubles - 1;
  ibsn::CostRef cost{prob->C, prob->ldc, prob->cost_kind, prob->grid_w, prob->cost_scale};
  const unsigned vb = (unsigned)((n + 255) / 256);
  k_sum_vectors<<<vb, 256, 0, st>>>(n, Gamma, gamma, G);
  k_log_vec<<<vb, 256, 0, st>>>(n, prob->b, logb);
  k_plan_noalloc<<<nbl, kNoAllocThreads, 0, st>>>(cost, m, n, rpb, logb, G, (double)(k + 1) / prob->eta,
                                                  1.0 / prob->eta, prob->a, part);
  k_plan_noalloc_finish<<<1, 1024, 0, st>>>(n, nbl, part, prob->b, colsum, g2);
  if (cudaGetLastError() != cudaSuccess) return IBSN_ERR_CUDA;
  if (grad_norm) {
    double h = 0.0;
    if (cudaMemcpyAsync(&h, g2, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) return IBSN_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return IBSN_ERR_CUDA;
    *grad_norm = std::sqrt(h);
  }
  return IBSN_OK;
}
