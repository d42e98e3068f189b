// Learned warm start: forward pass, backward pass and Adam step of the
// warm-start network, as kernels of this library.
//
// The network maps the two point clouds of a squared-Euclidean OT problem and
// their marginals to a prediction gamma_hat of the optimal dual potential
// (cost units, centred), which replaces the zero start gamma^{0,0} of Alg. 2.
// Three layers of width 128 with bfloat16 weights and float32 arithmetic:
//   e_i = relu(W_s [x_i, m a_i] + b_s)   (source points)
//   h_j = relu(W_t [y_j, n b_j] + b_t)   (target points)
//   p_s = mean_i e_i,  p_t = mean_j h_j
//   z_j = W_h [h_j; p_s; p_t] + b_h,  o_j = w_o . relu(z_j) + b_o
//   gamma_hat_j = o_j - mean_l o_l
// The per-problem context part of the head, W_h[:,128:384] [p_s; p_t] + b_h,
// is one 128-vector per problem, so the per-point head is a 128x128 product.
//
// Layout in device memory (rows of each problem follow those of the previous
// problems; one row of 128 floats per point and layer):
//   pre_s (sum m x 128), pre_t / z / dz / dpre_t (sum n x 128), features
//   (rows of 4 floats), pools and contexts (per problem).
// Every reduction runs in a fixed order (tile partials, then a sequential
// sum over tiles), so results do not depend on scheduling; there are no
// atomics and no waits between blocks.
//
// These are small contractions (K = 3, 128, 256) over at most a few hundred
// thousand points: the kernels use float32 FMA on CUDA cores with the weight
// matrix staged once per block in shared memory as bfloat16.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <vector>

#include "../../include/ibsn.h"
#include "dense.cuh"
#include "internal.h"

namespace {

constexpr int kH = IBSN_WS_HIDDEN;  // 128
constexpr int kOffWs = 0;                     // W_s 128 x 3
constexpr int kOffBs = kOffWs + kH * 3;       // b_s
constexpr int kOffWt = kOffBs + kH;           // W_t 128 x 3
constexpr int kOffBt = kOffWt + kH * 3;       // b_t
constexpr int kOffWh = kOffBt + kH;           // W_h 128 x 384
constexpr int kOffBh = kOffWh + kH * 3 * kH;  // b_h
constexpr int kOffWo = kOffBh + kH;           // w_o
constexpr int kOffBo = kOffWo + kH;           // b_o
constexpr int kParams = kOffBo + 1;
static_assert(kParams == IBSN_WS_PARAM_COUNT, "parameter layout");
constexpr int kLdWh = 3 * kH;

constexpr int kPtTile = 64;     // points per block: encoder, column sums, source backward
constexpr int kHeadTile = 16;   // target points per block: head forward / backward
constexpr int kSplitRows = 256; // rows per split of a weight-gradient reduction
constexpr int kWgTile = 32;     // output tile edge of a weight-gradient block

__device__ __forceinline__ float bf(const __nv_bfloat16* w, int i) { return __bfloat162float(w[i]); }

// ---------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------

__global__ void k_ws_round(int count, const float* __restrict__ p, __nv_bfloat16* __restrict__ w) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    w[i] = __float2bfloat16_rn(p[i]);
}

// Encoder of one cloud (side 0: source, side 1: target): features
// [coordinate 1, coordinate 2, count * weight] and pre-activations
// W f + b of kPtTile points of problem blockIdx.y.  Block: kH threads.
__global__ void __launch_bounds__(kH) k_ws_encode(const int64_t* __restrict__ off, const double* __restrict__ pts,
                                                  const double* __restrict__ wts, const __nv_bfloat16* __restrict__ wb,
                                                  int offW, int offB, float* __restrict__ feat,
                                                  float* __restrict__ pre) {
  const int q = blockIdx.y;
  const int64_t r0 = off[q], cnt = off[q + 1] - r0;
  const int64_t t0 = (int64_t)blockIdx.x * kPtTile;
  if (t0 >= cnt) return;
  const int rows = (int)(cnt - t0 < kPtTile ? cnt - t0 : kPtTile);
  __shared__ float sf[kPtTile][4];
  const int h = threadIdx.x;
  if (h < rows) {
    const int64_t r = r0 + t0 + h;
    const float f0 = (float)pts[2 * r], f1 = (float)pts[2 * r + 1];
    const float f2 = (float)((double)cnt * wts[r]);
    sf[h][0] = f0;
    sf[h][1] = f1;
    sf[h][2] = f2;
    sf[h][3] = 0.f;
    reinterpret_cast<float4*>(feat)[r] = make_float4(f0, f1, f2, 0.f);
  }
  __syncthreads();
  const float w0 = bf(wb, offW + 3 * h), w1 = bf(wb, offW + 3 * h + 1), w2 = bf(wb, offW + 3 * h + 2);
  const float bias = bf(wb, offB + h);
  for (int j = 0; j < rows; ++j) {
    const float v = fmaf(w2, sf[j][2], fmaf(w1, sf[j][1], fmaf(w0, sf[j][0], bias)));
    pre[(r0 + t0 + j) * kH + h] = v;
  }
}

// Column sums over kPtTile rows of a (rows x 128) matrix per problem
// (optionally of relu of it): partial[(q * tiles + tile) * kH + h].
__global__ void __launch_bounds__(kH) k_ws_colsum_tiles(const int64_t* __restrict__ off, const float* __restrict__ mat,
                                                        int relu, int tiles, float* __restrict__ partial) {
  const int q = blockIdx.y;
  const int64_t r0 = off[q], cnt = off[q + 1] - r0;
  const int64_t t0 = (int64_t)blockIdx.x * kPtTile;
  if (t0 >= cnt) return;
  const int rows = (int)(cnt - t0 < kPtTile ? cnt - t0 : kPtTile);
  const int h = threadIdx.x;
  float s = 0.f;
  for (int j = 0; j < rows; ++j) {
    const float v = mat[(r0 + t0 + j) * kH + h];
    s += relu ? fmaxf(v, 0.f) : v;
  }
  partial[((int64_t)q * tiles + blockIdx.x) * kH + h] = s;
}

// out[q * ldo + h] = (sum over the problem's tiles, in tile order) * (mean ? 1/count : 1)
__global__ void __launch_bounds__(kH) k_ws_colsum_finish(const int64_t* __restrict__ off,
                                                         const float* __restrict__ partial, int tiles, int mean,
                                                         float* __restrict__ out, int ldo) {
  const int q = blockIdx.x, h = threadIdx.x;
  const int64_t cnt = off[q + 1] - off[q];
  const int nt = (int)((cnt + kPtTile - 1) / kPtTile);
  float s = 0.f, c = 0.f;  // compensated sum over the tiles
  for (int t = 0; t < nt; ++t) {
    const float y = partial[((int64_t)q * tiles + t) * kH + h] - c;
    const float u = s + y;
    c = (u - s) - y;
    s = u;
  }
  out[(int64_t)q * ldo + h] = mean ? s / (float)cnt : s;
}

// Per-problem context of the head: b_h + W_h[:, 128:384] [p_s; p_t].
__global__ void __launch_bounds__(kH) k_ws_context(const float* __restrict__ pool, const __nv_bfloat16* __restrict__ wb,
                                                   float* __restrict__ ctx) {
  const int q = blockIdx.x, h = threadIdx.x;
  const float* p = pool + (int64_t)q * 2 * kH;
  const __nv_bfloat16* w = wb + kOffWh + (int64_t)h * kLdWh + kH;
  float acc = bf(wb, kOffBh + h);
  for (int k = 0; k < 2 * kH; ++k) acc = fmaf(__bfloat162float(w[k]), p[k], acc);
  ctx[(int64_t)q * kH + h] = acc;
}

// Head for kHeadTile target points: z = ctx + W_h[:, 0:128] relu(pre_t),
// o = w_o . relu(z) + b_o.  Thread h owns hidden unit h; W_h[:, 0:128] is
// staged transposed in shared memory (row pitch 129 avoids bank conflicts).
__global__ void __launch_bounds__(kH) k_ws_head_fwd(const int64_t* __restrict__ off, const float* __restrict__ pre_t,
                                                    const float* __restrict__ ctx,
                                                    const __nv_bfloat16* __restrict__ wb, float* __restrict__ z,
                                                    float* __restrict__ out) {
  const int q = blockIdx.y;
  const int64_t r0 = off[q], cnt = off[q + 1] - r0;
  const int64_t t0 = (int64_t)blockIdx.x * kHeadTile;
  if (t0 >= cnt) return;
  const int rows = (int)(cnt - t0 < kHeadTile ? cnt - t0 : kHeadTile);
  __shared__ __nv_bfloat16 sW[kH * (kH + 1)];  // sW[k * 129 + h] = W_h[h][k]
  __shared__ float sX[kHeadTile][kH];
  __shared__ float sRed[kH / 32][kHeadTile];
  const int tid = threadIdx.x;
  for (int i = tid; i < kH * kH; i += kH) {
    const int hh = i / kH, k = i % kH;
    sW[k * (kH + 1) + hh] = wb[kOffWh + hh * kLdWh + k];
  }
  for (int i = tid; i < kHeadTile * kH; i += kH) {
    const int j = i / kH, k = i % kH;
    sX[j][k] = j < rows ? fmaxf(pre_t[(r0 + t0 + j) * kH + k], 0.f) : 0.f;
  }
  __syncthreads();
  const int h = tid;
  float acc[kHeadTile];
  const float base = ctx[(int64_t)q * kH + h];
#pragma unroll
  for (int j = 0; j < kHeadTile; ++j) acc[j] = base;
  for (int k = 0; k < kH; ++k) {
    const float w = __bfloat162float(sW[k * (kH + 1) + h]);
#pragma unroll
    for (int j = 0; j < kHeadTile; ++j) acc[j] = fmaf(w, sX[j][k], acc[j]);
  }
  const float wo = bf(wb, kOffWo + h);
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int j = 0; j < kHeadTile; ++j) {
    if (j < rows) z[(r0 + t0 + j) * kH + h] = acc[j];
    float v = wo * fmaxf(acc[j], 0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sRed[warp][j] = v;
  }
  __syncthreads();
  if (tid < rows)
    out[r0 + t0 + tid] = ((sRed[0][tid] + sRed[1][tid]) + (sRed[2][tid] + sRed[3][tid])) + bf(wb, kOffBo);
}

// Deterministic block sum (power-of-two block size NT).
template <int NT, typename T>
__device__ T block_sum(T v, T* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
#pragma unroll
  for (int s = NT / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const T r = sh[0];
  __syncthreads();
  return r;
}

// Centring per problem: gamma_hat = o - mean(o).  With targets: the problem's
// loss (1/n) ||gamma_hat - centred gamma*||^2 and d loss / d o (the batch loss
// is the mean over the Q problems).
constexpr int kCenterThreads = 256;
__global__ void __launch_bounds__(kCenterThreads) k_ws_center(const int64_t* __restrict__ off,
                                                              const float* __restrict__ out, int Q,
                                                              const double* __restrict__ gstar,
                                                              double* __restrict__ gamma_hat,
                                                              double* __restrict__ lossq, float* __restrict__ dout) {
  __shared__ double shd[kCenterThreads];
  const int q = blockIdx.x;
  const int64_t r0 = off[q], n = off[q + 1] - r0;
  double so = 0.0, sg = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += kCenterThreads) {
    so += (double)out[r0 + j];
    if (gstar) sg += gstar[r0 + j];
  }
  const double omean = block_sum<kCenterThreads>(so, shd) / (double)n;
  const double gmean = gstar ? block_sum<kCenterThreads>(sg, shd) / (double)n : 0.0;
  if (gamma_hat)
    for (int64_t j = threadIdx.x; j < n; j += kCenterThreads) gamma_hat[r0 + j] = (double)out[r0 + j] - omean;
  if (!gstar) return;
  double s1 = 0.0, s2 = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += kCenterThreads) {
    const double d = ((double)out[r0 + j] - omean) - (gstar[r0 + j] - gmean);
    s1 += d;
    s2 += d * d;
  }
  const double dsum = block_sum<kCenterThreads>(s1, shd);
  const double d2 = block_sum<kCenterThreads>(s2, shd);
  if (threadIdx.x == 0) lossq[q] = d2 / (double)n;
  const double dmean = dsum / (double)n;
  const double sc = 2.0 / ((double)n * (double)Q);
  for (int64_t j = threadIdx.x; j < n; j += kCenterThreads) {
    const double d = ((double)out[r0 + j] - omean) - (gstar[r0 + j] - gmean);
    dout[r0 + j] = (float)(sc * (d - dmean));
  }
}

// ---------------------------------------------------------------------------
// Backward
// ---------------------------------------------------------------------------

// dz = dout w_o [z > 0], over all target rows.
__global__ void k_ws_dz(int64_t rows, const float* __restrict__ z, const float* __restrict__ dout,
                        const __nv_bfloat16* __restrict__ wb, float* __restrict__ dz) {
  const int64_t total = rows * kH;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int h = (int)(i % kH);
    dz[i] = z[i] > 0.f ? dout[i / kH] * bf(wb, kOffWo + h) : 0.f;
  }
}

// Gradients reaching the pools: dpool[q] = [W_h[:,128:256]^T sdz_q ; W_h[:,256:384]^T sdz_q]
// where sdz_q = sum over the problem's targets of dz.
__global__ void __launch_bounds__(kH) k_ws_dpool(const float* __restrict__ sdz, const __nv_bfloat16* __restrict__ wb,
                                                 float* __restrict__ dpool) {
  const int q = blockIdx.x, k = threadIdx.x;
  const float* s = sdz + (int64_t)q * kH;
  float ps = 0.f, pt = 0.f;
  for (int h = 0; h < kH; ++h) {
    const float v = s[h];
    ps = fmaf(bf(wb, kOffWh + h * kLdWh + kH + k), v, ps);
    pt = fmaf(bf(wb, kOffWh + h * kLdWh + 2 * kH + k), v, pt);
  }
  dpool[(int64_t)q * 2 * kH + k] = ps;
  dpool[(int64_t)q * 2 * kH + kH + k] = pt;
}

// Target encoder gradient for kHeadTile points:
// dpre_t = (W_h[:, 0:128]^T dz + dp_t / n) [pre_t > 0].  Thread k owns input unit k.
__global__ void __launch_bounds__(kH) k_ws_head_bwd(const int64_t* __restrict__ off, const float* __restrict__ dz,
                                                    const float* __restrict__ pre_t, const float* __restrict__ dpool,
                                                    const __nv_bfloat16* __restrict__ wb,
                                                    float* __restrict__ dpre_t) {
  const int q = blockIdx.y;
  const int64_t r0 = off[q], cnt = off[q + 1] - r0;
  const int64_t t0 = (int64_t)blockIdx.x * kHeadTile;
  if (t0 >= cnt) return;
  const int rows = (int)(cnt - t0 < kHeadTile ? cnt - t0 : kHeadTile);
  __shared__ __nv_bfloat16 sW[kH * (kH + 1)];  // sW[h * 129 + k] = W_h[h][k]
  __shared__ float sD[kHeadTile][kH];
  const int tid = threadIdx.x;
  for (int i = tid; i < kH * kH; i += kH) {
    const int hh = i / kH, k = i % kH;
    sW[hh * (kH + 1) + k] = wb[kOffWh + hh * kLdWh + k];
  }
  for (int i = tid; i < kHeadTile * kH; i += kH) {
    const int j = i / kH, hh = i % kH;
    sD[j][hh] = j < rows ? dz[(r0 + t0 + j) * kH + hh] : 0.f;
  }
  __syncthreads();
  const int k = tid;
  float acc[kHeadTile];
  const float base = dpool[(int64_t)q * 2 * kH + kH + k] / (float)cnt;
#pragma unroll
  for (int j = 0; j < kHeadTile; ++j) acc[j] = base;
  for (int hh = 0; hh < kH; ++hh) {
    const float w = __bfloat162float(sW[hh * (kH + 1) + k]);
#pragma unroll
    for (int j = 0; j < kHeadTile; ++j) acc[j] = fmaf(w, sD[j][hh], acc[j]);
  }
#pragma unroll
  for (int j = 0; j < kHeadTile; ++j) {
    if (j < rows) {
      const int64_t i = (r0 + t0 + j) * kH + k;
      dpre_t[i] = pre_t[i] > 0.f ? acc[j] : 0.f;
    }
  }
}

// Source encoder gradient: dpre_s = (dp_s / m) [pre_s > 0] for kPtTile points.
__global__ void __launch_bounds__(kH) k_ws_src_bwd(const int64_t* __restrict__ off, const float* __restrict__ pre_s,
                                                   const float* __restrict__ dpool, float* __restrict__ dpre_s) {
  const int q = blockIdx.y;
  const int64_t r0 = off[q], cnt = off[q + 1] - r0;
  const int64_t t0 = (int64_t)blockIdx.x * kPtTile;
  if (t0 >= cnt) return;
  const int rows = (int)(cnt - t0 < kPtTile ? cnt - t0 : kPtTile);
  const int k = threadIdx.x;
  const float g = dpool[(int64_t)q * 2 * kH + k] / (float)cnt;
  for (int j = 0; j < rows; ++j) {
    const int64_t i = (r0 + t0 + j) * kH + k;
    dpre_s[i] = pre_s[i] > 0.f ? g : 0.f;
  }
}

// Weight gradient G[r][c] = sum over rows of A[row][r] X[row][c] for r < R and
// c < CX, plus a column c = CX of ones (the bias) when `ones` is set.
// Block (split s, output tile): the rows [s kSplitRows, (s+1) kSplitRows) and
// a kWgTile x kWgTile output tile; 256 threads, 4 outputs each.  Partial sums
// go to partial[(s R + r) CXp + c], CXp = CX + ones.
struct WgArgs {
  int64_t rows;
  const float* A;
  int lda, R;
  const float* X;
  int ldx, CX, relu, ones;
  float* partial;
};

__global__ void __launch_bounds__(256) k_ws_wgrad(WgArgs g, int ctiles) {
  __shared__ float sA[kWgTile][kWgTile + 1];
  __shared__ float sX[kWgTile][kWgTile + 4];
  const int s = blockIdx.x;
  const int rt = blockIdx.y / ctiles, ct = blockIdx.y % ctiles;
  const int r0 = rt * kWgTile, c0 = ct * kWgTile;
  const int CXp = g.CX + g.ones;
  const int64_t beg = (int64_t)s * kSplitRows;
  const int64_t end = beg + kSplitRows < g.rows ? beg + kSplitRows : g.rows;
  const int tid = threadIdx.x, tr = tid / 8, tc = tid % 8;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int64_t rb = beg; rb < end; rb += kWgTile) {
    for (int i = tid; i < kWgTile * kWgTile; i += 256) {
      const int ii = i / kWgTile, jj = i % kWgTile;
      const int64_t row = rb + ii;
      const int r = r0 + jj, c = c0 + jj;
      sA[ii][jj] = (row < end && r < g.R) ? g.A[row * g.lda + r] : 0.f;
      float xv = 0.f;
      if (row < end) {
        if (c < g.CX) {
          xv = g.X[row * g.ldx + c];
          if (g.relu) xv = fmaxf(xv, 0.f);
        } else if (c == g.CX && g.ones) {
          xv = 1.f;
        }
      }
      sX[ii][jj] = xv;
    }
    __syncthreads();
#pragma unroll 8
    for (int ii = 0; ii < kWgTile; ++ii) {
      const float a = sA[ii][tr];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fmaf(a, sX[ii][tc * 4 + u], acc[u]);
    }
    __syncthreads();
  }
  const int r = r0 + tr;
  if (r >= g.R) return;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int c = c0 + tc * 4 + u;
    if (c < CXp) g.partial[((int64_t)s * g.R + r) * CXp + c] = acc[u];
  }
}

// Sum of the split partials in split order, written into the gradient vector:
// G[r][c] -> grad[offW + r ldW + c] (c < CX), bias column -> grad[offB + r].
__global__ void k_ws_wgrad_finish(int splits, int R, int CX, int ones, const float* __restrict__ partial,
                                  float* __restrict__ grad, int offW, int ldW, int offB) {
  const int CXp = CX + ones;
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= R * CXp) return;
  const int r = o / CXp, c = o % CXp;
  float s = 0.f, comp = 0.f;
  for (int k = 0; k < splits; ++k) {
    const float y = partial[((int64_t)k * R + r) * CXp + c] - comp;
    const float u = s + y;
    comp = (u - s) - y;
    s = u;
  }
  if (c < CX) grad[offW + r * ldW + c] = s;
  else grad[offB + r] = s;
}

// Adam (Kingma & Ba 2015, Algorithm 1); omb1 = 1 - beta1, omb2 = 1 - beta2,
// bc1 = 1 - beta1^t, bc2 = 1 - beta2^t, each formed in float64 on the host
// (1 - beta2 formed in float32 from beta2 = 0.999 would be off by 1e-5).
__global__ void k_ws_adam(int64_t count, float* __restrict__ p, float* __restrict__ m1, float* __restrict__ m2,
                          const float* __restrict__ g, float lr, float b1, float b2, float omb1, float omb2,
                          float eps, float bc1, float bc2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = fmaf(b1, m1[i], omb1 * gi);
    const float v = fmaf(b2, m2[i], omb2 * gi * gi);
    m1[i] = a;
    m2[i] = v;
    p[i] -= lr * (a / bc1) / (sqrtf(v / bc2) + eps);
  }
}

// ---------------------------------------------------------------------------
// Judge of a start: the semi-dual objective L^0 (Eq. 5 at k = 0), float64.
// Row i contributes a_i (log a_i + M_i + log S_i) with v_ij = log b_j +
// (gamma_j - C_ij)/eta, M_i = max_j v_ij and S_i = sum_j exp(v_ij - M_i),
// accumulated per thread as a running (max, scaled sum) pair and combined
// across the block in a fixed tree.
// ---------------------------------------------------------------------------
constexpr int kSdThreads = 256;

__device__ __forceinline__ void lse_merge(double& m1, double& s1, double m2, double s2) {
  if (m2 == -INFINITY) return;
  if (m1 == -INFINITY) {
    m1 = m2;
    s1 = s2;
    return;
  }
  if (m2 > m1) {
    s1 = s1 * exp(m1 - m2) + s2;
    m1 = m2;
  } else {
    s1 += s2 * exp(m2 - m1);
  }
}

__global__ void __launch_bounds__(kSdThreads) k_semidual0_rows(ibsn::CostRef cost, int m, int64_t n, double inv_eta,
                                                               const double* __restrict__ a,
                                                               const double* __restrict__ logb,
                                                               const double* __restrict__ gam,
                                                               double* __restrict__ rowval) {
  __shared__ double sm[kSdThreads], ss[kSdThreads];
  const int tid = threadIdx.x;
  for (int i = blockIdx.x; i < m; i += gridDim.x) {
    double mx = -INFINITY, s = 0.0;
    for (int64_t j = tid; j < n; j += kSdThreads) {
      const double v = logb[j] + ((gam ? gam[j] : 0.0) - ibsn::cost_at(cost, i, j)) * inv_eta;
      lse_merge(mx, s, v, 1.0);
    }
    sm[tid] = mx;
    ss[tid] = s;
    __syncthreads();
    for (int st = kSdThreads / 2; st > 0; st >>= 1) {
      if (tid < st) {
        double m1 = sm[tid], s1 = ss[tid];
        lse_merge(m1, s1, sm[tid + st], ss[tid + st]);
        sm[tid] = m1;
        ss[tid] = s1;
      }
      __syncthreads();
    }
    if (tid == 0) rowval[i] = a[i] * (log(a[i]) + sm[0] + log(ss[0]));
    __syncthreads();
  }
}

// out = eta sum_i rowval_i - b^T gamma (one block, fixed order)
__global__ void __launch_bounds__(kSdThreads) k_semidual0_finish(int m, int64_t n, double eta,
                                                                 const double* __restrict__ rowval,
                                                                 const double* __restrict__ b,
                                                                 const double* __restrict__ gam,
                                                                 double* __restrict__ out) {
  __shared__ double sh[kSdThreads];
  double r = 0.0, d = 0.0;
  for (int i = threadIdx.x; i < m; i += kSdThreads) r += rowval[i];
  if (gam)
    for (int64_t j = threadIdx.x; j < n; j += kSdThreads) d += b[j] * gam[j];
  const double rs = block_sum<kSdThreads>(r, sh);
  const double ds = block_sum<kSdThreads>(d, sh);
  if (threadIdx.x == 0) *out = eta * rs - ds;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct WsGeom {
  int Q = 0;
  int64_t Ms = 0, Nt = 0, maxm = 0, maxn = 0;
  int tiles_s = 0, tiles_t = 0;  // kPtTile tiles of the largest problem
  int64_t splits = 0;            // weight-gradient splits of the longest row set
};

struct WsBufs {
  int64_t* soff;
  int64_t* toff;
  __nv_bfloat16* wb;
  float *feat_s, *feat_t, *pre_s, *pre_t, *z, *dz, *dpre_t, *dpre_s;
  float *pool, *ctx, *sdz, *dpool, *out, *dout, *tilepart, *wpart;
  double* lossq;
};

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

int ws_geom(const ibsn_ws_batch* B, WsGeom* g) {
  if (!B || B->count < 1 || B->count > 65535 || !B->m || !B->n) return IBSN_ERR_INVALID_ARG;
  g->Q = B->count;
  for (int q = 0; q < B->count; ++q) {
    const int64_t m = B->m[q], n = B->n[q];
    if (m < 1 || n < 1) return IBSN_ERR_INVALID_ARG;
    if (m > IBSN_WS_MAX_POINTS || n > IBSN_WS_MAX_POINTS) return IBSN_ERR_UNSUPPORTED;
    g->Ms += m;
    g->Nt += n;
    g->maxm = m > g->maxm ? m : g->maxm;
    g->maxn = n > g->maxn ? n : g->maxn;
  }
  g->tiles_s = (int)((g->maxm + kPtTile - 1) / kPtTile);
  g->tiles_t = (int)((g->maxn + kPtTile - 1) / kPtTile);
  const int64_t longest = g->Ms > g->Nt ? g->Ms : g->Nt;
  g->splits = (longest + kSplitRows - 1) / kSplitRows;
  return IBSN_OK;
}

// Carve the workspace (base may be null to only count bytes).
size_t ws_carve(const WsGeom& g, char* base, WsBufs* b) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += up256(bytes);
    return p;
  };
  const int64_t Q = g.Q;
  const int tiles = g.tiles_s > g.tiles_t ? g.tiles_s : g.tiles_t;
  b->soff = (int64_t*)take(sizeof(int64_t) * (Q + 1));
  b->toff = (int64_t*)take(sizeof(int64_t) * (Q + 1));
  b->wb = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * kParams);
  b->feat_s = (float*)take(sizeof(float) * 4 * g.Ms);
  b->feat_t = (float*)take(sizeof(float) * 4 * g.Nt);
  b->pre_s = (float*)take(sizeof(float) * kH * g.Ms);
  b->pre_t = (float*)take(sizeof(float) * kH * g.Nt);
  b->z = (float*)take(sizeof(float) * kH * g.Nt);
  b->dz = (float*)take(sizeof(float) * kH * g.Nt);
  b->dpre_t = (float*)take(sizeof(float) * kH * g.Nt);
  b->dpre_s = (float*)take(sizeof(float) * kH * g.Ms);
  b->pool = (float*)take(sizeof(float) * 2 * kH * Q);
  b->ctx = (float*)take(sizeof(float) * kH * Q);
  b->sdz = (float*)take(sizeof(float) * kH * Q);
  b->dpool = (float*)take(sizeof(float) * 2 * kH * Q);
  b->out = (float*)take(sizeof(float) * g.Nt);
  b->dout = (float*)take(sizeof(float) * g.Nt);
  b->tilepart = (float*)take(sizeof(float) * kH * Q * tiles);
  b->wpart = (float*)take(sizeof(float) * (size_t)g.splits * kH * (2 * kH + 1));
  b->lossq = (double*)take(sizeof(double) * Q);
  return off;
}

int check_ws(const WsGeom& g, void* ws, size_t bytes, WsBufs* b) {
  if (!ws || ((uintptr_t)ws & 255) != 0) return IBSN_ERR_WORKSPACE;
  WsBufs probe;
  if (ws_carve(g, nullptr, &probe) > bytes) return IBSN_ERR_WORKSPACE;
  ws_carve(g, (char*)ws, b);
  return IBSN_OK;
}

int launched(void) { return cudaGetLastError() == cudaSuccess ? IBSN_OK : IBSN_ERR_CUDA; }

// Row offsets to the device, weights rounded, encoders, pools, context, head,
// centring.  With gstar: per-problem losses and d loss / d o as well.
int run_forward(const ibsn_ws_batch* B, const WsGeom& g, const WsBufs& w, const float* params, const double* gstar,
                double* gamma_hat, cudaStream_t st) {
  std::vector<int64_t> offs(2 * (g.Q + 1));
  offs[0] = 0;
  offs[g.Q + 1] = 0;
  for (int q = 0; q < g.Q; ++q) {
    offs[q + 1] = offs[q] + B->m[q];
    offs[g.Q + 2 + q] = offs[g.Q + 1 + q] + B->n[q];
  }
  if (cudaMemcpyAsync(w.soff, offs.data(), sizeof(int64_t) * (g.Q + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(w.toff, offs.data() + g.Q + 1, sizeof(int64_t) * (g.Q + 1), cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
    return IBSN_ERR_CUDA;
  // the host vector must outlive the copies
  if (cudaStreamSynchronize(st) != cudaSuccess) return IBSN_ERR_CUDA;
  k_ws_round<<<(kParams + 255) / 256, 256, 0, st>>>(kParams, params, w.wb);
  k_ws_encode<<<dim3(g.tiles_s, g.Q), kH, 0, st>>>(w.soff, B->x, B->a, w.wb, kOffWs, kOffBs, w.feat_s, w.pre_s);
  k_ws_encode<<<dim3(g.tiles_t, g.Q), kH, 0, st>>>(w.toff, B->y, B->b, w.wb, kOffWt, kOffBt, w.feat_t, w.pre_t);
  const int tiles = g.tiles_s > g.tiles_t ? g.tiles_s : g.tiles_t;
  k_ws_colsum_tiles<<<dim3(g.tiles_s, g.Q), kH, 0, st>>>(w.soff, w.pre_s, 1, tiles, w.tilepart);
  k_ws_colsum_finish<<<g.Q, kH, 0, st>>>(w.soff, w.tilepart, tiles, 1, w.pool, 2 * kH);
  k_ws_colsum_tiles<<<dim3(g.tiles_t, g.Q), kH, 0, st>>>(w.toff, w.pre_t, 1, tiles, w.tilepart);
  k_ws_colsum_finish<<<g.Q, kH, 0, st>>>(w.toff, w.tilepart, tiles, 1, w.pool + kH, 2 * kH);
  k_ws_context<<<g.Q, kH, 0, st>>>(w.pool, w.wb, w.ctx);
  const int htiles = (int)((g.maxn + kHeadTile - 1) / kHeadTile);
  k_ws_head_fwd<<<dim3(htiles, g.Q), kH, 0, st>>>(w.toff, w.pre_t, w.ctx, w.wb, w.z, w.out);
  k_ws_center<<<g.Q, kCenterThreads, 0, st>>>(w.toff, w.out, g.Q, gstar, gamma_hat, w.lossq, w.dout);
  ibsn::note_launch(10);
  return launched();
}

void wgrad(const WgArgs& a, int offW, int ldW, int offB, float* grad, cudaStream_t st) {
  const int CXp = a.CX + a.ones;
  const int splits = (int)((a.rows + kSplitRows - 1) / kSplitRows);
  const int rtiles = (a.R + kWgTile - 1) / kWgTile, ctiles = (CXp + kWgTile - 1) / kWgTile;
  k_ws_wgrad<<<dim3(splits, rtiles * ctiles), 256, 0, st>>>(a, ctiles);
  k_ws_wgrad_finish<<<(a.R * CXp + 255) / 256, 256, 0, st>>>(splits, a.R, a.CX, a.ones, a.partial, grad, offW, ldW,
                                                              offB);
  ibsn::note_launch(2);
}

int run_backward(const WsGeom& g, const WsBufs& w, float* grad, cudaStream_t st) {
  const int tiles = g.tiles_s > g.tiles_t ? g.tiles_s : g.tiles_t;
  const int64_t zt = g.Nt * kH;
  const int zb = (int)((zt + 255) / 256 < 4096 ? (zt + 255) / 256 : 4096);
  k_ws_dz<<<zb, 256, 0, st>>>(g.Nt, w.z, w.dout, w.wb, w.dz);
  k_ws_colsum_tiles<<<dim3(g.tiles_t, g.Q), kH, 0, st>>>(w.toff, w.dz, 0, tiles, w.tilepart);
  k_ws_colsum_finish<<<g.Q, kH, 0, st>>>(w.toff, w.tilepart, tiles, 0, w.sdz, kH);
  k_ws_dpool<<<g.Q, kH, 0, st>>>(w.sdz, w.wb, w.dpool);
  const int htiles = (int)((g.maxn + kHeadTile - 1) / kHeadTile);
  k_ws_head_bwd<<<dim3(htiles, g.Q), kH, 0, st>>>(w.toff, w.dz, w.pre_t, w.dpool, w.wb, w.dpre_t);
  k_ws_src_bwd<<<dim3(g.tiles_s, g.Q), kH, 0, st>>>(w.soff, w.pre_s, w.dpool, w.dpre_s);
  ibsn::note_launch(6);
  // w_o, b_o: A = dout (one column), X = relu(z)
  wgrad(WgArgs{g.Nt, w.dout, 1, 1, w.z, kH, kH, 1, 1, w.wpart}, kOffWo, 0, kOffBo, grad, st);
  // W_h[:, 0:128], b_h: A = dz, X = relu(pre_t)
  wgrad(WgArgs{g.Nt, w.dz, kH, kH, w.pre_t, kH, kH, 1, 1, w.wpart}, kOffWh, kLdWh, kOffBh, grad, st);
  // W_h[:, 128:384]: rows are problems, A = sdz, X = [p_s; p_t]
  wgrad(WgArgs{(int64_t)g.Q, w.sdz, kH, kH, w.pool, 2 * kH, 2 * kH, 0, 0, w.wpart}, kOffWh + kH, kLdWh, 0, grad, st);
  // W_t, b_t and W_s, b_s: A = dpre, X = features
  wgrad(WgArgs{g.Nt, w.dpre_t, kH, kH, w.feat_t, 4, 3, 0, 1, w.wpart}, kOffWt, 3, kOffBt, grad, st);
  wgrad(WgArgs{g.Ms, w.dpre_s, kH, kH, w.feat_s, 4, 3, 0, 1, w.wpart}, kOffWs, 3, kOffBs, grad, st);
  return launched();
}

bool batch_ptrs_ok(const ibsn_ws_batch* B) { return B->x && B->y && B->a && B->b; }

}  // namespace

extern "C" int64_t ibsn_ws_param_count(void) { return kParams; }

extern "C" void ibsn_ws_adam_default(ibsn_ws_adam* hp) {
  if (!hp) return;
  hp->lr = 1e-3;
  hp->beta1 = 0.9;
  hp->beta2 = 0.999;
  hp->eps = 1e-8;
}

extern "C" int ibsn_ws_workspace_size(const ibsn_ws_batch* batch, size_t* bytes) {
  if (!bytes) return IBSN_ERR_INVALID_ARG;
  WsGeom g;
  const int r = ws_geom(batch, &g);
  if (r != IBSN_OK) return r;
  WsBufs b;
  *bytes = ws_carve(g, nullptr, &b);
  return IBSN_OK;
}

extern "C" int ibsn_ws_predict(const ibsn_ws_batch* batch, const float* params, double* gamma_hat, void* workspace,
                               size_t workspace_bytes, void* stream) {
  WsGeom g;
  int r = ws_geom(batch, &g);
  if (r != IBSN_OK) return r;
  if (!params || !gamma_hat || !batch_ptrs_ok(batch)) return IBSN_ERR_INVALID_ARG;
  WsBufs w;
  r = check_ws(g, workspace, workspace_bytes, &w);
  if (r != IBSN_OK) return r;
  return run_forward(batch, g, w, params, nullptr, gamma_hat, (cudaStream_t)stream);
}

extern "C" int ibsn_ws_loss_grad(const ibsn_ws_batch* batch, const float* params, const double* gamma_star,
                                 double* loss, float* grad, double* gamma_hat, void* workspace,
                                 size_t workspace_bytes, void* stream) {
  WsGeom g;
  int r = ws_geom(batch, &g);
  if (r != IBSN_OK) return r;
  if (!params || !gamma_star || !grad || !batch_ptrs_ok(batch)) return IBSN_ERR_INVALID_ARG;
  WsBufs w;
  r = check_ws(g, workspace, workspace_bytes, &w);
  if (r != IBSN_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  r = run_forward(batch, g, w, params, gamma_star, gamma_hat, st);
  if (r != IBSN_OK) return r;
  r = run_backward(g, w, grad, st);
  if (r != IBSN_OK) return r;
  if (loss) {
    std::vector<double> lq(g.Q);
    if (cudaMemcpyAsync(lq.data(), w.lossq, sizeof(double) * g.Q, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return IBSN_ERR_CUDA;
    double s = 0.0;
    for (double v : lq) s += v;
    *loss = s / (double)g.Q;
  }
  return IBSN_OK;
}

extern "C" int ibsn_ws_adam_step(int64_t count, float* params, float* m1, float* m2, const float* grad, int64_t t,
                                 const ibsn_ws_adam* hp, void* stream) {
  if (count < 1 || !params || !m1 || !m2 || !grad || t < 1 || !hp) return IBSN_ERR_INVALID_ARG;
  if (!(hp->lr > 0.0) || !(hp->beta1 >= 0.0 && hp->beta1 < 1.0) || !(hp->beta2 >= 0.0 && hp->beta2 < 1.0) ||
      !(hp->eps > 0.0))
    return IBSN_ERR_INVALID_ARG;
  const double bc1 = 1.0 - std::pow(hp->beta1, (double)t);
  const double bc2 = 1.0 - std::pow(hp->beta2, (double)t);
  const int64_t blocks = (count + 255) / 256 < 4096 ? (count + 255) / 256 : 4096;
  k_ws_adam<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
      count, params, m1, m2, grad, (float)hp->lr, (float)hp->beta1, (float)hp->beta2, (float)(1.0 - hp->beta1),
      (float)(1.0 - hp->beta2), (float)hp->eps, (float)bc1, (float)bc2);
  ibsn::note_launch();
  return launched();
}

namespace ibsn {

cudaError_t launch_semidual0(const CostRef& cost, int m, int64_t n, double eta, const double* a, const double* b,
                             const double* logb, const double* gamma, double* rowval, double* out, cudaStream_t st) {
  const int blocks = m < 4096 ? m : 4096;
  k_semidual0_rows<<<blocks, kSdThreads, 0, st>>>(cost, m, n, 1.0 / eta, a, logb, gamma, rowval);
  k_semidual0_finish<<<1, kSdThreads, 0, st>>>(m, n, eta, rowval, b, gamma, out);
  note_launch(2);
  return cudaGetLastError();
}

}  // namespace ibsn
