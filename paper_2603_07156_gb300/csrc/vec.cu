// O(m + n) vector kernels of the IBSN control flow: column-partial reduction,
// Sinkhorn potential update, centring, Armijo preparation and acceptance,
// rounding preparation (Alg. 3) and input validation.  Reductions are done
// in a fixed order, so results do not depend on scheduling.
#include "common.cuh"
#include "internal.h"

namespace ibsn {

namespace {

constexpr int kVB = 1024;  // threads of the single-block kernels

// write a per-column value to its float and float64 copies (either may be null)
__device__ __forceinline__ void put2(float* f, double* d, int64_t j, double x) {
  if (f) f[j] = (float)x;
  if (d) d[j] = x;
}

// block-wide sum / max over kVB threads, result on every thread
__device__ __forceinline__ double bsum(double v, double* sh) {
  double t[1] = {v};
  block_sum<kVB, 1>(t, sh);
  return t[0];
}
__device__ __forceinline__ double bmax(double v, double* sh) { return block_max<kVB>(v, sh); }

// ---------------------------------------------------------------------------
__global__ void k_finish_cols(const double* __restrict__ colpart, int nb, int64_t ldk, int64_t n,
                              const double* __restrict__ b, double* c_out, double* g_out,
                              const double* __restrict__ rowpart, int nrp, double* scal, unsigned int* counter,
                              double* blockbuf) {
  __shared__ double sh[8];
  __shared__ bool last;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double g2 = 0.0;
  if (j < n) {
    double c = 0.0;
    for (int q = 0; q < nb; ++q) c += colpart[(int64_t)q * ldk + j];
    if (c_out) c_out[j] = c;
    if (b) {
      const double g = c - b[j];
      if (g_out) g_out[j] = g;
      g2 = g * g;
    }
  }
  double t[1] = {g2};
  block_sum<256, 1>(t, sh);
  if (threadIdx.x == 0) {
    blockbuf[blockIdx.x] = t[0];
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (unsigned q = 0; q < gridDim.x; ++q) s += ((volatile double*)blockbuf)[q];
      scal[S_GN2] = s;
      *counter = 0u;
    }
    if (threadIdx.x < nrp) {
      double s = 0.0;
      for (int q = 0; q < nb; ++q) s += rowpart[q * kRowParts + threadIdx.x];
      scal[S_ROW0 + threadIdx.x] = s;
    }
  }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kVB) k_set_anchor(int64_t n, int64_t ldk, double eta, const double* Gam, double* gam,
                                                   double* ganc, const double* logb, double* wv, float* wvh,
                                                   float* wvl, double* dd, float* d32, double* d64) {
  for (int64_t j = threadIdx.x; j < ldk; j += kVB) {
    if (j < n) {
      const double G = (Gam ? Gam[j] : 0.0);
      ganc[j] = gam[j];
      const double w = logb[j] + (G + gam[j]) / eta;
      wv[j] = w;
      const float h = (float)w;
      wvh[j] = h;
      wvl[j] = (float)(w - (double)h);
      dd[j] = 0.0;
    }
    put2(d32, d64, j, 0.0);
  }
}

__global__ void __launch_bounds__(kVB) k_sinkhorn_update(int64_t n, double eta, const double* b, const double* c,
                                                        double* gam, const double* ganc, double* dd, float* d32,
                                                        double* d64, bool fp64, double* scal) {
  __shared__ double sh[64];
  double mx = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += kVB) {
    // a column whose plan entries all underflowed has c_j = 0; the floor keeps
    // the step finite (it only bounds the first steps of such columns)
    const double gj = gam[j] + eta * (log(b[j]) - log(fmax(c[j], fp64 ? 1e-300 : 1e-45)));
    gam[j] = gj;
    const double d = (gj - ganc[j]) / eta;
    dd[j] = d;
    put2(d32, d64, j, d);
    mx = fmax(mx, fabs(d));
  }
  mx = bmax(mx, sh);
  if (threadIdx.x == 0) scal[S_DMAX] = mx;
}

__global__ void __launch_bounds__(kVB) k_center(int64_t n, double eta, double* gam, const double* ganc, double* dd,
                                               float* d32, double* d64, double* scal) {
  __shared__ double sh[64];
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += kVB) s += gam[j];
  const double mean = bsum(s, sh) / (double)n;
  double mx = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += kVB) {
    const double gj = gam[j] - mean;
    gam[j] = gj;
    const double d = (gj - ganc[j]) / eta;
    dd[j] = d;
    put2(d32, d64, j, d);
    mx = fmax(mx, fabs(d));
  }
  mx = bmax(mx, sh);
  if (threadIdx.x == 0) {
    scal[S_DMAX] = mx;
    scal[S_MEAN] = mean;
  }
}

__global__ void __launch_bounds__(kVB) k_dir_post(int64_t n, double eta, double* delta, const double* g, double* scal) {
  __shared__ double sh[64];
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += kVB) s += delta[j];
  const double mean = bsum(s, sh) / (double)n;
  double sl = 0.0, mx = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += kVB) {
    const double dj = delta[j] - mean;
    delta[j] = dj;
    sl += g[j] * dj;
    mx = fmax(mx, fabs(dj));
  }
  sl = bsum(sl, sh);
  mx = bmax(mx, sh);
  if (threadIdx.x == 0) {
    scal[S_SLOPE] = sl;
    scal[S_DELTAMAX] = mx / eta;
  }
}

// phi(x) = expm1(x) - x, second order; Taylor series for small |x|
__device__ __forceinline__ double phi_expm1_minus(double x) {
  if (fabs(x) < 1e-3) return x * x * (0.5 + x * (1.0 / 6.0 + x * (1.0 / 24.0 + x * (1.0 / 120.0 + x / 720.0))));
  return expm1(x) - x;
}

__global__ void __launch_bounds__(kVB) k_armijo_prep(int64_t n, int64_t ldk, double eta, double t, const double* delta,
                                                    const double* c, float* em32, double* em64, double* scal) {
  __shared__ double sh[64];
  double ps = 0.0;
  for (int64_t j = threadIdx.x; j < ldk; j += kVB) {
    if (j < n) {
      const double x = t * delta[j] / eta;
      put2(em32, em64, j, expm1(x));
      ps += c[j] * phi_expm1_minus(x);
    } else {
      put2(em32, em64, j, 0.0);
    }
  }
  ps = bsum(ps, sh);
  if (threadIdx.x == 0) scal[S_PHI] = ps;
}

__global__ void __launch_bounds__(kVB) k_armijo_accept(int64_t n, double eta, double t, const double* delta,
                                                      double* gam, const double* ganc, double* dd, float* d32,
                                                      double* d64, const double* cnew, const double* b, double* g,
                                                      double* scal) {
  __shared__ double sh[64];
  double mx = 0.0, g2 = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += kVB) {
    const double gj = gam[j] + t * delta[j];
    gam[j] = gj;
    const double d = (gj - ganc[j]) / eta;
    dd[j] = d;
    put2(d32, d64, j, d);
    mx = fmax(mx, fabs(d));
    const double gr = cnew[j] - b[j];
    g[j] = gr;
    g2 += gr * gr;
  }
  mx = bmax(mx, sh);
  g2 = bsum(g2, sh);
  if (threadIdx.x == 0) {
    scal[S_DMAX] = mx;
    scal[S_GN2] = g2;
  }
}

// Alg. 3 with z = 1: y_j = min(b_j/c_j, 1), omega_j = 1 - y_j = max(0, g_j/c_j),
// e_c,j = b_j - y_j c_j = max(0, -g_j), S = ||e_c||_1.
__global__ void __launch_bounds__(kVB) k_round_prep(int64_t n, const double* b, const double* c, const double* g,
                                                   RoundVecs R, double* scal) {
  __shared__ double sh[64];
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += kVB) s += fmax(0.0, -g[j]);
  s = bsum(s, sh);
  const double invS = s > 0.0 ? 1.0 / s : 0.0;
  for (int64_t j = threadIdx.x; j < n; j += kVB) {
    const double cj = c[j];
    const double y = fmin(b[j] / cj, 1.0);
    const double om = fmax(0.0, g[j] / cj);
    const double ec = fmax(0.0, -g[j]);
    put2(R.y32, R.y64, j, y);
    put2(R.om32, R.om64, j, om);
    put2(R.ec32, R.ec64, j, ec);
    put2(R.ecs32, R.ecs64, j, ec * invS);
    R.ecsl32[j] = (float)(ec * invS - (double)(float)(ec * invS));
    put2(R.lec32, R.lec64, j, log(ec));
  }
  if (threadIdx.x == 0) scal[S_ECSUM] = s;
}

// column marginal violation of Xhat and b^T gamma
__global__ void __launch_bounds__(kVB) k_certify_cols(int64_t n, const double* b, const double* colF, const double* c,
                                                     const double* gam, double ersum, double* scal) {
  __shared__ double sh[64];
  double es = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += kVB) es += fmax(0.0, b[j] - c[j]);
  es = bsum(es, sh);
  const double f = es > 0.0 ? ersum / es : 0.0;
  double viol = 0.0, bg = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += kVB) {
    const double ec = fmax(0.0, b[j] - c[j]);
    viol += fabs(colF[j] + ec * f - b[j]);
    bg += b[j] * gam[j];
  }
  viol = bsum(viol, sh);
  bg = bsum(bg, sh);
  if (threadIdx.x == 0) {
    scal[S_COLVIOL] = viol;
    scal[S_BGAM] = bg;
  }
}

__global__ void __launch_bounds__(kVB) k_validate_marginals(int64_t m, int64_t n, const double* a, const double* b,
                                                           double* scal) {
  __shared__ double sh[64];
  double amin = kInf, asum = 0.0, bad = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += kVB) {
    const double v = a[i];
    if (!isfinite(v)) bad += 1.0; else { amin = fmin(amin, v); asum += v; }
  }
  double bmin = kInf, bsm = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += kVB) {
    const double v = b[j];
    if (!isfinite(v)) bad += 1.0; else { bmin = fmin(bmin, v); bsm += v; }
  }
  amin = -bmax(-amin, sh);
  bmin = -bmax(-bmin, sh);
  asum = bsum(asum, sh);
  bsm = bsum(bsm, sh);
  bad = bsum(bad, sh);
  if (threadIdx.x == 0) {
    scal[S_AMIN] = amin; scal[S_ASUM] = asum; scal[S_BMIN] = bmin; scal[S_BSUM] = bsm; scal[S_ABAD] = bad;
  }
}

__global__ void k_validate_cost(int64_t m, int64_t n, const void* C, int64_t ldc, int kind, double* scal) {
  unsigned int bad = 0;
  double cmax = 0.0;
  const int64_t total = m * n;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / n, j = q - i * n;
    const double v = kind == 0 ? static_cast<const double*>(C)[i * ldc + j]
                               : (double)static_cast<const float*>(C)[i * ldc + j];
    if (!(v >= 0.0) || !isfinite(v)) ++bad;
    else cmax = fmax(cmax, v);
  }
  bad = (unsigned)warp_sum((int)bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(&scal[S_CBAD], (double)bad);
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(&scal[S_CMAX]), (unsigned long long)__double_as_longlong(cmax));
}

// float copy of gamma and max_j |gamma_j| for the certificate's float32 c-transform scan
__global__ void __launch_bounds__(kVB) k_certify_prep(int64_t n, const double* gam, float* gam32, double* scal) {
  __shared__ double sh[kVB / 32];
  double mx = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += kVB) {
    gam32[j] = (float)gam[j];
    mx = fmax(mx, fabs(gam[j]));
  }
  mx = bmax(mx, sh);
  if (threadIdx.x == 0) scal[S_GMAX] = mx;
}

__global__ void k_set_slot(double* scal, int slot, double v) { scal[slot] = v; }

__global__ void k_fill_pad(void* v, int64_t n, int64_t ldk, bool fp64, double value) {
  const int64_t j = n + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < ldk) {
    if (fp64) static_cast<double*>(v)[j] = value; else static_cast<float*>(v)[j] = (float)value;
  }
}

__global__ void k_neg(int64_t n, const double* x, double* y) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) y[j] = -x[j];
}

}  // namespace

cudaError_t launch_finish_cols(const double* colpart, int nb, int64_t ldk, int64_t n, const double* b,
                               double* c_out, double* g_out, const double* rowpart, int nrp, double* scal,
                               unsigned int* counter, double* blockbuf, cudaStream_t st) {
  const int nbk = (int)((n + 255) / 256);
  k_finish_cols<<<nbk, 256, 0, st>>>(colpart, nb, ldk, n, b, c_out, g_out, rowpart, nrp, scal, counter, blockbuf);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_set_anchor(int64_t n, int64_t ldk, double eta, const double* Gam, double* gam, double* ganc,
                              const double* logb, double* wv, float* wvh, float* wvl, double* dd, float* d32,
                              double* d64, cudaStream_t st) {
  k_set_anchor<<<1, kVB, 0, st>>>(n, ldk, eta, Gam, gam, ganc, logb, wv, wvh, wvl, dd, d32, d64);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_sinkhorn_update(int64_t n, double eta, const double* b, const double* c, double* gam,
                                   const double* ganc, double* dd, float* d32, double* d64, bool fp64,
                                   double* scal, cudaStream_t st) {
  k_sinkhorn_update<<<1, kVB, 0, st>>>(n, eta, b, c, gam, ganc, dd, d32, d64, fp64, scal);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_center(int64_t n, double eta, double* gam, const double* ganc, double* dd, float* d32,
                          double* d64, double* scal, cudaStream_t st) {
  k_center<<<1, kVB, 0, st>>>(n, eta, gam, ganc, dd, d32, d64, scal);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_dir_post(int64_t n, double eta, double* delta, const double* g, double* scal, cudaStream_t st) {
  k_dir_post<<<1, kVB, 0, st>>>(n, eta, delta, g, scal);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_armijo_prep(int64_t n, int64_t ldk, double eta, double t, const double* delta, const double* c,
                               float* em32, double* em64, double* scal, cudaStream_t st) {
  k_armijo_prep<<<1, kVB, 0, st>>>(n, ldk, eta, t, delta, c, em32, em64, scal);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_armijo_accept(int64_t n, double eta, double t, const double* delta, double* gam,
                                 const double* ganc, double* dd, float* d32, double* d64, const double* cnew,
                                 const double* b, double* g, double* scal, cudaStream_t st) {
  k_armijo_accept<<<1, kVB, 0, st>>>(n, eta, t, delta, gam, ganc, dd, d32, d64, cnew, b, g, scal);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_round_prep(int64_t n, const double* b, const double* c, const double* g, const RoundVecs& R,
                              double* scal, cudaStream_t st) {
  k_round_prep<<<1, kVB, 0, st>>>(n, b, c, g, R, scal);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_certify_cols(int64_t n, const double* b, const double* colF, const double*, const double* c,
                                const double* gam, double ersum, double* scal, cudaStream_t st) {
  k_certify_cols<<<1, kVB, 0, st>>>(n, b, colF, c, gam, ersum, scal);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_validate_marginals(int64_t m, int64_t n, const double* a, const double* b, double* scal,
                                      cudaStream_t st) {
  k_validate_marginals<<<1, kVB, 0, st>>>(m, n, a, b, scal);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_validate_cost(int64_t m, int64_t n, const void* C, int64_t ldc, int kind, double* scal,
                                 cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(&scal[S_CBAD], 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(&scal[S_CMAX], 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  if (kind != 0 && kind != 1) return cudaSuccess;
  k_validate_cost<<<1216, 256, 0, st>>>(m, n, C, ldc, kind, scal);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_certify_prep(int64_t n, const double* gam, float* gam32, double* scal, cudaStream_t st) {
  k_certify_prep<<<1, kVB, 0, st>>>(n, gam, gam32, scal);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_set_slot(double* scal, int slot, double v, cudaStream_t st) {
  k_set_slot<<<1, 1, 0, st>>>(scal, slot, v);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_fill_pad(void* v, int64_t n, int64_t ldk, bool fp64, double value, cudaStream_t st) {
  if (ldk <= n) return cudaSuccess;
  k_fill_pad<<<1, 64, 0, st>>>(v, n, ldk, fp64, value);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_neg(int64_t n, const double* x, double* y, cudaStream_t st) {
  k_neg<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, y);
  note_launch();
  return cudaGetLastError();
}

}  // namespace ibsn
