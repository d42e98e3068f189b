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
// ... and to the float-float lo part x - fl32(x) (may be null)
__device__ __forceinline__ void put3(float* f, float* lo, double* d, int64_t j, double x) {
  const float h = (float)x;
  if (f) f[j] = h;
  if (lo) lo[j] = (float)(x - (double)h);
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
// Grid-wide reductions of the O(n) kernels.  Every block reduces its K values
// (sum, or max for the values flagged in kMax), writes them to blockbuf and
// counts itself in; the last block to arrive combines the block results in
// block order, so the totals do not depend on scheduling.  The O(n) kernels
// run on many blocks: float64 arithmetic on one SM alone is slow.
// ---------------------------------------------------------------------------
constexpr int kRB = 256;  // threads per block of the O(n) kernels

template <int K>
__device__ __forceinline__ bool reduce_last(double (&v)[K], unsigned kMax, const RedBuf& rb) {
  __shared__ double sh[K][kRB / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double x = v[q];
    const bool mx = (kMax >> q) & 1u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_xor_sync(0xffffffffu, x, o);
      x = mx ? fmax(x, y) : x + y;
    }
    if (lane == 0) sh[q][w] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      double x = sh[q][0];
      const bool mx = (kMax >> q) & 1u;
      for (int u = 1; u < kRB / 32; ++u) x = mx ? fmax(x, sh[q][u]) : x + sh[q][u];
      rb.blockbuf[(size_t)q * gridDim.x + blockIdx.x] = x;
    }
    __threadfence();
    last = atomicAdd(rb.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  if (threadIdx.x != 0) return false;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const bool mx = (kMax >> q) & 1u;
    double x = ((volatile double*)rb.blockbuf)[(size_t)q * gridDim.x];
    for (unsigned b = 1; b < gridDim.x; ++b) {
      const double y = ((volatile double*)rb.blockbuf)[(size_t)q * gridDim.x + b];
      x = mx ? fmax(x, y) : x + y;
    }
    v[q] = x;
  }
  *rb.counter = 0u;  // ready for the next kernel on the stream
  return true;
}

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * kRB + threadIdx.x; }

// Column sums of the per-block partials of a dense pass: c = sum_q colpart[q],
// g = c - b, ||g||^2 and ||max(0, -g)||_1 (the rounding's S), and the totals of
// the first nrp row partials.  A block handles 32 columns x 8 slices of the
// partials; the slices are added in slice order.
__global__ void __launch_bounds__(kRB) k_finish_cols(const double* __restrict__ colpart, bool ffpart, int nb,
                                                     int64_t ldk, int64_t n, const double* __restrict__ b,
                                                     double* c_out, double* g_out, const double* __restrict__ rowpart,
                                                     int nrp, double* scal, RedBuf rb) {
  __shared__ double part[8][33];
  const int lane = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * 32 + lane;
  double c = 0.0;
  if (j < n) {
    if (ffpart) {  // float-float partials of the float passes: added in float-float
      const float2* p2 = reinterpret_cast<const float2*>(colpart);
      FF s{0.f, 0.f};
      for (int q = sl; q < nb; q += 8) {
        const float2 v = p2[(int64_t)q * ldk + j];
        s = ff_add(s, FF{v.x, v.y});
      }
      c = (double)s.hi + (double)s.lo;
    } else {
      for (int q = sl; q < nb; q += 8) c += colpart[(int64_t)q * ldk + j];
    }
  }
  part[sl][lane] = c;
  __syncthreads();
  double v[2] = {0.0, 0.0};
  if (sl == 0 && j < n) {
    double t = part[0][lane];
#pragma unroll
    for (int u = 1; u < 8; ++u) t += part[u][lane];
    if (c_out) c_out[j] = t;
    if (b) {
      const double g = t - b[j];
      if (g_out) g_out[j] = g;
      v[0] = g * g;
      v[1] = fmax(0.0, -g);
    }
  }
  if (reduce_last<2>(v, 0u, rb)) {
    if (b) {  // the gradient's totals stay valid until the next gradient
      scal[S_GN2] = v[0];
      scal[S_ECSUM] = v[1];
    }
    for (int q = 0; q < nrp; ++q) {
      double s = 0.0;
      for (int u = 0; u < nb; ++u) s += rowpart[u * kRowParts + q];
      scal[S_ROW0 + q] = s;
    }
  }
}

// Row scalars of the float-float plan and Armijo passes (which store S_i, M_i
// per row instead of forming float64 logs on their serial per-row path).
// plan:   lse_i = M_i + log S0_i -> rowout; sum_i a_i lse_i -> scal[S_ROW0]
// Armijo: s_i = S1_i / S0_i; rowout = M_i + log S0_i + log1p(s_i);
//         sum_i a_i psi(s_i) -> scal[S_ROW0], sum_i a_i log1p(s_i) -> scal[S_ROW0 + 1]
__global__ void __launch_bounds__(kRB) k_rows_ff(int64_t m, bool armijo, const double* a, const double* S0,
                                                const double* S1, const double* M, double* rowout, double* scal,
                                                RedBuf rb) {
  const int64_t i = gtid();
  double v[2] = {0.0, 0.0};
  if (i < m) {
    // the passes store S0, S1 as float-float pairs and M as a float
    const float2 s0 = reinterpret_cast<const float2*>(S0)[i];
    const double S0i = (double)s0.x + (double)s0.y;
    const double Mi = (double)reinterpret_cast<const float*>(M)[i];
    const double ls = log(S0i);
    if (armijo) {
      const float2 s1 = reinterpret_cast<const float2*>(S1)[i];
      const double si = ((double)s1.x + (double)s1.y) / S0i;
      const double l1p = log1p(si);
      v[0] = a[i] * psi_log1p_minus(si);
      v[1] = a[i] * l1p;
      if (rowout) rowout[i] = Mi + ls + l1p;
    } else {
      const double lse = Mi + ls;
      v[0] = a[i] * lse;
      if (rowout) rowout[i] = lse;
    }
  }
  if (reduce_last<2>(v, 0u, rb)) {
    scal[S_ROW0] = v[0];
    if (armijo) scal[S_ROW0 + 1] = v[1];
  }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRB) k_set_anchor(int64_t n, int64_t ldk, double eta, const double* Gam,
                                                   double* gam, double* ganc, const double* logb, double* wv,
                                                   float* wvh, float* wvl, double* dd, float* d32, float* dlo,
                                                   double* d64) {
  const int64_t j = gtid();
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
  if (j < ldk) put3(d32, dlo, d64, j, 0.0);
}

__global__ void __launch_bounds__(kRB) k_sinkhorn_update(int64_t n, double eta, const double* b, const double* c,
                                                        double* gam, const double* ganc, double* dd, float* d32,
                                                        float* dlo, double* d64, bool fp64, double* scal, RedBuf rb) {
  const int64_t j = gtid();
  double v[1] = {0.0};
  if (j < n) {
    // a column whose plan entries all underflowed has c_j = 0; the floor keeps
    // the step finite (it only bounds the first steps of such columns)
    const double gj = gam[j] + eta * (log(b[j]) - log(fmax(c[j], fp64 ? 1e-300 : 1e-45)));
    gam[j] = gj;
    const double d = (gj - ganc[j]) / eta;
    dd[j] = d;
    put3(d32, dlo, d64, j, d);
    v[0] = fabs(d);
  }
  if (reduce_last<1>(v, 1u, rb)) scal[S_DMAX] = v[0];
}

// sum of x into scal[slot] (first phase of a centring)
__global__ void __launch_bounds__(kRB) k_sum_into(int64_t n, const double* x, double* scal, int slot, RedBuf rb) {
  const int64_t j = gtid();
  double v[1] = {j < n ? x[j] : 0.0};
  if (reduce_last<1>(v, 0u, rb)) scal[slot] = v[0];
}

__global__ void __launch_bounds__(kRB) k_center(int64_t n, double eta, double* gam, const double* ganc, double* dd,
                                               float* d32, float* dlo, double* d64, double* scal, RedBuf rb) {
  const double mean = scal[S_MEAN] / (double)n;
  const int64_t j = gtid();
  double v[1] = {0.0};
  if (j < n) {
    const double gj = gam[j] - mean;
    gam[j] = gj;
    const double d = (gj - ganc[j]) / eta;
    dd[j] = d;
    put3(d32, dlo, d64, j, d);
    v[0] = fabs(d);
  }
  if (reduce_last<1>(v, 1u, rb)) {
    scal[S_DMAX] = v[0];
    scal[S_MEAN] = mean;
  }
}

__global__ void __launch_bounds__(kRB) k_dir_post(int64_t n, double eta, double* delta, const double* g, double* scal,
                                                 RedBuf rb) {
  const double mean = scal[S_TMP] / (double)n;
  const int64_t j = gtid();
  double v[2] = {0.0, 0.0};
  if (j < n) {
    const double dj = delta[j] - mean;
    delta[j] = dj;
    v[0] = g[j] * dj;
    v[1] = fabs(dj);
  }
  if (reduce_last<2>(v, 2u, rb)) {
    scal[S_SLOPE] = v[0];
    scal[S_DELTAMAX] = v[1] / eta;
  }
}

// phi(x) = expm1(x) - x, second order; Taylor series for small |x|
__device__ __forceinline__ double phi_expm1_minus(double x) {
  if (fabs(x) < 1e-3) return x * x * (0.5 + x * (1.0 / 6.0 + x * (1.0 / 24.0 + x * (1.0 / 120.0 + x / 720.0))));
  return expm1(x) - x;
}

__global__ void __launch_bounds__(kRB) k_armijo_prep(int64_t n, int64_t ldk, double eta, double t, const double* delta,
                                                    const double* c, float* em32, float* emlo, double* em64,
                                                    double* scal, RedBuf rb) {
  const int64_t j = gtid();
  double v[1] = {0.0};
  if (j < n) {
    const double x = t * delta[j] / eta;
    put3(em32, emlo, em64, j, expm1(x));
    v[0] = c[j] * phi_expm1_minus(x);
  } else if (j < ldk) {
    put3(em32, emlo, em64, j, 0.0);
  }
  if (reduce_last<1>(v, 0u, rb)) scal[S_PHI] = v[0];
}

__global__ void __launch_bounds__(kRB) k_armijo_accept(int64_t n, double eta, double t, const double* delta,
                                                      double* gam, const double* ganc, double* dd, float* d32,
                                                      float* dlo, double* d64, const double* cnew, const double* b,
                                                      double* g, double* scal, RedBuf rb) {
  const int64_t j = gtid();
  double v[3] = {0.0, 0.0, 0.0};
  if (j < n) {
    const double gj = gam[j] + t * delta[j];
    gam[j] = gj;
    const double d = (gj - ganc[j]) / eta;
    dd[j] = d;
    put3(d32, dlo, d64, j, d);
    const double gr = cnew[j] - b[j];
    g[j] = gr;
    v[0] = fabs(d);
    v[1] = gr * gr;
    v[2] = fmax(0.0, -gr);
  }
  if (reduce_last<3>(v, 1u, rb)) {
    scal[S_DMAX] = v[0];
    scal[S_GN2] = v[1];
    scal[S_ECSUM] = v[2];
  }
}

// Alg. 3 with z = 1: y_j = min(b_j/c_j, 1), omega_j = 1 - y_j = max(0, g_j/c_j),
// e_c,j = b_j - y_j c_j = max(0, -g_j); S = ||e_c||_1 was formed with g.  For
// the grid cost also the moments of w = e_c / S that give sum_j C_ij w_j in
// closed form per row (S_W0 .. S_W0 + 3).
__global__ void __launch_bounds__(kRB) k_round_prep(int64_t n, const double* b, const double* c, const double* g,
                                                   RoundVecs R, const int* rc, double* scal, RedBuf rb) {
  const int64_t j = gtid();
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const double s = scal[S_ECSUM];
  const double invS = s > 0.0 ? 1.0 / s : 0.0;
  if (j < n) {
    const double cj = c[j];
    const double y = fmin(b[j] / cj, 1.0);
    const double om = fmax(0.0, g[j] / cj);
    const double ec = fmax(0.0, -g[j]);
    const double w = ec * invS;
    put3(R.y32, R.ylo32, R.y64, j, y);
    put3(R.om32, R.omlo32, R.om64, j, om);
    put2(R.ec32, R.ec64, j, ec);
    put2(R.ecs32, R.ecs64, j, w);
    R.ecsl32[j] = (float)(w - (double)(float)w);
    put2(R.lec32, R.lec64, j, log(ec));
    put2(R.hom32, R.hom64, j, om > 0.0 ? (1.0 - om) * log1p(-om) + om : 0.0);
    if (rc) {
      const double r = (double)(rc[j] & 0xffff), q = (double)(rc[j] >> 16);
      v[0] = w;
      v[1] = r * w;
      v[2] = q * w;
      v[3] = (r * r + q * q) * w;
    }
  }
  if (rc == nullptr) return;
  if (reduce_last<4>(v, 0u, rb))
    for (int q = 0; q < 4; ++q) scal[S_W0 + q] = v[q];
}

// bin coordinates of the grid cost, packed row | col << 16
__global__ void k_grid_rc(int64_t n, int gw, int* rc) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) {
    const int r = (int)(j / gw), q = (int)(j - (int64_t)r * gw);
    rc[j] = r | (q << 16);
  }
}

// Row scalars of the float-float certificate pass from its per-row results
// rowbuf = [sum_j P_ij omega_j | sum_j P_ij | sum_j C_ij a_i P_ij y_j |
//           a_i sum_j P_ij (C_ij - zeta_i - gamma_j) | zeta_i | sum_j C_ij e_c,j / S]
// (the last is formed here for the grid cost from the moments S_W0..).
// e_r,i = a_i Q0, row residual a_i (Q1 - 1); totals into S_ROW0 + 0..6 as the
// single-pass certificate writes them (slot 5: sum C^2, formed once per context).
__global__ void __launch_bounds__(kRB) k_rows_cert(int64_t m, const double* a, const double* rb_, const int* rc,
                                                  double scale, double* zeta_out, double* er_out, double* scal,
                                                  RedBuf rb) {
  const int64_t i = gtid();
  double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (i < m) {
    const double ai = a[i];
    const float2* f2 = reinterpret_cast<const float2*>(rb_);  // float-float planes 0..3 and 5
    auto plane = [&](int q) { const float2 v = f2[q * m + i]; return (double)v.x + (double)v.y; };
    const double q0 = plane(0), q1 = plane(1), q2 = plane(2), q3 = plane(3), zeta = rb_[4 * m + i];
    double cw;
    if (rc) {
      const double r = (double)(rc[i] & 0xffff), q = (double)(rc[i] >> 16);
      cw = scale * ((r * r + q * q) * scal[S_W0] - 2.0 * (r * scal[S_W0 + 1] + q * scal[S_W0 + 2]) + scal[S_W0 + 3]);
    } else {
      cw = plane(5);
    }
    const double er = ai * q0;
    const double rv = ai * (q1 - 1.0);
    v[0] = q2 + er * cw;
    v[1] = ai * zeta;
    v[2] = fabs(rv);
    v[3] = er;
    v[4] = q3;
    v[5] = rv * rv;
    if (zeta_out) zeta_out[i] = zeta;
    if (er_out) er_out[i] = er;
  }
  if (reduce_last<6>(v, 0u, rb)) {
    scal[S_ROW0 + 0] = v[0];
    scal[S_ROW0 + 1] = v[1];
    scal[S_ROW0 + 2] = v[2];
    scal[S_ROW0 + 3] = v[3];
    scal[S_ROW0 + 4] = v[4];
    scal[S_ROW0 + 5] = scal[S_C2SUM];
    scal[S_ROW0 + 6] = v[5];
  }
}

// column marginal violation of Xhat and b^T gamma; sum_j max(0, b_j - c_j) = S
__global__ void __launch_bounds__(kRB) k_certify_cols(int64_t n, const double* b, const double* colF, const double* c,
                                                     const double* gam, double ersum, double* scal, RedBuf rb) {
  const double es = scal[S_ECSUM];
  const double f = es > 0.0 ? ersum / es : 0.0;
  const int64_t j = gtid();
  double v[2] = {0.0, 0.0};
  if (j < n) {
    const double ec = fmax(0.0, b[j] - c[j]);
    v[0] = fabs(colF[j] + ec * f - b[j]);
    v[1] = b[j] * gam[j];
  }
  if (reduce_last<2>(v, 0u, rb)) {
    scal[S_COLVIOL] = v[0];
    scal[S_BGAM] = v[1];
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

__global__ void k_validate_cost(int64_t m, int64_t n, const void* C, int64_t ldc, int kind, const double* px,
                                const double* py, int dim, double scale, double* scal) {
  unsigned int bad = 0;
  double cmax = 0.0, c2 = 0.0;
  const int64_t total = m * n;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / n, j = q - i * n;
    double v;
    if (kind == 3) {  // points: C_ij = scale ||x_i - y_j||^2 (non-finite coordinates give NaN)
      double s = 0.0;
      for (int k = 0; k < dim; ++k) {
        const double t = px[i * dim + k] - py[j * dim + k];
        s = fma(t, t, s);
      }
      v = scale * s;
    } else {
      v = kind == 0 ? static_cast<const double*>(C)[i * ldc + j] : (double)static_cast<const float*>(C)[i * ldc + j];
    }
    if (!(v >= 0.0) || !isfinite(v)) ++bad;
    else { cmax = fmax(cmax, v); c2 += v * v; }
  }
  bad = (unsigned)warp_sum((int)bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(&scal[S_CBAD], (double)bad);
  // sum C^2 (normalises Delta_kkt only: the summation order is not fixed)
  c2 = warp_sum(c2);
  if ((threadIdx.x & 31) == 0 && c2 > 0.0) atomicAdd(&scal[S_C2SUM], c2);
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(&scal[S_CMAX]), (unsigned long long)__double_as_longlong(cmax));
}

// float copy of gamma and max_j |gamma_j| for the certificate's float32 c-transform scan
__global__ void __launch_bounds__(kRB) k_certify_prep(int64_t n, const double* gam, float* gam32, float* gamlo,
                                                     double* scal, RedBuf rb) {
  const int64_t j = gtid();
  double v[1] = {0.0};
  if (j < n) {
    put3(gam32, gamlo, nullptr, j, gam[j]);
    v[0] = fabs(gam[j]);
  }
  if (reduce_last<1>(v, 1u, rb)) scal[S_GMAX] = v[0];
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

static unsigned nblk(int64_t n) { return (unsigned)((n + kRB - 1) / kRB); }

cudaError_t launch_rows_ff(int64_t m, bool armijo, const double* a, const double* S0, const double* S1,
                           const double* M, double* rowout, double* scal, const RedBuf& rb, cudaStream_t st) {
  k_rows_ff<<<nblk(m), kRB, 0, st>>>(m, armijo, a, S0, S1, M, rowout, scal, rb);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_finish_cols(const double* colpart, bool ffpart, int nb, int64_t ldk, int64_t n, const double* b,
                               double* c_out, double* g_out, const double* rowpart, int nrp, double* scal,
                               const RedBuf& rb, cudaStream_t st) {
  k_finish_cols<<<(unsigned)((n + 31) / 32), kRB, 0, st>>>(colpart, ffpart, nb, ldk, n, b, c_out, g_out, rowpart, nrp,
                                                          scal, rb);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_set_anchor(int64_t n, int64_t ldk, double eta, const double* Gam, double* gam, double* ganc,
                              const double* logb, double* wv, float* wvh, float* wvl, double* dd, float* d32,
                              float* dlo, double* d64, cudaStream_t st) {
  k_set_anchor<<<nblk(ldk), kRB, 0, st>>>(n, ldk, eta, Gam, gam, ganc, logb, wv, wvh, wvl, dd, d32, dlo, d64);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_sinkhorn_update(int64_t n, double eta, const double* b, const double* c, double* gam,
                                   const double* ganc, double* dd, float* d32, float* dlo, double* d64, bool fp64,
                                   double* scal, const RedBuf& rb, cudaStream_t st) {
  k_sinkhorn_update<<<nblk(n), kRB, 0, st>>>(n, eta, b, c, gam, ganc, dd, d32, dlo, d64, fp64, scal, rb);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_center(int64_t n, double eta, double* gam, const double* ganc, double* dd, float* d32,
                          float* dlo, double* d64, double* scal, const RedBuf& rb, cudaStream_t st) {
  k_sum_into<<<nblk(n), kRB, 0, st>>>(n, gam, scal, S_MEAN, rb);
  k_center<<<nblk(n), kRB, 0, st>>>(n, eta, gam, ganc, dd, d32, dlo, d64, scal, rb);
  note_launch(2);
  return cudaGetLastError();
}
cudaError_t launch_dir_post(int64_t n, double eta, double* delta, const double* g, double* scal, const RedBuf& rb,
                            cudaStream_t st) {
  k_sum_into<<<nblk(n), kRB, 0, st>>>(n, delta, scal, S_TMP, rb);
  k_dir_post<<<nblk(n), kRB, 0, st>>>(n, eta, delta, g, scal, rb);
  note_launch(2);
  return cudaGetLastError();
}
cudaError_t launch_armijo_prep(int64_t n, int64_t ldk, double eta, double t, const double* delta, const double* c,
                               float* em32, float* emlo, double* em64, double* scal, const RedBuf& rb,
                               cudaStream_t st) {
  k_armijo_prep<<<nblk(ldk), kRB, 0, st>>>(n, ldk, eta, t, delta, c, em32, emlo, em64, scal, rb);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_armijo_accept(int64_t n, double eta, double t, const double* delta, double* gam,
                                 const double* ganc, double* dd, float* d32, float* dlo, double* d64,
                                 const double* cnew, const double* b, double* g, double* scal, const RedBuf& rb,
                                 cudaStream_t st) {
  k_armijo_accept<<<nblk(n), kRB, 0, st>>>(n, eta, t, delta, gam, ganc, dd, d32, dlo, d64, cnew, b, g, scal, rb);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_round_prep(int64_t n, const double* b, const double* c, const double* g, const RoundVecs& R,
                              const int* grid_rc, double* scal, const RedBuf& rb, cudaStream_t st) {
  k_round_prep<<<nblk(n), kRB, 0, st>>>(n, b, c, g, R, grid_rc, scal, rb);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_grid_rc(int64_t n, int gw, int* rc, cudaStream_t st) {
  k_grid_rc<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, gw, rc);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_rows_cert(int64_t m, const double* a, const double* rowbuf, const int* grid_rc, double scale,
                             double* zeta_out, double* er_out, double* scal, const RedBuf& rb, cudaStream_t st) {
  k_rows_cert<<<nblk(m), kRB, 0, st>>>(m, a, rowbuf, grid_rc, scale, zeta_out, er_out, scal, rb);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_certify_cols(int64_t n, const double* b, const double* colF, const double* c, const double* gam,
                                double ersum, double* scal, const RedBuf& rb, cudaStream_t st) {
  k_certify_cols<<<nblk(n), kRB, 0, st>>>(n, b, colF, c, gam, ersum, scal, rb);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_validate_marginals(int64_t m, int64_t n, const double* a, const double* b, double* scal,
                                      cudaStream_t st) {
  k_validate_marginals<<<1, kVB, 0, st>>>(m, n, a, b, scal);
  note_launch();
  return cudaGetLastError();
}
// c-transform zeta_i = min_j C_ij - gamma_j of the grid cost (App. C.1) by
// separability: with C = s ((r_i - r_j)^2 + (c_i - c_j)^2),
//   zeta(r, c) = min_{r'} [ s (r - r')^2 + h(r', c) ],
//   h(r', c) = min_{c'} [ s (c - c')^2 - gamma(r', c') ],
// the same minimum as the scan over all n bins (it differs only in rounding
// order), at 2 w h (h + w) float64 operations instead of (h w)^2.
__global__ void k_ctransform_grid_cols(int h, int w, double s, const double* __restrict__ gam, double* __restrict__ hmin) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= h * w) return;
  const int r = q / w, c = q - r * w;
  const double* g = gam + (int64_t)r * w;
  double best = kInf;
  for (int c2 = 0; c2 < w; ++c2) {
    const double d = (double)(c - c2);
    best = fmin(best, s * (d * d) - g[c2]);
  }
  hmin[q] = best;
}
__global__ void k_ctransform_grid_rows(int h, int w, double s, const double* __restrict__ hmin, double* __restrict__ zeta) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= h * w) return;
  const int r = q / w, c = q - r * w;
  double best = kInf;
  for (int r2 = 0; r2 < h; ++r2) {
    const double d = (double)(r - r2);
    best = fmin(best, s * (d * d) + hmin[(int64_t)r2 * w + c]);
  }
  zeta[q] = best;
}
cudaError_t launch_ctransform_grid(int h, int w, double s, const double* gam, double* hmin, double* zeta,
                                   cudaStream_t st) {
  const unsigned nb = (unsigned)((h * w + 255) / 256);
  k_ctransform_grid_cols<<<nb, 256, 0, st>>>(h, w, s, gam, hmin);
  k_ctransform_grid_rows<<<nb, 256, 0, st>>>(h, w, s, hmin, zeta);
  note_launch(2);
  return cudaGetLastError();
}

// coordinates as float pairs (hi, lo) with hi + lo = x to 2^-48 relative
__global__ void k_split_coords(int64_t count, const double* __restrict__ x, float2* __restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < count) {
    const double v = x[q];
    const float h = (float)v;
    out[q] = make_float2(h, (float)(v - (double)h));
  }
}
cudaError_t launch_split_coords(int64_t count, const double* x, float2* out, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  k_split_coords<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(count, x, out);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_validate_cost(int64_t m, int64_t n, const void* C, int64_t ldc, int kind, const double* px,
                                 const double* py, int dim, double scale, double* scal,
                                 cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(&scal[S_CBAD], 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(&scal[S_CMAX], 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(&scal[S_C2SUM], 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  if (kind != 0 && kind != 1 && kind != 3) return cudaSuccess;  // the grid cost needs no check
  k_validate_cost<<<1216, 256, 0, st>>>(m, n, C, ldc, kind, px, py, dim, scale, scal);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_certify_prep(int64_t n, const double* gam, float* gam32, float* gamlo, double* scal,
                                const RedBuf& rb, cudaStream_t st) {
  k_certify_prep<<<nblk(n), kRB, 0, st>>>(n, gam, gam32, gamlo, scal, rb);
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
