// Sparsified Hessian H_rho of Alg. 1 in CSR/CSC form and the Newton-direction
// solve of Alg. 2 by Jacobi-preconditioned CG in one persistent kernel.
//
// H_rho v = (c_rho o v - P_rho^T (a o (P_rho v))) / eta, with c_rho = P_rho^T a,
// is applied matrix-free: a row phase (u = P_rho v over CSR rows, row i* dense)
// and a column phase (P_rho^T w over CSC columns).  The CSC copy is built
// deterministically: block b of the sparsify pass owns rows [b*rpb, (b+1)*rpb),
// its per-column counts are prefix-summed over blocks, and each block scatters
// its rows in row order.
#include <type_traits>

#include <atomic>
#include <mutex>

#include "../../include/ibsn.h"
#include "common.cuh"
#include "internal.h"

namespace ibsn {

namespace {

__global__ void k_colscan(const int32_t* __restrict__ blkcnt, int32_t* __restrict__ blkpre, int nb, int64_t ldk,
                          int64_t n, int64_t* colptr) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int64_t run = 0;
  for (int q = 0; q < nb; ++q) {
    blkpre[(int64_t)q * ldk + j] = (int32_t)run;
    run += blkcnt[(int64_t)q * ldk + j];
  }
  colptr[j + 1] = run;
}

__global__ void __launch_bounds__(1024) k_scan_colptr(int64_t n, int64_t* colptr) {
  __shared__ long long sh[32];
  const int64_t per = (n + 1023) / 1024;
  const int64_t j0 = (int64_t)threadIdx.x * per;
  const int64_t j1 = j0 + per < n ? j0 + per : n;
  long long s = 0;
  for (int64_t j = j0; j < j1; ++j) s += colptr[j + 1];
  // block exclusive scan of s
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long x = s;
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  long long base = 0;
  for (int q = 0; q < w; ++q) base += sh[q];
  long long run = base + x - s;
  __syncthreads();
  for (int64_t j = j0; j < j1; ++j) {
    const long long t = colptr[j + 1];
    colptr[j] = run;
    run += t;
  }
  if (threadIdx.x == 1023) colptr[n] = run;
  // colptr[j] for j < n now holds the start of column j; colptr[n] = nnz
}

template <typename T>
__global__ void k_scatter(const int32_t* __restrict__ pool_col, const T* __restrict__ pool_val,
                          const int64_t* __restrict__ row_start, const int32_t* __restrict__ row_len,
                          const int32_t* __restrict__ blkpre, const int64_t* __restrict__ colptr,
                          int32_t* __restrict__ csc_row, T* __restrict__ csc_val, int m, int64_t n, int64_t ldk,
                          int rpb) {
  extern __shared__ int32_t cursor[];
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) cursor[j] = blkpre[(int64_t)blockIdx.x * ldk + j];
  __syncthreads();
  const int r0 = blockIdx.x * rpb, r1 = min(m, r0 + rpb);
  for (int i = r0; i < r1; ++i) {
    const int64_t s = row_start[i];
    const int len = row_len[i];
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
      const int32_t j = pool_col[s + k];
      const int64_t pos = colptr[j] + cursor[j];
      cursor[j] += 1;  // columns are distinct within a row
      csc_row[pos] = i;
      csc_val[pos] = pool_val[s + k];
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void k_colstats(const int64_t* __restrict__ colptr, const int32_t* __restrict__ csc_row,
                           const T* __restrict__ csc_val, const T* __restrict__ prow, const double* __restrict__ a,
                           int istar, int64_t n, double eta, double* crho, double* diag) {
  const int lane = threadIdx.x & 31;
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= n) return;
  double s1 = 0.0, s2 = 0.0;
  for (int64_t k = colptr[j] + lane; k < colptr[j + 1]; k += 32) {
    const double v = (double)csc_val[k];
    const double av = a[csc_row[k]] * v;
    s1 += av;
    s2 += av * v;
  }
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  if (lane == 0) {
    const double p = (double)prow[j];
    const double as = a[istar];
    s1 += as * p;
    s2 += as * p * p;
    crho[j] = s1;
    diag[j] = (s1 - s2) / eta;
  }
}

template <typename T>
__global__ void k_export_sparse(const int32_t* __restrict__ pool_col, const T* __restrict__ pool_val,
                                const int64_t* __restrict__ row_start, const int32_t* __restrict__ row_len,
                                const T* __restrict__ prow, int m, int64_t n, int istar, double* out) {
  const int lane = threadIdx.x & 31;
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (i >= m) return;
  if (i == istar) {
    for (int64_t j = lane; j < n; j += 32) out[(int64_t)i * n + j] = (double)prow[j];
    return;
  }
  const int64_t s = row_start[i];
  for (int k = lane; k < row_len[i]; k += 32) out[(int64_t)i * n + pool_col[s + k]] = (double)pool_val[s + k];
}

// ---------------------------------------------------------------------------
// Persistent preconditioned CG in the Chronopoulos-Gear arrangement: both
// inner products of an iteration are formed after its single operator
// application, so an iteration needs two grid barriers:
//   R (rows):  t_i = a_i sum_j P_ij u_j, u = M^{-1} r formed on the fly from the
//              packed column state; row i* (dense) as per-block partial dots
//   C (cols):  s = w + beta s, p = u + beta p, x += alpha p, r -= alpha s,
//              u = M^{-1} r, w = A u with A = (diag(c_rho) - P^T diag(a) P)/eta
//              + shift I; partials of (r,u), (w,u), (r,r)
// Rows and columns are handled by groups of G lanes; each lane keeps up to E
// entries of its row and of its column in registers for the whole solve, the
// rest is streamed.  Column state is packed per column as {r, w} {s, 1/diag}.
// ---------------------------------------------------------------------------
constexpr int kPcgThreads = 512;

template <typename T>
struct PcgArgs {
  const int64_t* row_start;
  const int32_t* row_len;
  const int32_t* col;
  const T* val;
  const int64_t* colptr;
  const int32_t* crow;
  const T* cval;
  const T* prow;
  const double* a;
  const double* crho;
  const double* diag;
  const double* rhs;
  double* x;
  double* p;
  double2* cs;   // 2n: [2j] = {r_j, w_j}, [2j+1] = {s_j, 1/diag_j}
  float4* cs32;  // n: float copy {r, w, s, 1/diag} gathered by the float32 row phase
  T* t;          // m
  float2* part;  // [6][nb] float-float block partials
  unsigned int* bar;
  int* err;
  double* scal;
  int m, istar;
  int64_t n;
  double inv_eta, shift, rtol;
  int maxit;
  unsigned long long budget_ns;
};

template <int G>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// u_j = (r_j - alpha (w_j + beta s_j)) / diag_j from the packed state
__device__ __forceinline__ double u_from(const double2* cs, int64_t j, double alpha, double beta) {
  const double2 rw = __ldcg(cs + 2 * j);
  const double2 sd = __ldcg(cs + 2 * j + 1);
  return (rw.x - alpha * (rw.y + beta * sd.x)) * sd.y;
}
// the same from the float copy (float32 Hessian: the product needs no more)
__device__ __forceinline__ float u_from32(const float4* cs, int64_t j, float alpha, float beta) {
  const float4 c = __ldcg(cs + j);
  return (c.x - alpha * (c.y + beta * c.z)) * c.w;
}
template <typename T>
__device__ __forceinline__ T u_at(const double2* cs, const float4* cs32, int64_t j, double alpha, double beta,
                                  float alpha32, float beta32) {
  if constexpr (std::is_same<T, float>::value) {
    return u_from32(cs32, j, alpha32, beta32);
  } else {
    return u_from(cs, j, alpha, beta);
  }
}
template <int G, typename V>
__device__ __forceinline__ V group_sum_t(V v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T, int G, int E>
__global__ void __launch_bounds__(kPcgThreads, 1) k_pcg(PcgArgs<T> A) {
  __shared__ float sh[2 * 6 * 32];
  const int nb = gridDim.x;
  const int gl = threadIdx.x & (G - 1);
  const int gid = (int)(((int64_t)blockIdx.x * kPcgThreads + threadIdx.x) / G);
  const int ngroups = nb * (kPcgThreads / G);
  const int64_t gtid = (int64_t)blockIdx.x * kPcgThreads + threadIdx.x;
  const int64_t nthr = (int64_t)nb * kPcgThreads;

  // registers: the first row and the first column of this group
  const int i0 = gid;
  int r_len = 0;
  int64_t r_start = 0;
  int r_col[E];
  T r_val[E];
  if (i0 < A.m && i0 != A.istar) {
    r_start = A.row_start[i0];
    r_len = A.row_len[i0];
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = gl + e * G;
    r_col[e] = k < r_len ? A.col[r_start + k] : 0;
    r_val[e] = k < r_len ? A.val[r_start + k] : T(0);
  }
  const int64_t j0 = gid;
  int64_t c_start = 0;
  int c_len = 0;
  int c_row[E];
  T c_val[E];
  if (j0 < A.n) {
    c_start = A.colptr[j0];
    c_len = (int)(A.colptr[j0 + 1] - c_start);
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = gl + e * G;
    c_row[e] = k < c_len ? A.crow[c_start + k] : 0;
    c_val[e] = k < c_len ? A.cval[c_start + k] : T(0);
  }

  // state: r = rhs, w = 0, s = 0, p = 0, x = 0.  Row i* of P_rho (dense, q)
  // enters H u through the scalar q^T u; for the next u = (r - alpha (w +
  // beta s)) / diag it is Qr - alpha (Qw + beta Qs) with Qv = sum_j q_j v_j / diag_j
  // over the stored state, so those three sums ride along with the CG dots.
  constexpr bool F32 = std::is_same<T, float>::value;
  double red[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t j = gtid; j < A.n; j += nthr) {
    const double dinv = 1.0 / A.diag[j];
    __stcg(A.cs + 2 * j, make_double2(A.rhs[j], 0.0));
    __stcg(A.cs + 2 * j + 1, make_double2(0.0, dinv));
    if constexpr (F32) __stcg(A.cs32 + j, make_float4((float)A.rhs[j], 0.f, 0.f, (float)dinv));
    __stcg(A.p + j, 0.0);
    __stcg(A.x + j, 0.0);
    red[3] += (double)A.prow[j] * dinv * A.rhs[j];
  }
  if (!grid_allreduce<kPcgThreads, 6>(red, A.part, A.bar, A.err, A.budget_ns, sh)) return;
  double Qr = red[3], Qw = 0.0, Qs = 0.0;

  double alpha = 0.0, beta = 0.0, gam = 0.0, bnorm = 0.0, rr = 0.0;
  bool warm = true;
  int it = 0;
  for (;;) {
    // ---- R: t = a o (P u); the trip count is uniform so group shuffles never diverge
    const float alpha32 = (float)alpha, beta32 = (float)beta;
    const int qr = (A.m + ngroups - 1) / ngroups;
    for (int q = 0; q < qr; ++q) {
      const int i = i0 + q * ngroups;
      T acc = T(0);
      if (i < A.m && i != A.istar) {
        if (q == 0) {
#pragma unroll
          for (int e = 0; e < E; ++e)
            if (gl + e * G < r_len) acc += r_val[e] * u_at<T>(A.cs, A.cs32, r_col[e], alpha, beta, alpha32, beta32);
          for (int k = gl + E * G; k < r_len; k += G)
            acc += A.val[r_start + k] * u_at<T>(A.cs, A.cs32, A.col[r_start + k], alpha, beta, alpha32, beta32);
        } else {
          const int64_t st = A.row_start[i];
          const int ln = A.row_len[i];
          for (int k = gl; k < ln; k += G)
            acc += A.val[st + k] * u_at<T>(A.cs, A.cs32, A.col[st + k], alpha, beta, alpha32, beta32);
        }
      }
      acc = group_sum_t<G>(acc);
      if (gl == 0 && i < A.m && i != A.istar) __stcg(A.t + i, (T)(A.a[i] * (double)acc));
    }
    if (!grid_barrier(A.bar, nullptr, A.err, A.budget_ns)) return;
    // ---- C: vector updates, w = A u, partial dots
    const double tstar = A.a[A.istar] * (Qr - alpha * (Qw + beta * Qs));
    double dg = 0.0, dd = 0.0, dr = 0.0, qr2 = 0.0, qw2 = 0.0, qs2 = 0.0;
    const int64_t qc = (A.n + ngroups - 1) / ngroups;
    for (int64_t q = 0; q < qc; ++q) {
      const int64_t j = j0 + q * ngroups;
      T acc = T(0);
      if (j >= A.n) {
        // no column for this group in this round
      } else if (q == 0) {
#pragma unroll
        for (int e = 0; e < E; ++e)
          if (gl + e * G < c_len) acc += c_val[e] * __ldcg(A.t + c_row[e]);
        for (int k = gl + E * G; k < c_len; k += G) acc += A.cval[c_start + k] * __ldcg(A.t + A.crow[c_start + k]);
      } else {
        const int64_t k0 = A.colptr[j], k1 = A.colptr[j + 1];
        for (int64_t k = k0 + gl; k < k1; k += G) acc += A.cval[k] * __ldcg(A.t + A.crow[k]);
      }
      acc = group_sum_t<G>(acc);
      if (gl == 0 && j < A.n) {
        const double2 rw = __ldcg(A.cs + 2 * j);
        const double2 sd = __ldcg(A.cs + 2 * j + 1);
        const double qj = (double)A.prow[j];
        const double s_new = rw.y + beta * sd.x;
        const double p_new = rw.x * sd.y + beta * __ldcg(A.p + j);
        const double r_new = rw.x - alpha * s_new;
        const double u_new = r_new * sd.y;
        const double v = (double)acc + qj * tstar;
        const double w_new = (A.crho[j] * u_new - v) * A.inv_eta + A.shift * u_new;
        __stcg(A.x + j, __ldcg(A.x + j) + alpha * p_new);
        __stcg(A.p + j, p_new);
        __stcg(A.cs + 2 * j, make_double2(r_new, w_new));
        __stcg(A.cs + 2 * j + 1, make_double2(s_new, sd.y));
        if constexpr (F32) __stcg(A.cs32 + j, make_float4((float)r_new, (float)w_new, (float)s_new, (float)sd.y));
        dg += r_new * u_new;
        dd += w_new * u_new;
        dr += r_new * r_new;
        const double qd = qj * sd.y;
        qr2 += qd * r_new;
        qw2 += qd * w_new;
        qs2 += qd * s_new;
      }
    }
    double t6[6] = {dg, dd, dr, qr2, qw2, qs2};
    if (!grid_allreduce<kPcgThreads, 6>(t6, A.part, A.bar, A.err, A.budget_ns, sh)) return;
    const double g1 = t6[0];
    const double d1v = t6[1];
    rr = t6[2];
    Qr = t6[3];
    Qw = t6[4];
    Qs = t6[5];
    if (warm) {
      warm = false;
      bnorm = sqrt(rr);
      if (bnorm == 0.0 || !(d1v > 0.0)) break;
      alpha = g1 / d1v;
      beta = 0.0;
      gam = g1;
      continue;
    }
    ++it;
    if (sqrt(rr) <= A.rtol * bnorm || it >= A.maxit) break;
    beta = g1 / gam;
    const double den = d1v - beta * g1 / alpha;
    if (!(den > 0.0)) break;
    alpha = g1 / den;
    gam = g1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.scal[S_CG_ITERS] = (double)it;
    A.scal[S_CG_RES] = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
  }
}

__global__ void k_len_stats(const int32_t* __restrict__ row_len, const int64_t* __restrict__ colptr, int m, int64_t n,
                            double* scal) {
  __shared__ int sh[64];
  int mr = 0, mc = 0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) mr = max(mr, row_len[i]);
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) mc = max(mc, (int)(colptr[j + 1] - colptr[j]));
  for (int o = 16; o > 0; o >>= 1) {
    mr = max(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    mc = max(mc, __shfl_xor_sync(0xffffffffu, mc, o));
  }
  if ((threadIdx.x & 31) == 0) {
    sh[threadIdx.x >> 5] = mr;
    sh[32 + (threadIdx.x >> 5)] = mc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      mr = max(mr, sh[w]);
      mc = max(mc, sh[32 + w]);
    }
    scal[S_MAXROW] = mr;
    scal[S_MAXCOL] = mc;
  }
}

// ---------------------------------------------------------------------------
// Float32 CG for a float32 sparsified Hessian (mixed precision).  Same
// Chronopoulos-Gear arrangement as k_pcg; the vectors, recurrences and
// products are float32 (the operator itself is float32-accurate and the
// solve stops at a relative residual >= 1e-6), the inner products are
// accumulated in float-float and alpha, beta are formed in float64.
// Column state per column: {r, w, s, 1/diag} (float4); x, p float.
// ---------------------------------------------------------------------------
// Grid all-reduce of the six float CG sums for k_pcg32 (float-float, fixed
// order).  Every block publishes its six partials as one 64-byte record
// (float2 x 6, padded to 8), arrives at the grid counter and waits (bounded as
// in grid_barrier); then one thread per block partial loads that block's
// record with three 16-byte loads, so all partials are in flight at once, and
// the block's warps reduce them.  Only thread 0 receives the totals (tot, as
// float-float pairs); the caller broadcasts what the other threads need.
// Returns false to every thread when the wait ran out or *err was set.
__device__ __forceinline__ bool pcg_allreduce6(const float (&vin)[6], FF (&tot)[6], float4* part,
                                               unsigned int* count, int* err, unsigned long long budget_ns,
                                               float* sh) {
  constexpr int NW = kPcgThreads / 32;
  __shared__ int s_ok;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nb = (int)gridDim.x;
  FF f[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) f[q] = warp_sum_ff(FF{vin[q], 0.f});
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      sh[2 * (q * NW + w)] = f[q].hi;
      sh[2 * (q * NW + w) + 1] = f[q].lo;
    }
  }
  __syncthreads();
  if (w == 0) {
    FF t[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      t[q] = lane < NW ? FF{sh[2 * (q * NW + lane)], sh[2 * (q * NW + lane) + 1]} : FF{0.f, 0.f};
      t[q] = warp_sum_ff(t[q]);
    }
    if (lane == 0) {
      float4* rec = part + (size_t)blockIdx.x * 4;
      __stcg(rec + 0, make_float4(t[0].hi, t[0].lo, t[1].hi, t[1].lo));
      __stcg(rec + 1, make_float4(t[2].hi, t[2].lo, t[3].hi, t[3].lo));
      __stcg(rec + 2, make_float4(t[4].hi, t[4].lo, t[5].hi, t[5].lo));
      int ok = 1;
      unsigned int old;
      asm volatile("fence.acq_rel.gpu;\n\tatom.add.release.gpu.u32 %0, [%1], 1;" : "=r"(old) : "l"(count) : "memory");
      const unsigned int target = (old / gridDim.x + 1u) * gridDim.x;
      unsigned int spins = 0;
      unsigned long long t0 = 0;
      for (;;) {
        unsigned int cur;
        asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(cur) : "l"(count) : "memory");
        if ((int)(cur - target) >= 0) break;
        if ((++spins & 63u) == 0) {
          if (*(volatile int*)err != 0) { ok = 0; break; }
          const unsigned long long now = globaltimer_ns();
          if (t0 == 0) {
            t0 = now;
          } else if (now - t0 > budget_ns) {
            atomicExch(err, (int)kDevTimeout);
            ok = 0;
            break;
          }
        }
      }
      s_ok = ok;
    }
  }
  __syncthreads();
  if (!s_ok) return false;
  // partial records: thread b loads block b's (b < nb <= kPcgThreads); the
  // warp sums go to shared memory (reusing sh: all earlier reads are done)
  constexpr int kRec = 12;  // floats per record in use
  float* shr = sh;
  const int nwr = (nb + 31) >> 5;
  if (w < nwr) {
    FF r[6];
    const int b = threadIdx.x;
    if (b < nb) {
      const float4* rec = part + (size_t)b * 4;
      const float4 v0 = __ldcg(rec + 0), v1 = __ldcg(rec + 1), v2 = __ldcg(rec + 2);
      r[0] = FF{v0.x, v0.y};
      r[1] = FF{v0.z, v0.w};
      r[2] = FF{v1.x, v1.y};
      r[3] = FF{v1.z, v1.w};
      r[4] = FF{v2.x, v2.y};
      r[5] = FF{v2.z, v2.w};
    } else {
#pragma unroll
      for (int q = 0; q < 6; ++q) r[q] = FF{0.f, 0.f};
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) r[q] = warp_sum_ff(r[q]);
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        shr[w * kRec + 2 * q] = r[q].hi;
        shr[w * kRec + 2 * q + 1] = r[q].lo;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      FF a{0.f, 0.f};
      for (int u = 0; u < nwr; ++u) a = ff_add(a, FF{shr[u * kRec + 2 * q], shr[u * kRec + 2 * q + 1]});
      tot[q] = a;
    }
  }
  return true;
}

struct Pcg32Args {
  const int64_t* row_start;
  const int32_t* row_len;
  const int32_t* col;
  const float* val;
  const int64_t* colptr;
  const int32_t* crow;
  const float* cval;
  const float* prow;
  const float* a32;
  const double* crho;
  const double* diag;
  const double* rhs;
  double* x_out;
  float* x;
  float* p;
  float4* cs;
  float* t;
  float* crho32;
  float4* part;
  unsigned int* bar;
  int* err;
  double* scal;
  int m, istar;
  int64_t n;
  float inv_eta, shift;
  double rtol;
  int maxit;
  unsigned long long budget_ns;
};

template <int G, int E>
__global__ void __launch_bounds__(kPcgThreads, 1) k_pcg32(Pcg32Args A) {
  __shared__ float sh[2 * 6 * 32];
  const int nb = gridDim.x;
  const int gl = threadIdx.x & (G - 1);
  const int gid = (int)(((int64_t)blockIdx.x * kPcgThreads + threadIdx.x) / G);
  const int ngroups = nb * (kPcgThreads / G);
  const int64_t gtid = (int64_t)blockIdx.x * kPcgThreads + threadIdx.x;
  const int64_t nthr = (int64_t)nb * kPcgThreads;

  const int i0 = gid;
  int r_len = 0;
  int64_t r_start = 0;
  int r_col[E];
  float r_val[E];
  if (i0 < A.m && i0 != A.istar) {
    r_start = A.row_start[i0];
    r_len = A.row_len[i0];
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = gl + e * G;
    r_col[e] = k < r_len ? A.col[r_start + k] : 0;
    r_val[e] = k < r_len ? A.val[r_start + k] : 0.f;
  }
  const int64_t j0 = gid;
  int64_t c_start = 0;
  int c_len = 0;
  int c_row[E];
  float c_val[E];
  if (j0 < A.n) {
    c_start = A.colptr[j0];
    c_len = (int)(A.colptr[j0 + 1] - c_start);
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = gl + e * G;
    c_row[e] = k < c_len ? A.crow[c_start + k] : 0;
    c_val[e] = k < c_len ? A.cval[c_start + k] : 0.f;
  }

  // state r = rhs, w = s = p = x = 0; row i* (q) enters through q^T u, formed
  // from three sums over the stored state as in k_pcg
  float red[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int64_t j = gtid; j < A.n; j += nthr) {
    const float dinv = (float)(1.0 / A.diag[j]);
    const float r0 = (float)A.rhs[j];
    __stcg(A.cs + j, make_float4(r0, 0.f, 0.f, dinv));
    __stcg(A.p + j, 0.f);
    __stcg(A.x + j, 0.f);
    __stcg(A.crho32 + j, (float)A.crho[j]);
    red[3] += A.prow[j] * dinv * r0;
  }
  // The CG scalars live in thread 0; the other threads receive alpha, beta
  // and t* through shared memory after each reduction.  alpha and beta are
  // float (the vectors are float, so their rounding is of the same order);
  // the totals arrive as float-float sums and t* = a_i* q^T u, a difference
  // that can cancel, is formed in float-float.  No float64 work on this
  // serial path: it runs once per iteration between two grid-wide waits.
  __shared__ float s_a32, s_b32, s_tstar;
  __shared__ int s_done;
  FF tot[6];
  if (!pcg_allreduce6(red, tot, A.part, A.bar, A.err, A.budget_ns, sh)) return;
  FF Qr = tot[3], Qw{0.f, 0.f}, Qs{0.f, 0.f};
  float alpha = 0.f, beta = 0.f, gam = 0.f, rr0 = 0.f, rr = 0.f;
  const float rtol2 = (float)(A.rtol * A.rtol);
  const float astar = A.a32[A.istar];
  bool warm = true;
  int it = 0;
  if (threadIdx.x == 0) {
    s_a32 = 0.f;
    s_b32 = 0.f;
    s_tstar = astar * Qr.hi;
  }
  __syncthreads();
  for (;;) {
    const float a32 = s_a32, b32 = s_b32, tstar = s_tstar;
    // ---- R: t = a o (P u)
    const int qr = (A.m + ngroups - 1) / ngroups;
    for (int q = 0; q < qr; ++q) {
      const int i = i0 + q * ngroups;
      float acc = 0.f;
      if (i < A.m && i != A.istar) {
        if (q == 0) {
#pragma unroll
          for (int e = 0; e < E; ++e)
            if (gl + e * G < r_len) acc += r_val[e] * u_from32(A.cs, r_col[e], a32, b32);
          for (int k = gl + E * G; k < r_len; k += G) acc += A.val[r_start + k] * u_from32(A.cs, A.col[r_start + k], a32, b32);
        } else {
          const int64_t st = A.row_start[i];
          const int ln = A.row_len[i];
          for (int k = gl; k < ln; k += G) acc += A.val[st + k] * u_from32(A.cs, A.col[st + k], a32, b32);
        }
      }
      acc = group_sum_t<G>(acc);
      if (gl == 0 && i < A.m && i != A.istar) __stcg(A.t + i, A.a32[i] * acc);
    }
    if (!grid_barrier(A.bar, nullptr, A.err, A.budget_ns)) return;
    // ---- C
    float dsum[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int64_t qc = (A.n + ngroups - 1) / ngroups;
    for (int64_t q = 0; q < qc; ++q) {
      const int64_t j = j0 + q * ngroups;
      float acc = 0.f;
      if (j >= A.n) {
      } else if (q == 0) {
#pragma unroll
        for (int e = 0; e < E; ++e)
          if (gl + e * G < c_len) acc += c_val[e] * __ldcg(A.t + c_row[e]);
        for (int k = gl + E * G; k < c_len; k += G) acc += A.cval[c_start + k] * __ldcg(A.t + A.crow[c_start + k]);
      } else {
        const int64_t k0 = A.colptr[j], k1 = A.colptr[j + 1];
        for (int64_t k = k0 + gl; k < k1; k += G) acc += A.cval[k] * __ldcg(A.t + A.crow[k]);
      }
      acc = group_sum_t<G>(acc);
      if (gl == 0 && j < A.n) {
        const float4 c = __ldcg(A.cs + j);
        const float qj = A.prow[j];
        const float s_new = c.y + b32 * c.z;
        const float p_new = c.x * c.w + b32 * __ldcg(A.p + j);
        const float r_new = c.x - a32 * s_new;
        const float u_new = r_new * c.w;
        const float v = acc + qj * tstar;
        const float w_new = (__ldcg(A.crho32 + j) * u_new - v) * A.inv_eta + A.shift * u_new;
        __stcg(A.x + j, __ldcg(A.x + j) + a32 * p_new);
        __stcg(A.p + j, p_new);
        __stcg(A.cs + j, make_float4(r_new, w_new, s_new, c.w));
        const float qd = qj * c.w;
        dsum[0] += r_new * u_new;
        dsum[1] += w_new * u_new;
        dsum[2] += r_new * r_new;
        dsum[3] += qd * r_new;
        dsum[4] += qd * w_new;
        dsum[5] += qd * s_new;
      }
    }
    if (!pcg_allreduce6(dsum, tot, A.part, A.bar, A.err, A.budget_ns, sh)) return;
    if (threadIdx.x == 0) {
      // Chronopoulos-Gear update (one thread per block; every block forms the
      // same values from the same totals)
      const float g1 = tot[0].hi;
      const float d1v = tot[1].hi;
      rr = tot[2].hi;
      Qr = tot[3];
      Qw = tot[4];
      Qs = tot[5];
      int done = 0;
      if (warm) {
        warm = false;
        rr0 = rr;
        if (!(rr0 > 0.f) || !(d1v > 0.f)) {
          done = 1;
        } else {
          alpha = g1 / d1v;
          beta = 0.f;
          gam = g1;
        }
      } else {
        ++it;
        if (rr <= rtol2 * rr0 || it >= A.maxit) {
          done = 1;
        } else {
          beta = g1 / gam;
          const float den = d1v - beta * (g1 / alpha);
          if (!(den > 0.f)) {
            done = 1;
          } else {
            alpha = g1 / den;
            gam = g1;
          }
        }
      }
      s_done = done;
      s_a32 = alpha;
      s_b32 = beta;
      // row i* enters through q^T u = Qr - alpha (Qw + beta Qs) of the next iteration
      const FF qu = ff_add(Qr, ff_neg(ff_mul_f(ff_add(Qw, ff_mul_f(Qs, beta)), alpha)));
      s_tstar = astar * qu.hi;
    }
    __syncthreads();
    if (s_done) break;
  }
  for (int64_t j = gtid; j < A.n; j += nthr) A.x_out[j] = (double)__ldcg(A.x + j);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.scal[S_CG_ITERS] = (double)it;
    A.scal[S_CG_RES] = rr0 > 0.f ? sqrt((double)rr / (double)rr0) : 0.0;
  }
}

}  // namespace

int pcg_max_blocks(int nsm) { return nsm; }

cudaError_t launch_len_stats(const SparseBufs& S, int m, int64_t n, double* scal, cudaStream_t st) {
  k_len_stats<<<1, 1024, 0, st>>>(S.row_len, S.colptr, m, n, scal);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_csc_build(const SparseBufs& S, int m, int64_t n, int64_t ldk, int nb, int rpb, bool fp64,
                             const double* a, int istar, double eta, cudaStream_t st) {
  k_colscan<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S.blkcnt, S.blkpre, nb, ldk, n, S.colptr);
  k_scan_colptr<<<1, 1024, 0, st>>>(n, S.colptr);
  note_launch(4);
  const size_t smem = (size_t)n * sizeof(int32_t);
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    cudaFuncSetAttribute(k_scatter<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_scatter<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  if (fp64) {
    k_scatter<double><<<nb, 256, smem, st>>>(S.pool_col, (const double*)S.pool_val, S.row_start, S.row_len,
                                             S.blkpre, S.colptr, S.csc_row, (double*)S.csc_val, m, n, ldk, rpb);
    k_colstats<double><<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(
        S.colptr, S.csc_row, (const double*)S.csc_val, (const double*)S.prow, a, istar, n, eta, S.crho, S.diag);
  } else {
    k_scatter<float><<<nb, 256, smem, st>>>(S.pool_col, (const float*)S.pool_val, S.row_start, S.row_len,
                                            S.blkpre, S.colptr, S.csc_row, (float*)S.csc_val, m, n, ldk, rpb);
    k_colstats<float><<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(
        S.colptr, S.csc_row, (const float*)S.csc_val, (const float*)S.prow, a, istar, n, eta, S.crho, S.diag);
  }
  return cudaGetLastError();
}

cudaError_t launch_export_sparse(const SparseBufs& S, int m, int64_t n, int istar, bool fp64, double* out,
                                 cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * (size_t)m * (size_t)n, st);
  if (e != cudaSuccess) return e;
  const unsigned nbk = (unsigned)(((int64_t)m * 32 + 255) / 256);
  note_launch();
  if (fp64)
    k_export_sparse<double><<<nbk, 256, 0, st>>>(S.pool_col, (const double*)S.pool_val, S.row_start, S.row_len,
                                                 (const double*)S.prow, m, n, istar, out);
  else
    k_export_sparse<float><<<nbk, 256, 0, st>>>(S.pool_col, (const float*)S.pool_val, S.row_start, S.row_len,
                                                (const float*)S.prow, m, n, istar, out);
  return cudaGetLastError();
}

template <int G, int E>
static cudaError_t launch_pcg32_g(Pcg32Args& A, int nsm, cudaStream_t st) {
  static std::atomic<int> occ_cache{0};
  int occ = occ_cache.load();
  if (occ == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg32<G, E>, kPcgThreads, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorCooperativeLaunchTooLarge;
    occ_cache.store(occ);
  }
  // pcg_allreduce6 gives one thread of a block to each block's partial record
  if (nsm > kPcgThreads) return cudaErrorInvalidConfiguration;
  void* args[] = {(void*)&A};
  note_launch();
  return cudaLaunchCooperativeKernel((const void*)k_pcg32<G, E>, dim3(nsm), dim3(kPcgThreads), args, 0, st);
}

template <typename T, int G, int E>
static cudaError_t launch_pcg_g(PcgArgs<T>& A, int nsm, cudaStream_t st) {
  static std::atomic<int> occ_cache{0};
  int occ = occ_cache.load();
  if (occ == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg<T, G, E>, kPcgThreads, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorCooperativeLaunchTooLarge;
    occ_cache.store(occ);
  }
  // one block per SM keeps the barriers short; all blocks are co-resident
  const int nb = nsm;
  void* args[] = {(void*)&A};
  note_launch();
  return cudaLaunchCooperativeKernel((const void*)k_pcg<T, G, E>, dim3(nb), dim3(kPcgThreads), args, 0, st);
}

template <typename T>
static cudaError_t launch_pcg_t(const SparseBufs& S, const PcgBufs& B, int m, int64_t n, int istar,
                                const double* a, double eta, double shift, double rtol, int maxit, double timeout_s,
                                int nsm, int64_t nnz, double* scal, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(B.bar, 0, 2 * sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(B.err, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  PcgArgs<T> A;
  A.row_start = S.row_start;
  A.row_len = S.row_len;
  A.col = S.pool_col;
  A.val = (const T*)S.pool_val;
  A.colptr = S.colptr;
  A.crow = S.csc_row;
  A.cval = (const T*)S.csc_val;
  A.prow = (const T*)S.prow;
  A.a = a;
  A.crho = S.crho;
  A.diag = S.diag;
  A.rhs = B.rhs;
  A.x = B.x;
  A.p = B.p;
  A.cs = reinterpret_cast<double2*>(B.cs);
  A.cs32 = reinterpret_cast<float4*>(B.cs32);
  A.t = reinterpret_cast<T*>(B.t);
  A.part = reinterpret_cast<float2*>(B.part);
  A.bar = B.bar;
  A.err = B.err;
  A.scal = scal;
  A.m = m;
  A.istar = istar;
  A.n = n;
  A.inv_eta = 1.0 / eta;
  A.shift = shift;
  A.rtol = rtol;
  A.maxit = maxit;
  A.budget_ns = (unsigned long long)(timeout_s * 1e9);  // bound on each barrier wait
  // group width from the mean row length (rows and columns have the same mean)
  const double avg = (double)nnz / (double)(m > 1 ? m : 1);
  if (avg <= 12.0) return launch_pcg_g<T, 4, 4>(A, nsm, st);
  if (avg <= 28.0) return launch_pcg_g<T, 8, 4>(A, nsm, st);
  return launch_pcg_g<T, 32, 4>(A, nsm, st);
}

cudaError_t launch_pcg(const SparseBufs& S, const PcgBufs& B, int m, int64_t n, int istar, bool fp64,
                       const double* a, const float* a32, double eta, double shift, double rtol, int maxit,
                       double timeout_s, int nsm, int64_t nnz, double* scal, cudaStream_t st) {
  if (fp64)
    return launch_pcg_t<double>(S, B, m, n, istar, a, eta, shift, rtol, maxit, timeout_s, nsm, nnz, scal, st);
  cudaError_t e = cudaMemsetAsync(B.bar, 0, 2 * sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(B.err, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  Pcg32Args A;
  A.row_start = S.row_start;
  A.row_len = S.row_len;
  A.col = S.pool_col;
  A.val = (const float*)S.pool_val;
  A.colptr = S.colptr;
  A.crow = S.csc_row;
  A.cval = (const float*)S.csc_val;
  A.prow = (const float*)S.prow;
  A.a32 = a32;
  A.crho = S.crho;
  A.diag = S.diag;
  A.rhs = B.rhs;
  A.x_out = B.x;
  // float vectors carved from the float64 buffers (each has room for 2n floats)
  A.x = reinterpret_cast<float*>(B.p);
  A.p = reinterpret_cast<float*>(B.p) + n;
  A.cs = reinterpret_cast<float4*>(B.cs32);
  A.t = reinterpret_cast<float*>(B.t);
  A.crho32 = reinterpret_cast<float*>(B.cs);
  A.part = reinterpret_cast<float4*>(B.part);
  A.bar = B.bar;
  A.err = B.err;
  A.scal = scal;
  A.m = m;
  A.istar = istar;
  A.n = n;
  A.inv_eta = (float)(1.0 / eta);
  A.shift = (float)shift;
  A.rtol = rtol;
  A.maxit = maxit;
  A.budget_ns = (unsigned long long)(timeout_s * 1e9);
  const double avg = (double)nnz / (double)(m > 1 ? m : 1);
  if (avg <= 12.0) return launch_pcg32_g<4, 4>(A, nsm, st);
  if (avg <= 28.0) return launch_pcg32_g<8, 4>(A, nsm, st);
  return launch_pcg32_g<32, 4>(A, nsm, st);
}

}  // namespace ibsn

// ---------------------------------------------------------------------------
// Check of the bounded grid-wide wait that the persistent PCG kernels use
// (grid_barrier).  Every block except, when `withhold` is set, block 0 arrives
// at one grid barrier; with a block withheld the count can never reach its
// target, so the others wait out `budget_ns`, record kDevTimeout and return.
namespace ibsn {
namespace {
__global__ void k_wait_probe(unsigned int* count, int* err, int withhold, unsigned long long budget_ns) {
  if (withhold && blockIdx.x == 0) return;
  grid_barrier(count, nullptr, err, budget_ns);
}
}  // namespace
}  // namespace ibsn

extern "C" int ibsn_wait_probe(int blocks, int withhold, double timeout_s, void* scratch, void* stream) {
  using namespace ibsn;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IBSN_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return IBSN_ERR_CUDA;
  if (!scratch || (reinterpret_cast<uintptr_t>(scratch) & 7u) || blocks < 2 || blocks > nsm ||
      !(timeout_s > 0.0) || timeout_s > 10.0)
    return IBSN_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned int* count = static_cast<unsigned int*>(scratch);
  int* err = reinterpret_cast<int*>(count + 1);
  if (cudaMemsetAsync(scratch, 0, 2 * sizeof(unsigned int), st) != cudaSuccess) return IBSN_ERR_CUDA;
  int wh = withhold ? 1 : 0;
  unsigned long long budget = (unsigned long long)(timeout_s * 1e9);
  void* args[] = {(void*)&count, (void*)&err, (void*)&wh, (void*)&budget};
  if (cudaLaunchCooperativeKernel((const void*)k_wait_probe, dim3(blocks), dim3(32), args, 0, st) != cudaSuccess)
    return IBSN_ERR_CUDA;
  note_launch();
  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return IBSN_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return IBSN_ERR_CUDA;
  return h == kDevTimeout ? IBSN_ERR_TIMEOUT : IBSN_OK;
}
