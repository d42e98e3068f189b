// Device helpers shared by the IBSN kernels: vector types, warp/block
// reductions, compensated accumulators, and a bounded grid barrier.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace ibsn {

constexpr double kInf = __builtin_huge_val();

// Error flag values written by kernels into the context flag word.
enum DevError : int { kDevOk = 0, kDevTimeout = 1, kDevCapacity = 2 };

template <typename T>
struct VecT;
template <>
struct VecT<float> {
  using type = float4;
  static constexpr int N = 4;
};
template <>
struct VecT<double> {
  using type = double2;
  static constexpr int N = 2;
};

template <typename T>
__device__ __forceinline__ void load_vec(const T* __restrict__ p, T (&v)[VecT<T>::N]) {
  using V = typename VecT<T>::type;
  V x = *reinterpret_cast<const V*>(p);
  if constexpr (VecT<T>::N == 4) {
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else {
    v[0] = x.x; v[1] = x.y;
  }
}

template <typename T>
__device__ __forceinline__ void store_vec(T* __restrict__ p, const T (&v)[VecT<T>::N]) {
  using V = typename VecT<T>::type;
  V x;
  if constexpr (VecT<T>::N == 4) {
    x.x = v[0]; x.y = v[1]; x.z = v[2]; x.w = v[3];
  } else {
    x.x = v[0]; x.y = v[1];
  }
  *reinterpret_cast<V*>(p) = x;
}

// Streaming load that does not keep the line in L1 (the big matrices are read once).
template <typename T>
__device__ __forceinline__ void load_vec_stream(const T* __restrict__ p, T (&v)[VecT<T>::N]) {
  using V = typename VecT<T>::type;
  V x = __ldcs(reinterpret_cast<const V*>(p));
  if constexpr (VecT<T>::N == 4) {
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else {
    v[0] = x.x; v[1] = x.y;
  }
}

// exp in the pass precision.  float: one MUFU ex2 after scaling by log2(e).
__device__ __forceinline__ float exp_t(float x) { return exp2f(x * 1.4426950408889634f); }
__device__ __forceinline__ double exp_t(double x) { return exp(x); }

template <typename T>
__device__ __forceinline__ T neg_inf() { return -__builtin_huge_valf(); }
template <>
__device__ __forceinline__ double neg_inf<double>() { return -__builtin_huge_val(); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide reductions for blocks of NT threads (NT a multiple of 32).  `sh`
// must hold NT/32 values; every thread gets the result.  The leading barrier
// makes back-to-back calls on the same scratch safe.
template <int NT, int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* sh) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = warp_sum(v[q]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) sh[q * NW + w] = v[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double t = 0.0;
    if constexpr (NW == 1) {
      t = sh[q];
    } else {
      t = (lane < NW) ? sh[q * NW + lane] : 0.0;
      t = warp_sum(t);
    }
    v[q] = t;
  }
}

template <int NT, typename T>
__device__ __forceinline__ T block_max(T v, T* sh) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if constexpr (NW == 1) {
    return sh[0];
  } else {
    T t = (lane < NW) ? sh[lane] : neg_inf<T>();
    return warp_max(t);
  }
}

template <int NT>
__device__ __forceinline__ int block_exclusive_scan(int v, int* sh, int* total) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) sh[w] = x;
  __syncthreads();
  int base = 0, tot = 0;
#pragma unroll
  for (int q = 0; q < NW; ++q) {
    int s = sh[q];
    if (q < w) base += s;
    tot += s;
  }
  *total = tot;
  return base + x - v;
}

// ---------------------------------------------------------------------------
// Float-float arithmetic (an unevaluated sum hi + lo of two floats, ~48-bit
// significand).  On sm_103a a dependent float64 add costs ~64 cycles against
// ~4.5 for float32, so sums that need more than float32 accuracy are reduced
// in this form (error-free transformations of Knuth's TwoSum and Dekker's
// FastTwoSum) and converted to float64 once at the end.
// ---------------------------------------------------------------------------
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float err = (a - (s - bb)) + (b - bb);
  return {s, err};
}
__device__ __forceinline__ FF ff_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const FF s = ff_two_sum(a.hi, b.hi);
  return ff_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
// x * y for a float-float x and a float y (TwoProduct of the hi parts)
__device__ __forceinline__ FF ff_mul_f(FF x, float y) {
  const float p = x.hi * y;
  return ff_fast_two_sum(p, fmaf(x.hi, y, -p) + x.lo * y);
}
__device__ __forceinline__ FF ff_neg(FF x) { return {-x.hi, -x.lo}; }
// (a.hi + a.lo) / (b.hi + b.lo) to about 2^-46 relative (one correction step)
__device__ __forceinline__ FF ff_div(FF a, FF b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const float p = q1 * b.hi;
  const float pe = fmaf(q1, b.hi, -p);
  const float r = ((a.hi - p) - pe) + (a.lo - q1 * b.lo);
  return ff_fast_two_sum(q1, __fdiv_rn(r, b.hi));
}
__device__ __forceinline__ FF ff_from(double v) {
  const float hi = (float)v;
  return {hi, (float)(v - (double)hi)};
}
__device__ __forceinline__ double ff_to(FF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ FF warp_sum_ff(FF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    FF t;
    t.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    t.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = ff_add(v, t);
  }
  return v;
}

// Block sum of K float64 values in float-float; `sh` holds 2*K*NT/32 floats.
template <int NT, int K>
__device__ __forceinline__ void block_sum_ff(double (&v)[K], float* sh) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  FF f[K];
#pragma unroll
  for (int q = 0; q < K; ++q) f[q] = warp_sum_ff(ff_from(v[q]));
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      sh[2 * (q * NW + w)] = f[q].hi;
      sh[2 * (q * NW + w) + 1] = f[q].lo;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) {
    FF t = lane < NW ? FF{sh[2 * (q * NW + lane)], sh[2 * (q * NW + lane) + 1]} : FF{0.f, 0.f};
    if constexpr (NW > 1) t = warp_sum_ff(t);
    v[q] = ff_to(t);
  }
}

// Block sum of K float-float values, result on every thread (no float64
// arithmetic); `sh` holds 2*K*NT/32 floats.
template <int NT, int K>
__device__ __forceinline__ void block_sum_ffv(FF (&v)[K], float* sh) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = warp_sum_ff(v[q]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      sh[2 * (q * NW + w)] = v[q].hi;
      sh[2 * (q * NW + w) + 1] = v[q].lo;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) {
    FF t = lane < NW ? FF{sh[2 * (q * NW + lane)], sh[2 * (q * NW + lane) + 1]} : FF{0.f, 0.f};
    if constexpr (NW > 1) t = warp_sum_ff(t);
    v[q] = t;
  }
}

// Block sum of K floats (float32 passes, whose accuracy is float32 anyway).
template <int NT, int K>
__device__ __forceinline__ void block_sum_f(float (&v)[K], float* sh) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = warp_sum(v[q]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) sh[q * NW + w] = v[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) {
    float t = lane < NW ? sh[q * NW + lane] : 0.f;
    if constexpr (NW > 1) t = warp_sum(t);
    v[q] = t;
  }
}

// psi(s) = log1p(s) - s (Armijo difference form)
__device__ __forceinline__ double psi_log1p_minus(double s) {
  // log1p(s) - s; Taylor series for small |s| to avoid cancellation
  if (fabs(s) < 1e-3) {
    const double s2 = s * s;
    return s2 * (-0.5 + s * (1.0 / 3.0 + s * (-0.25 + s * (0.2 - s / 6.0))));
  }
  return log1p(s) - s;
}
__device__ __forceinline__ float psi_log1p_minus(float s) {
  // float: series sum_{k>=2} (-1)^(k+1) s^k / k to s^10 for |s| < 0.1
  if (fabsf(s) < 0.1f) {
    const float s2 = s * s;
    return s2 * (-0.5f + s * (1.f / 3.f + s * (-0.25f + s * (0.2f + s * (-1.f / 6.f + s * (1.f / 7.f + s * (
                     -0.125f + s * (1.f / 9.f + s * -0.1f))))))));
  }
  return log1pf(s) - s;
}

// Minimum of a float64 value over a block without float64 arithmetic: doubles
// are mapped to integers with the same order and reduced with integer ops.
__device__ __forceinline__ long long dbl_order(double v) {
  const long long b = __double_as_longlong(v);
  return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dbl_unorder(long long k) {
  return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffLL));
}
template <int NT>
__device__ __forceinline__ double block_min_exact(double v, long long* sh) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long k = dbl_order(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long o2 = __shfl_xor_sync(0xffffffffu, k, o);
    k = o2 < k ? o2 : k;
  }
  __syncthreads();
  if (lane == 0) sh[w] = k;
  __syncthreads();
  long long t = lane < NW ? sh[lane] : 0x7fffffffffffffffLL;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long o2 = __shfl_xor_sync(0xffffffffu, t, o);
    t = o2 < t ? o2 : t;
  }
  return dbl_unorder(t);
}

// Compensated (Kahan) accumulator for float; plain for double.
template <typename T>
struct Acc;
template <>
struct Acc<float> {
  float s, c;
  __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
  __device__ __forceinline__ void add(float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
  // s += w x with the product fused into the compensated step
  __device__ __forceinline__ void add_prod(float w, float x) {
    const float y = fmaf(w, x, -c);
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
};
template <>
struct Acc<double> {
  double s;
  __device__ __forceinline__ void zero() { s = 0.0; }
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ void add_prod(double w, double x) { s = fma(w, x, s); }
  __device__ __forceinline__ double value() const { return s; }
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for a cooperatively launched grid (all blocks co-resident).
// `count` only grows: every block adds 1 per barrier (release), then waits
// (acquire loads) until the count reaches the next multiple of gridDim.x.  The
// wait is bounded: after `budget_ns` of waiting (globaltimer) the block
// records kDevTimeout in *err and returns false; once *err is set every later
// call returns false at once, so all blocks leave the kernel.  The counter
// must be zeroed before the launch.
__device__ __forceinline__ bool grid_barrier(unsigned int* count, unsigned int* /*unused*/, int* err,
                                             unsigned long long budget_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
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
  __syncthreads();
  return s_ok != 0;
}

// Grid-wide all-reduce (sum) of K float64 values per thread fused with a grid
// barrier, two __syncthreads per call, sums in float-float: warp sums go to
// shared memory; warp 0 forms the block partials, publishes them (st.cg),
// arrives at the barrier (release), waits (acquire, bounded like
// grid_barrier), sums all blocks' partials in a fixed order and broadcasts the
// totals.  `part` holds 2 * K * gridDim.x floats, `sh` 2 * K * 32 + K doubles'
// worth of space.  Returns false when the wait ran out (or *err was set); the
// values in v are then unspecified.
template <int NT, int K>
__device__ __forceinline__ bool grid_allreduce(double (&v)[K], float2* part, unsigned int* count, int* err,
                                               unsigned long long budget_ns, float* sh) {
  constexpr int NW = NT / 32;
  __shared__ int s_ok;
  __shared__ double s_tot[K];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  FF f[K];
#pragma unroll
  for (int q = 0; q < K; ++q) f[q] = warp_sum_ff(ff_from(v[q]));
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      sh[2 * (q * NW + w)] = f[q].hi;
      sh[2 * (q * NW + w) + 1] = f[q].lo;
    }
  }
  __syncthreads();
  if (w == 0) {
    const int nb = (int)gridDim.x;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      FF t = lane < NW ? FF{sh[2 * (q * NW + lane)], sh[2 * (q * NW + lane) + 1]} : FF{0.f, 0.f};
      t = warp_sum_ff(t);
      if (lane == 0) __stcg(part + (size_t)q * nb + blockIdx.x, make_float2(t.hi, t.lo));
    }
    int ok = 1;
    if (lane == 0) {
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
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) {
#pragma unroll
      for (int q = 0; q < K; ++q) {
        FF t{0.f, 0.f};
        for (int b = lane; b < nb; b += 32) {
          const float2 pv = __ldcg(part + (size_t)q * nb + b);
          t = ff_add(t, FF{pv.x, pv.y});
        }
        t = warp_sum_ff(t);
        if (lane == 0) s_tot[q] = ff_to(t);
      }
    }
    if (lane == 0) s_ok = ok;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = s_tot[q];
  return s_ok != 0;
}

// grid_allreduce for float inputs (no float64 conversion on the way in): the
// float values are summed in float-float and returned as float64 totals.
template <int NT, int K>
__device__ __forceinline__ bool grid_allreduce_f(const float (&vin)[K], double (&out)[K], float2* part,
                                                 unsigned int* count, int* err, unsigned long long budget_ns,
                                                 float* sh) {
  constexpr int NW = NT / 32;
  __shared__ int s_ok;
  __shared__ double s_tot[K];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  FF f[K];
#pragma unroll
  for (int q = 0; q < K; ++q) f[q] = warp_sum_ff(FF{vin[q], 0.f});
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      sh[2 * (q * NW + w)] = f[q].hi;
      sh[2 * (q * NW + w) + 1] = f[q].lo;
    }
  }
  __syncthreads();
  if (w == 0) {
    const int nb = (int)gridDim.x;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      FF t = lane < NW ? FF{sh[2 * (q * NW + lane)], sh[2 * (q * NW + lane) + 1]} : FF{0.f, 0.f};
      t = warp_sum_ff(t);
      if (lane == 0) __stcg(part + (size_t)q * nb + blockIdx.x, make_float2(t.hi, t.lo));
    }
    int ok = 1;
    if (lane == 0) {
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
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) {
      FF t[K];
#pragma unroll
      for (int q = 0; q < K; ++q) t[q] = FF{0.f, 0.f};
      for (int b = lane; b < nb; b += 32) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
          const float2 pv = __ldcg(part + (size_t)q * nb + b);
          t[q] = ff_add(t[q], FF{pv.x, pv.y});
        }
      }
#pragma unroll
      for (int q = 0; q < K; ++q) {
        t[q] = warp_sum_ff(t[q]);
        if (lane == 0) s_tot[q] = ff_to(t[q]);
      }
    }
    if (lane == 0) s_ok = ok;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) out[q] = s_tot[q];
  return s_ok != 0;
}

}  // namespace ibsn
