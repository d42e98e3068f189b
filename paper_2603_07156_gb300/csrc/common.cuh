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
};
template <>
struct Acc<double> {
  double s;
  __device__ __forceinline__ void zero() { s = 0.0; }
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for a cooperatively launched grid (all blocks co-resident).
// The wait is bounded: after `budget_ns` of waiting (globaltimer) the block
// records kDevTimeout in *err and returns false; once *err is set every later
// call returns false at once, so all blocks leave the kernel.
__device__ __forceinline__ bool grid_barrier(unsigned int* count, unsigned int* gen, int* err,
                                             unsigned long long budget_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* vgen = gen;
    volatile int* verr = err;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int prev = atomicAdd(count, 1u);
    if (prev == gridDim.x - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      unsigned int spins = 0;
      unsigned long long t0 = 0;
      while (*vgen == g) {
        if (*verr != 0) { ok = 0; break; }
        if ((++spins & 255u) == 0) {
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
    __threadfence();
    if (*verr != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace ibsn
