// Dense m x n row passes of IBSN.  Each block owns a contiguous range of rows
// and streams them once; one row at a time is held in registers, spread over
// the block's TG threads (thread t owns columns (s*TG + t)*V + e, s < CH,
// e < V).  Row reductions are block reductions; column sums are accumulated
// per thread in registers (float: Kahan) or in shared memory (double) and
// written once per block as a partial, reduced deterministically afterwards.
//
// The exponent of every pass is x_ij = K_ij + d_j, where K is the anchored
// matrix built by k_reanchor and d_j = (gamma_j - gamma^anc_j)/eta, so that
// P^k(gamma)_ij = exp(x_ij - lse_i) (Eq. 6).
#pragma once

#include <type_traits>

#include "common.cuh"
#include "ffmath.cuh"
#include "internal.h"

namespace ibsn {

template <typename T>
struct DenseArgs {
  const T* K;
  int64_t ldk;
  int m, n, rows_per_block, istar;
  const T* dv;         // d_j, padded with 0 to ldk
  const T* v1;         // per-column input 1 (variant specific)
  const T* v2;         // per-column input 2
  const T* v3;         // per-column input 3
  const T* v4;         // per-column input 4
  const double* a;     // m
  const T* aT;         // m, a in the pass precision
  double* rowout;      // m, variant specific (lse, e_r, zeta)
  double* rowout2;     // m
  double* colpart;     // gridDim.x x ldk
  double* rowpart;     // gridDim.x x kRowParts
  double s1, s2;       // scalars (variant specific)
  // sparsify
  int32_t* pool_col;
  T* pool_val;
  int64_t* row_start;
  int32_t* row_len;
  int32_t* blkcnt;     // gridDim.x x ldk
  T* prow;             // row i* of P (dense, n)
  unsigned long long* pool_top;
  int64_t cap;
  int* err;
  // cost access (certify / reanchor)
  CostRef cost;
  const double* gam;   // gamma (certify)
  const double* wv;    // reanchor: log b_j + (Gamma_j + gamma_j)/eta
  double lam;          // reanchor: (k+1)/eta
  T* Kout;             // reanchor output
  double* plan_out;    // certify / export: m x n float64, nullable
  // float-float passes: K = K (hi plane) + Klo (lo plane); float64 copies of
  // the per-column inputs for the entries evaluated in float64
  const float* Klo;
  float* Klo_out;      // reanchor: lo plane output (nullable)
  const double* dv64;
  const double* v1d;
  const double* v2d;
  const double* v3d;
  const float* gam32;      // certify: float copy of gamma
  const float* v3lo;       // certify: v3d - v3 (float-float lo part)
  const double* bounds;    // certify: [0] max |C|, [1] max |gamma| (device)
  const double* zeta_in;   // certify, grid cost: the c-transform zeta_i, computed beforehand
  // no stored anchored matrix: every pass rebuilds K_ij from the cost, the
  // anchor-time w = (wvh, wvl), lam = (lamh, laml) and the row shifts rowMa,
  // with the arithmetic of the anchor pass (bitwise the same values)
  int recompute;
  int rc_lo;               // the anchor is the polish's (two planes): hi as it stores it, lo used
  float* rowMa;            // m anchor row shifts (written by the anchor pass, read by the others)
  // float-float anchor build: w_j as hi + lo floats, lam as hi + lo floats
  const float* wvh;
  const float* wvl;
  float lamh, laml;
  double* scal;            // slot S_DEVERR records a timed-out wait
  int stages;              // float row stream: row buffers in flight (1 or 2; 0 reads as 1)
  // float-float passes: per-row results for the row kernels, a_i - fl32(a_i)
  double* rowS0;
  double* rowS1;
  double* rowM;
  const float* alo;
  double* rowbuf;          // certificate: 6 planes of m per-row results
  // float-float lo parts of the per-column inputs: d, v1, v2, gamma
  const float* dvlo;
  const float* v1lo;
  const float* v2lo;
  const float* gamlo;
};

template <typename T, int TG, int CH>
struct Tile {
  static constexpr int V = VecT<T>::N;
  T x[CH][V];

  __device__ __forceinline__ static int64_t col(int s) {
    return (int64_t)(s * TG + (int)threadIdx.x) * V;
  }

  // x = K_i + d  (padding columns of K hold -inf)
  __device__ __forceinline__ void load(const T* __restrict__ row, const T* __restrict__ dv, int64_t ldk) {
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = col(s);
      if (c < ldk) {
        T kv[V], d[V];
        load_vec_stream(row + c, kv);
        load_vec(dv + c, d);
#pragma unroll
        for (int e = 0; e < V; ++e) x[s][e] = kv[e] + d[e];
      } else {
#pragma unroll
        for (int e = 0; e < V; ++e) x[s][e] = neg_inf<T>();
      }
    }
  }

  // x = K_i + d with the row of K in shared memory (float passes)
  __device__ __forceinline__ void load_smem(const T* row, const T* __restrict__ dv, int64_t ldk) {
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = col(s);
      if (c < ldk) {
        T kv[V], d[V];
        load_vec(row + c, kv);
        load_vec(dv + c, d);
#pragma unroll
        for (int e = 0; e < V; ++e) x[s][e] = kv[e] + d[e];
      } else {
#pragma unroll
        for (int e = 0; e < V; ++e) x[s][e] = neg_inf<T>();
      }
    }
  }

  __device__ __forceinline__ T local_max() const {
    T mx = neg_inf<T>();
#pragma unroll
    for (int s = 0; s < CH; ++s)
#pragma unroll
      for (int e = 0; e < V; ++e) mx = fmax(mx, x[s][e]);
    return mx;
  }

  // x <- exp(x - mx), returns the thread's sum
  __device__ __forceinline__ T exp_shift(T mx) {
    T ps = T(0);
#pragma unroll
    for (int s = 0; s < CH; ++s)
#pragma unroll
      for (int e = 0; e < V; ++e) {
        x[s][e] = exp_t(x[s][e] - mx);
        ps += x[s][e];
      }
    return ps;
  }
};

// Per-thread column accumulators.  float: registers with Kahan compensation;
// double: shared memory slots owned by the thread (no sharing, no atomics).
template <typename T, int TG, int CH>
struct ColAcc {
  static constexpr int V = VecT<T>::N;
  static constexpr bool kSmem = std::is_same<T, double>::value;
  Acc<float> r[kSmem ? 1 : CH][kSmem ? 1 : V];
  double* sm;
  int64_t ld;

  __device__ __forceinline__ void init(double* smem, int64_t ldk) {
    ld = ldk;
    if constexpr (kSmem) {
      sm = smem;
#pragma unroll
      for (int s = 0; s < CH; ++s) {
        const int64_t c = Tile<T, TG, CH>::col(s);
        if (c < ldk)
#pragma unroll
          for (int e = 0; e < V; ++e) sm[c + e] = 0.0;
      }
    } else {
#pragma unroll
      for (int s = 0; s < CH; ++s)
#pragma unroll
        for (int e = 0; e < V; ++e) r[s][e].zero();
    }
  }
  // columns past the padded row (tile wider than ldk) are not stored
  __device__ __forceinline__ void add(int s, int e, T v) {
    if constexpr (kSmem) {
      const int64_t c = Tile<T, TG, CH>::col(s) + e;
      if (c < ld) sm[c] += v;
    } else {
      r[s][e].add(v);
    }
  }
  __device__ __forceinline__ void add_prod(int s, int e, T w, T v) {
    if constexpr (kSmem) {
      const int64_t c = Tile<T, TG, CH>::col(s) + e;
      if (c < ld) sm[c] = fma(w, v, sm[c]);
    } else {
      r[s][e].add_prod(w, v);
    }
  }
  // float64 partials (float64 passes) or float-float pairs {s, -c} (float
  // passes: no float64 conversion here; the column finish adds the pairs)
  __device__ __forceinline__ void flush(double* __restrict__ out, int64_t ldk) {
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = Tile<T, TG, CH>::col(s);
      if (c < ldk) {
#pragma unroll
        for (int e = 0; e < V; ++e) {
          if constexpr (kSmem) {
            out[c + e] = sm[c + e];
          } else {
            reinterpret_cast<float2*>(out)[c + e] = make_float2(r[s][e].s, -r[s][e].c);
          }
        }
      }
    }
  }
};

__device__ __forceinline__ void row_range(int m, int rpb, int& r0, int& r1) {
  r0 = blockIdx.x * rpb;
  r1 = min(m, r0 + rpb);
}

// ---------------------------------------------------------------------------
// Row stream.  Float passes receive the rows of K in shared memory by a bulk
// asynchronous copy (TMA), issued by one thread and completed on an mbarrier
// with the transaction byte count; the copy of row i+1 is issued as soon as
// every thread holds row i in registers, so it runs under the reductions and
// arithmetic of row i.  Waits are bounded in time: a wait that runs out
// records scal[S_DEVERR] and the pass returns.  Float64 passes load rows from
// global memory directly (their shared memory holds the column accumulator).
// Dynamic shared memory of a float pass: [row buffer, ldk floats][column
// accumulator of a float-float pass, ldk doubles].
// ---------------------------------------------------------------------------
constexpr unsigned long long kRowWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait_parity(uint32_t bar, uint32_t parity) {
  uint32_t spins = 0;
  unsigned long long t0 = 0;
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((++spins & 255u) == 0) {
      const unsigned long long now = globaltimer_ns();
      if (t0 == 0) {
        t0 = now;
      } else if (now - t0 > kRowWaitNs) {
        return false;
      }
    }
  }
}

constexpr int kMaxRowStages = 3;

template <typename T>
struct RowStream {
  float* buf = nullptr;
  uint32_t bar0 = 0;       // shared address of the first stage's mbarrier (8 bytes apart)
  uint32_t parity = 0;     // bit s: phase parity stage s waits for next
  int ns = 1;              // stages: row copies kept in flight
  int base = 0;            // first row of the block

  __device__ __forceinline__ void issue(const DenseArgs<T>& A, int row, int stage) {  // one thread
    const uint32_t bytes = (uint32_t)(A.ldk * (int64_t)sizeof(float));
    const float* src = reinterpret_cast<const float*>(A.K) + (int64_t)row * A.ldk;
    const uint32_t bar = bar0 + 8u * (uint32_t)stage;
    // the block's reads of this stage's previous row (generic proxy) precede this write (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(buf + (int64_t)stage * A.ldk)), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
  }

  // set up the barriers and start the copies of the block's first rows;
  // mbar points to kMaxRowStages barriers, the dynamic shared memory holds
  // A.stages row buffers of ldk floats
  __device__ __forceinline__ void start(const DenseArgs<T>& A, double* dyn, unsigned long long* mbar, int r0, int r1) {
    if constexpr (std::is_same<T, float>::value) {
      if (A.recompute) return;  // rows are rebuilt from the cost: nothing to copy
      buf = reinterpret_cast<float*>(dyn);
      bar0 = smem_u32(mbar);
      ns = A.stages < 1 ? 1 : (A.stages > kMaxRowStages ? kMaxRowStages : A.stages);
      base = r0;
      if (threadIdx.x == 0) {
        for (int q = 0; q < ns; ++q)
          asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8u * (uint32_t)q) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int q = 0; q < ns && r0 + q < r1; ++q) issue(A, r0 + q, q);
      }
      __syncthreads();
    }
  }

  // row i into the tile; starts the copy of row i + ns into the freed stage.
  // False: a wait ran out (recorded); thread 0 then waits, again bounded, for
  // the block's other copy in flight, and every thread returns false together.
  template <int TG, int CH>
  __device__ __forceinline__ bool row(Tile<T, TG, CH>& t, const DenseArgs<T>& A, int i, int r1) {
    if constexpr (std::is_same<T, float>::value) {
      if (A.recompute) {
        rebuild_row(t, A, i);
        return true;
      }
      const int q = (i - base) % ns;
      const bool ok = mbar_wait_parity(bar0 + 8u * (uint32_t)q, (parity >> q) & 1u);
      parity ^= 1u << q;
      if (ok) t.load_smem(buf + (int64_t)q * A.ldk, A.dv, A.ldk);
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
          if (A.scal != nullptr) A.scal[S_DEVERR] = 1.0;
          // the copies of rows i+1 .. i+ns-1 may still be in flight: wait for them (bounded)
          for (int k = 1; k < ns && i + k < r1; ++k) {
            const int q2 = (i + k - base) % ns;
            mbar_wait_parity(bar0 + 8u * (uint32_t)q2, (parity >> q2) & 1u);
          }
        }
        __syncthreads();
        return false;
      }
      if (threadIdx.x == 0 && i + ns < r1) issue(A, i + ns, q);
    } else {
      t.load(A.K + (int64_t)i * A.ldk, A.dv, A.ldk);
    }
    return true;
  }
};

// Shift subtracted from a row's exponents before exp.  Float32 passes use 0:
// the anchored K is <= 0 with row maximum 0, the potential offsets d stay
// within [-16, 16] (the anchor is rebuilt beyond that) and an Armijo trial
// adds at most 60, so exp of every row maximum lies in [e^-76, e^76] and
// neither overflows a float row sum nor underflows the whole row.  Float64
// passes reduce the row maximum.
template <typename T, int TG, int CH>
__device__ __forceinline__ T row_shift(const Tile<T, TG, CH>& t, T* sht) {
  if constexpr (std::is_same<T, float>::value) {
    return 0.f;
  } else {
    return block_max<TG>(t.local_max(), sht);
  }
}

// Block sum of K per-thread sums: float32 in float32 passes (their accuracy is
// float32 anyway), float-float in float64 passes.  `shf` holds 8 * TG/32 floats.
template <typename T, int TG, int K>
__device__ __forceinline__ void row_sum(T (&v)[K], float* shf) {
  if constexpr (std::is_same<T, float>::value) {
    block_sum_f<TG, K>(v, shf);
  } else {
    block_sum_ff<TG, K>(v, shf);
  }
}

// ---------------------------------------------------------------------------
// Plan pass (Eqs. 6-7): lse_i, c_j = sum_i a_i P_ij, sum_i a_i lse_i.
// rowout = lse (nullable).
// ---------------------------------------------------------------------------
template <typename T, int TG, int CH>
__global__ void __launch_bounds__(TG) k_plan(DenseArgs<T> A) {
  extern __shared__ __align__(128) double dyn_sm[];
  __shared__ unsigned long long s_mbar[kMaxRowStages];
  __shared__ float shf[8 * (TG / 32)];
  __shared__ T sht[TG / 32];
  constexpr int V = VecT<T>::N;
  ColAcc<T, TG, CH> acc;
  acc.init(dyn_sm, A.ldk);
  int r0, r1;
  row_range(A.m, A.rows_per_block, r0, r1);
  RowStream<T> rs;
  rs.start(A, dyn_sm, s_mbar, r0, r1);
  T lpart = T(0);
  Tile<T, TG, CH> t;
  for (int i = r0; i < r1; ++i) {
    if (!rs.row(t, A, i, r1)) return;
    const T mx = row_shift<T, TG, CH>(t, sht);
    T S[1] = {t.exp_shift(mx)};
    row_sum<T, TG, 1>(S, shf);
    const T ai = A.aT[i];
    const T lse = mx + log(S[0]);
    lpart += ai * lse;
    if (A.rowout != nullptr && threadIdx.x == 0) A.rowout[i] = (double)lse;
    const T w = ai / S[0];
#pragma unroll
    for (int s = 0; s < CH; ++s)
#pragma unroll
      for (int e = 0; e < V; ++e) acc.add_prod(s, e, w, t.x[s][e]);
  }
  acc.flush(A.colpart + (int64_t)blockIdx.x * A.ldk, A.ldk);
  if (threadIdx.x == 0) A.rowpart[blockIdx.x * kRowParts + 0] = (double)lpart;
}

// ---------------------------------------------------------------------------
// Armijo trial (Alg. 2) in difference form.  v1 = em_j = expm1(t Delta_j/eta).
// Per row s_i = sum_j P_ij em_j; the new plan has row sums exp(lse_i)(1+s_i)
// and column sums c'_j = sum_i a_i P_ij (1 + em_j)/(1 + s_i).
// rowpart[0] = sum_i a_i psi(s_i), psi(s) = log1p(s) - s (second order),
// rowpart[1] = sum_i a_i log1p(s_i).  rowout = new lse (nullable).
// ---------------------------------------------------------------------------
// psi_log1p_minus: common.cuh

template <typename T, int TG, int CH>
__global__ void __launch_bounds__(TG) k_armijo(DenseArgs<T> A) {
  extern __shared__ __align__(128) double dyn_sm[];
  __shared__ unsigned long long s_mbar[kMaxRowStages];
  __shared__ float shf[8 * (TG / 32)];
  __shared__ T sht[TG / 32];
  constexpr int V = VecT<T>::N;
  ColAcc<T, TG, CH> acc;
  acc.init(dyn_sm, A.ldk);
  int r0, r1;
  row_range(A.m, A.rows_per_block, r0, r1);
  RowStream<T> rs;
  rs.start(A, dyn_sm, s_mbar, r0, r1);
  T ppsi = T(0), plog = T(0);
  Tile<T, TG, CH> t;
  for (int i = r0; i < r1; ++i) {
    if (!rs.row(t, A, i, r1)) return;
    const T mx = row_shift<T, TG, CH>(t, sht);
    T S[2] = {T(0), T(0)};
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = Tile<T, TG, CH>::col(s);
      T em[V];
      if (c < A.ldk) {
        load_vec(A.v1 + c, em);
      } else {
#pragma unroll
        for (int e = 0; e < V; ++e) em[e] = T(0);
      }
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const T ev = exp_t(t.x[s][e] - mx);
        t.x[s][e] = ev;
        S[0] += ev;
        S[1] += ev * em[e];
      }
    }
    row_sum<T, TG, 2>(S, shf);
    const T si = S[1] / S[0];
    const T ai = A.aT[i];
    const T l1p = log1p(si);
    ppsi += ai * psi_log1p_minus(si);
    plog += ai * l1p;
    if (A.rowout != nullptr && threadIdx.x == 0) A.rowout[i] = (double)(mx + log(S[0]) + l1p);
    const T w = ai / (S[0] * (T(1) + si));
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = Tile<T, TG, CH>::col(s);
      T em[V];
      if (c < A.ldk) {
        load_vec(A.v1 + c, em);
      } else {
#pragma unroll
        for (int e = 0; e < V; ++e) em[e] = T(0);
      }
#pragma unroll
      for (int e = 0; e < V; ++e) acc.add_prod(s, e, w, fma(t.x[s][e], em[e], t.x[s][e]));
    }
  }
  acc.flush(A.colpart + (int64_t)blockIdx.x * A.ldk, A.ldk);
  if (threadIdx.x == 0) {
    A.rowpart[blockIdx.x * kRowParts + 0] = (double)ppsi;
    A.rowpart[blockIdx.x * kRowParts + 1] = (double)plog;
  }
}

// ---------------------------------------------------------------------------
// Inexact stopping test (Eq. 8) with the rounding of Alg. 3.
// v1 = omega_j = 1 - y_j, v2 = e_c,j, v3 = log e_c,j, v4 = (1-omega) log(1-omega)
// + omega; S = ||e_c||_1 from scal[S_ECSUM].  e_r,i = a_i sum_j P_ij omega_j (z = 1: X = diag(a) P
// has row sums a).  D_phi = sum_ij T_ij, T = Xhat log(Xhat/X) - Xhat + X >= 0 with
// Xhat = X (1 - omega_j) + e_r,i e_c,j / S.  A column has omega_j > 0 or e_c,j > 0,
// never both, so per entry (X = e^LX, extra = e_r,i e_c,j / S, L = log(extra/X)):
//   e_c,j = 0:          T = X v4_j
//   e_r,i = 0:          T = 0
//   X <= tau extra:     T = extra (L - 1) + X (L + 1)   (error <= X tau / 2)
//   otherwise:          T = X h(extra / X), h(u) = (1+u) log1p(u) - u
// The second case, which holds for almost every entry off the plan's support,
// needs no transcendental: L comes from the exponent and the logs of the row
// and column factors.  rowout = e_r (nullable).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T h_of_1pu(T u) {
  // (1+u) log1p(u) - u; series sum_{k>=2} (-1)^k u^k / (k(k-1)) for small |u|
  if (fabs(u) < T(1e-2)) {
    const T u2 = u * u;
    return u2 * (T(0.5) + u * (T(-1.0 / 6.0) + u * (T(1.0 / 12.0) + u * (T(-1.0 / 20.0) + u * T(1.0 / 30.0)))));
  }
  if (u <= T(-1)) return T(1);
  return (T(1) + u) * log1p(u) - u;
}

template <typename T>
struct StopTau;
template <>
struct StopTau<float> {
  static constexpr float v = 0x1p-12f;
};
template <>
struct StopTau<double> {
  static constexpr double v = 0x1p-24;
};

template <typename T, int TG, int CH>
__global__ void __launch_bounds__(TG) k_stop(DenseArgs<T> A) {
  extern __shared__ __align__(128) double dyn_sm[];
  __shared__ unsigned long long s_mbar[kMaxRowStages];
  __shared__ float shf[8 * (TG / 32)];
  __shared__ T sht[TG / 32];
  constexpr int V = VecT<T>::N;
  constexpr T tau = StopTau<T>::v;
  int r0, r1;
  row_range(A.m, A.rows_per_block, r0, r1);
  RowStream<T> rs;
  rs.start(A, dyn_sm, s_mbar, r0, r1);
  const double S_ec = A.scal[S_ECSUM];  // ||e_c||_1, formed on the device with the gradient
  const T invS = (T)(S_ec > 0.0 ? 1.0 / S_ec : 0.0);
  T dpart = T(0);
  Tile<T, TG, CH> t;
  for (int i = r0; i < r1; ++i) {
    if (!rs.row(t, A, i, r1)) return;  // t.x keeps the exponents x_ij
    const T mx = row_shift<T, TG, CH>(t, sht);
    // row sum and sum_j e_ij omega_j in one reduction
    T R[2] = {T(0), T(0)};
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = Tile<T, TG, CH>::col(s);
      T om[V];
      if (c < A.ldk) {
        load_vec(A.v1 + c, om);
      } else {
#pragma unroll
        for (int e = 0; e < V; ++e) om[e] = T(0);
      }
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const T ev = exp_t(t.x[s][e] - mx);
        R[0] += ev;
        R[1] += ev * om[e];
      }
    }
    row_sum<T, TG, 2>(R, shf);
    const T invS0 = T(1) / R[0];
    const T ai = A.aT[i];
    const T er = ai * R[1] * invS0;
    if (A.rowout != nullptr && threadIdx.x == 0) A.rowout[i] = (double)er;
    const T logai_m = log(ai) - mx - log(R[0]);  // log X_ij = x_ij + this
    const T erS = er * invS;
    const T lerS = log(erS);                     // log of the row factor of extra
    const T aiS = ai * invS0;
    T D[1] = {T(0)};
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = Tile<T, TG, CH>::col(s);
      if (c < A.ldk) {
        T ec[V], lec[V], hom[V];
        load_vec(A.v2 + c, ec);
        load_vec(A.v3 + c, lec);
        load_vec(A.v4 + c, hom);
#pragma unroll
        for (int e = 0; e < V; ++e) {
          if (c + e >= A.n) continue;
          const T X = aiS * exp_t(t.x[s][e] - mx);
          const T extra = erS * ec[e];
          if (ec[e] <= T(0)) {
            D[0] += X * hom[e];
          } else if (!(extra > T(0))) {
            // e_r,i = 0: Xhat = X on this column, T = 0
          } else if (X <= tau * extra) {
            const T L = (lerS + lec[e]) - (t.x[s][e] + logai_m);
            D[0] += extra * (L - T(1)) + X * (L + T(1));
          } else {
            D[0] += X * h_of_1pu(extra / X);
          }
        }
      }
    }
    row_sum<T, TG, 1>(D, shf);
    dpart += D[0];
  }
  if (threadIdx.x == 0) A.rowpart[blockIdx.x * kRowParts + 0] = (double)dpart;
}

// ---------------------------------------------------------------------------
// Hessian sparsification (Alg. 1): keep P_ij >= rho (s1), renormalise the kept
// row to 1, write it to the CSR pool; row i* is written dense to prow.
// blkcnt[b][j] counts kept entries of block b in column j (for the CSC build).
// ---------------------------------------------------------------------------
template <typename T, int TG, int CH>
__global__ void __launch_bounds__(TG) k_sparsify(DenseArgs<T> A) {
  extern __shared__ __align__(128) double dyn_sm[];
  __shared__ unsigned long long s_mbar[kMaxRowStages];
  __shared__ float shf[8 * (TG / 32)];
  __shared__ T sht[TG / 32];
  __shared__ int shi[TG / 32];
  __shared__ unsigned long long s_base;
  constexpr int V = VecT<T>::N;
  int cnt[CH][V];
#pragma unroll
  for (int s = 0; s < CH; ++s)
#pragma unroll
    for (int e = 0; e < V; ++e) cnt[s][e] = 0;
  int r0, r1;
  row_range(A.m, A.rows_per_block, r0, r1);
  RowStream<T> rs;
  rs.start(A, dyn_sm, s_mbar, r0, r1);
  const T rho = (T)A.s1;
  Tile<T, TG, CH> t;
  for (int i = r0; i < r1; ++i) {
    if (!rs.row(t, A, i, r1)) return;
    const T mx = row_shift<T, TG, CH>(t, sht);
    T S[1] = {t.exp_shift(mx)};
    row_sum<T, TG, 1>(S, shf);
    const T invS0 = T(1) / S[0];
    if (i == A.istar) {
#pragma unroll
      for (int s = 0; s < CH; ++s) {
        const int64_t c = Tile<T, TG, CH>::col(s);
#pragma unroll
        for (int e = 0; e < V; ++e)
          if (c + e < A.n) A.prow[c + e] = t.x[s][e] * invS0;
      }
      if (threadIdx.x == 0) {
        A.row_len[i] = 0;
        A.row_start[i] = 0;
      }
      continue;
    }
    int kc = 0;
    T ks = T(0);
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = Tile<T, TG, CH>::col(s);
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const T P = t.x[s][e] * invS0;
        const bool keep = (c + e < A.n) && (P >= rho);
        t.x[s][e] = keep ? P : T(-1);
        if (keep) {
          ++kc;
          ks += P;
        }
      }
    }
    T KS[1] = {ks};
    row_sum<T, TG, 1>(KS, shf);
    int total = 0;
    const int off = block_exclusive_scan<TG>(kc, shi, &total);
    if (threadIdx.x == 0) {
      const unsigned long long base = atomicAdd(A.pool_top, (unsigned long long)total);
      s_base = base;
      if ((long long)(base + total) > A.cap) atomicExch(A.err, (int)kDevCapacity);
      A.row_start[i] = (int64_t)base;
      A.row_len[i] = ((long long)(base + total) > A.cap) ? 0 : total;
    }
    __syncthreads();
    const unsigned long long base = s_base;
    if ((long long)(base + total) > A.cap) continue;
    const T inv_ks = T(1) / KS[0];
    int64_t pos = (int64_t)base + off;
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = Tile<T, TG, CH>::col(s);
#pragma unroll
      for (int e = 0; e < V; ++e) {
        if (t.x[s][e] >= T(0)) {
          A.pool_col[pos] = (int32_t)(c + e);
          A.pool_val[pos] = t.x[s][e] * inv_ks;
          ++pos;
          cnt[s][e] += 1;
        }
      }
    }
  }
#pragma unroll
  for (int s = 0; s < CH; ++s) {
    const int64_t c = Tile<T, TG, CH>::col(s);
    if (c < A.ldk)
#pragma unroll
      for (int e = 0; e < V; ++e) A.blkcnt[(int64_t)blockIdx.x * A.ldk + c + e] = cnt[s][e];
  }
}

// ---------------------------------------------------------------------------
// Cost entry C_ij in float64 for the kinds of ibsn_cost_kind.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double cost_at(const CostRef& c, int i, int64_t j) {
  if (c.kind == 0) return __ldg(static_cast<const double*>(c.C) + (int64_t)i * c.ldc + j);
  if (c.kind == 1) return (double)__ldg(static_cast<const float*>(c.C) + (int64_t)i * c.ldc + j);
  if (c.kind == 3) {
    const double* xi = c.px + (int64_t)i * c.dim;
    const double* yj = c.py + j * c.dim;
    double q = 0.0;
    for (int k = 0; k < c.dim; ++k) {
      const double t = __ldg(xi + k) - __ldg(yj + k);
      q = fma(t, t, q);
    }
    return c.scale * q;
  }
  int ri, ci, rj, cj;
  if (c.rc != nullptr) {
    const int pi = __ldg(c.rc + i), pj = __ldg(c.rc + j);
    ri = pi & 0xffff, ci = pi >> 16, rj = pj & 0xffff, cj = pj >> 16;
  } else {
    ri = i / c.gw, ci = i - ri * c.gw, rj = (int)j / c.gw, cj = (int)j - rj * c.gw;
  }
  const int dr = ri - rj, dc = ci - cj;
  return c.scale * (double)(dr * dr + dc * dc);
}

// ---------------------------------------------------------------------------
// Certificate (App. A rounding, App. C.1 dual) at X = diag(a) P:
//   v1 = y_j, v2 = omega_j, v3 = e_c,j / S.
//   e_r,i = a_i sum_j P_ij omega_j,  Xhat_ij = a_i P_ij y_j + e_r,i e_c,j / S
//   rowpart: [0] sum_ij C_ij Xhat_ij, [1] sum_i a_i zeta_i,
//            [2] sum_i |a_i (sum_j P_ij - 1)|, [3] sum_i e_r,i,
//            [4] <X, C - zeta 1^T - 1 gamma^T>, [5] sum C_ij^2,
//            [6] sum_i (a_i (sum_j P_ij - 1))^2
//   colpart: sum_i a_i P_ij y_j;  rowout = zeta (nullable), plan_out nullable.
// ---------------------------------------------------------------------------
template <typename T, int TG, int CH>
__global__ void __launch_bounds__(TG) k_certify(DenseArgs<T> A) {
  extern __shared__ __align__(128) double dyn_sm[];
  __shared__ unsigned long long s_mbar[kMaxRowStages];
  __shared__ double shd[6 * (TG / 32)];
  __shared__ float shf[8 * (TG / 32)];
  __shared__ T sht[TG / 32];
  constexpr int V = VecT<T>::N;
  ColAcc<T, TG, CH> acc;
  acc.init(dyn_sm, A.ldk);
  int r0, r1;
  row_range(A.m, A.rows_per_block, r0, r1);
  RowStream<T> rs;
  rs.start(A, dyn_sm, s_mbar, r0, r1);
  double part[7] = {0, 0, 0, 0, 0, 0, 0};
  Tile<T, TG, CH> t;
  for (int i = r0; i < r1; ++i) {
    if (!rs.row(t, A, i, r1)) return;
    const T mx = row_shift<T, TG, CH>(t, sht);
    double S[1] = {(double)t.exp_shift(mx)};
    block_sum_ff<TG, 1>(S, shf);
    const double invS0 = 1.0 / S[0];
    const double ai = A.a[i];
    // sweep 1: P row sum, sum P omega, zeta_i = min_j C_ij - gamma_j, sum C^2
    double psum = 0.0, pom = 0.0, zmin = kInf, c2 = 0.0;
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = Tile<T, TG, CH>::col(s);
      if (c < A.ldk) {
        T om[V];
        load_vec(A.v2 + c, om);
#pragma unroll
        for (int e = 0; e < V; ++e) {
          if (c + e >= A.n) continue;
          const double P = (double)t.x[s][e] * invS0;
          psum += P;
          pom += P * (double)om[e];
          const double C = cost_at(A.cost, i, c + e);
          zmin = fmin(zmin, C - A.gam[c + e]);
          c2 += C * C;
        }
      }
    }
    double R[3] = {psum, pom, c2};
    block_sum_ff<TG, 3>(R, shf);
    const double zeta = -block_max<TG>(-zmin, reinterpret_cast<double*>(shd + 3 * (TG / 32)));
    const double er = ai * R[1];
    // sweep 2: primal and complementarity
    double pr = 0.0, cu = 0.0;
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = Tile<T, TG, CH>::col(s);
      if (c < A.ldk) {
        T y[V], ecs[V];
        load_vec(A.v1 + c, y);
        load_vec(A.v3 + c, ecs);
#pragma unroll
        for (int e = 0; e < V; ++e) {
          if (c + e >= A.n) continue;
          const double P = (double)t.x[s][e] * invS0;
          const double C = cost_at(A.cost, i, c + e);
          const double F = ai * P * (double)y[e];
          const double xh = F + er * (double)ecs[e];
          pr += C * xh;
          cu += ai * P * (C - zeta - A.gam[c + e]);
          acc.add(s, e, (T)F);
          if (A.plan_out != nullptr) A.plan_out[(int64_t)i * A.n + c + e] = xh;
        }
      }
    }
    double Q[2] = {pr, cu};
    block_sum_ff<TG, 2>(Q, shf);
    const double rv = ai * (R[0] - 1.0);
    part[0] += Q[0];
    part[1] += ai * zeta;
    part[2] += fabs(rv);
    part[3] += er;
    part[4] += Q[1];
    part[5] += R[2];
    part[6] += rv * rv;
    if (threadIdx.x == 0) {
      if (A.rowout != nullptr) A.rowout[i] = zeta;
      if (A.rowout2 != nullptr) A.rowout2[i] = er;
    }
  }
  acc.flush(A.colpart + (int64_t)blockIdx.x * A.ldk, A.ldk);
  if (threadIdx.x == 0)
    for (int q = 0; q < 7; ++q) A.rowpart[blockIdx.x * kRowParts + q] = part[q];
}

// ---------------------------------------------------------------------------
// Anchor build (outer update, Alg. 2): e_ij = w_j - lam C_ij in float64 with
// w_j = log b_j + (Gamma_j + gamma_j)/eta, lam = (k+1)/eta;
// K_ij = e_ij - max_l e_il, stored as T; padding columns get -inf.
// rowout = row maxima (nullable).
// ---------------------------------------------------------------------------
template <typename T, int TG, int CH>
__global__ void __launch_bounds__(TG) k_reanchor(DenseArgs<T> A) {
  __shared__ double shd[TG / 32];
  constexpr int V = VecT<T>::N;
  int r0, r1;
  row_range(A.m, A.rows_per_block, r0, r1);
  for (int i = r0; i < r1; ++i) {
    double ev[CH][V];
    double mx = -kInf;
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = Tile<T, TG, CH>::col(s);
#pragma unroll
      for (int e = 0; e < V; ++e) {
        if (c + e < A.n) {
          ev[s][e] = A.wv[c + e] - A.lam * cost_at(A.cost, i, c + e);
          mx = fmax(mx, ev[s][e]);
        } else {
          ev[s][e] = -kInf;
        }
      }
    }
    mx = block_max<TG>(mx, shd);
    if (A.rowout != nullptr && threadIdx.x == 0) A.rowout[i] = mx;
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = Tile<T, TG, CH>::col(s);
      if (c < A.ldk) {
        T kv[V];
#pragma unroll
        for (int e = 0; e < V; ++e) kv[e] = (c + e < A.n) ? (T)(ev[s][e] - mx) : neg_inf<T>();
        store_vec(A.Kout + (int64_t)i * A.ldk + c, kv);
        if constexpr (std::is_same<T, float>::value) {
          if (A.Klo_out != nullptr) {
            // float-float split: K = hi + lo with lo = fl32(K - hi)
            float lo[V];
#pragma unroll
            for (int e = 0; e < V; ++e)
              lo[e] = (c + e < A.n) ? (float)((ev[s][e] - mx) - (double)kv[e]) : 0.f;
            store_vec(A.Klo_out + (int64_t)i * A.ldk + c, lo);
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Plan export for checks: P_ij as float64 (m x n), same arithmetic as the passes.
// ---------------------------------------------------------------------------
template <typename T, int TG, int CH>
__global__ void __launch_bounds__(TG) k_export(DenseArgs<T> A) {
  extern __shared__ __align__(128) double dyn_sm[];
  __shared__ unsigned long long s_mbar[kMaxRowStages];
  __shared__ float shf[8 * (TG / 32)];
  __shared__ T sht[TG / 32];
  constexpr int V = VecT<T>::N;
  int r0, r1;
  row_range(A.m, A.rows_per_block, r0, r1);
  RowStream<T> rs;
  rs.start(A, dyn_sm, s_mbar, r0, r1);
  Tile<T, TG, CH> t;
  for (int i = r0; i < r1; ++i) {
    if (!rs.row(t, A, i, r1)) return;
    const T mx = row_shift<T, TG, CH>(t, sht);
    T S[1] = {t.exp_shift(mx)};
    row_sum<T, TG, 1>(S, shf);
    const T invS0 = T(1) / S[0];
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = Tile<T, TG, CH>::col(s);
#pragma unroll
      for (int e = 0; e < V; ++e)
        if (c + e < A.n) A.plan_out[(int64_t)i * A.n + c + e] = (double)(t.x[s][e] * invS0);
    }
  }
}


// ===========================================================================
// Float-float passes.  The anchored matrix is held as two float planes,
// K = Khi + Klo (Klo = fl32(K - Khi)).  A float32 evaluation of every entry
// selects the entries above 2^-64 of the row maximum; only those are evaluated
// in float64 from Khi + Klo + d, and only their Klo is read.  The others are
// dropped: each is below 2^-64 of its row's largest entry, so the row sums and
// the column sums sum_i a_i P_ij change by less than n 2^-64 < 1e-15 relative.
// ===========================================================================
constexpr float kFFKeep = 0x1p-64f;
constexpr float kFFLogKeep = -44.3614195558365f;  // log(2^-64)
__device__ __forceinline__ FF anchored_ff(const DenseArgs<float>& A, int i, int64_t j);

template <int TG, int CH>
struct FFRow {
  static constexpr int V = 4;
  // float64 exponent of entry (s, e) of row i relative to the shift M
  __device__ __forceinline__ static double x64(const DenseArgs<float>& A, int i, int64_t c, int e, double M) {
    if (A.recompute) {
      const FF k = anchored_ff(A, i, c + e);
      return ((double)k.hi + (double)k.lo) + A.dv64[c + e] - M;
    }
    const int64_t off = (int64_t)i * A.ldk + c + e;
    const double lo = A.Klo != nullptr ? (double)__ldg(A.Klo + off) : 0.0;  // no lo plane: float32 K
    return ((double)__ldg(A.K + off) + lo) + A.dv64[c + e] - M;
  }
};

// C_ij as an unevaluated float pair hi + lo with |hi + lo - C_ij| <= 2^-46 C_ij
// (exact for float costs; for grid costs C = scale q with the integer q exact in
// float and scale split as sh + sl).
__device__ __forceinline__ float2 cost_ff(const CostRef& c, int i, int64_t j, float sh, float sl) {
  if (c.kind == 1) return make_float2(__ldg(static_cast<const float*>(c.C) + (int64_t)i * c.ldc + j), 0.f);
  if (c.kind == 3) {
    // sum_k (x_ik - y_jk)^2 in float-float from the (hi, lo) coordinates:
    // each difference exactly as TwoSum(xh, -yh) + (xl - yl), its square by
    // TwoProduct, the sum and the final scale in float-float
    const float2* xi = c.xs + (int64_t)i * c.dim;
    const float2* yj = c.ys + j * c.dim;
    FF q{0.f, 0.f};
    for (int k = 0; k < c.dim; ++k) {
      const float2 xv = __ldg(xi + k), yv = __ldg(yj + k);
      const float dh = xv.x - yv.x;
      const float bv = dh - xv.x;
      const float err = (xv.x - (dh - bv)) + (-yv.x - bv);
      const FF d = ff_add(FF{dh, 0.f}, FF{err + (xv.y - yv.y), 0.f});
      const float p = d.hi * d.hi;
      const float pl = fmaf(d.hi, d.hi, -p) + 2.f * d.hi * d.lo;
      q = ff_add(q, FF{p, pl});
    }
    const float r = q.hi * sh;
    return make_float2(r, fmaf(q.hi, sh, -r) + fmaf(q.hi, sl, q.lo * sh));
  }
  if (c.kind == 0) {
    const double C = __ldg(static_cast<const double*>(c.C) + (int64_t)i * c.ldc + j);
    const float h = (float)C;
    return make_float2(h, (float)(C - (double)h));
  }
  int ri, ci, rj, cj;
  if (c.rc != nullptr) {
    const int pi = __ldg(c.rc + i), pj = __ldg(c.rc + j);
    ri = pi & 0xffff, ci = pi >> 16, rj = pj & 0xffff, cj = pj >> 16;
  } else {
    ri = i / c.gw, ci = i - ri * c.gw, rj = (int)j / c.gw, cj = (int)j - rj * c.gw;
  }
  const float q = (float)((ri - rj) * (ri - rj) + (ci - cj) * (ci - cj));
  const float p = q * sh;
  return make_float2(p, fmaf(q, sl, fmaf(q, sh, -p)));
}

// The cost accessors specialised on the cost kind (a template argument of the
// passes that read C for every entry, so each instantiation holds one kind's code).
template <int KIND>
__device__ __forceinline__ CostRef kind_ref(const CostRef& c) {
  CostRef r = c;
  r.kind = KIND;
  return r;
}

// s += x (float-float, TwoSum)
__device__ __forceinline__ void ff_acc(float& sh, float& sl, float x) {
  const float t = sh + x;
  const float bb = t - sh;
  sl += (sh - (t - bb)) + (x - bb);
  sh = t;
}

// Entries whose anchored exponent K exceeds -kFFLoBand can pass the filter of
// the float-float passes before the next anchor build: the filter keeps x - max
// above -44.4 (2^-64), the Armijo pass widens that by up to 2 * 30, and the
// offsets d_j move within [-16, 16] (the anchor is rebuilt beyond that).
constexpr float kFFLoBand = 144.f;

// Anchored exponent (hi, lo) of entry (i, j) exactly as k_reanchor_ff writes
// it (hi: the float plane; lo: the polish's lo plane, 0 outside the polish),
// for passes that rebuild it instead of reading the stored planes.
__device__ __forceinline__ FF anchored_ff(const DenseArgs<float>& A, int i, int64_t j) {
  if (j >= A.n) return FF{-__builtin_huge_valf(), 0.f};
  const float Mi = A.rowMa[i];
  const float csh = (float)A.cost.scale, csl = (float)(A.cost.scale - (double)csh);
  const float2 C = cost_ff(A.cost, i, j, csh, csl);
  const float p = A.lamh * C.x;
  const float pl = fmaf(A.lamh, C.x, -p) + fmaf(A.lamh, C.y, A.laml * C.x);
  const FF d = ff_add(FF{__ldg(A.wvh + j), __ldg(A.wvl + j)}, FF{-p, -pl});
  FF k = ff_add(FF{d.hi, d.lo}, FF{-Mi, 0.f});
  if (!A.rc_lo) return FF{k.hi, 0.f};
  if (k.hi > -kFFLoBand) {
    const double K64 = (A.wv[j] - A.lam * cost_at(A.cost, i, j)) - (double)Mi;
    k.hi = (float)K64;
    k.lo = (float)(K64 - (double)k.hi);
  }
  return k;
}

// A row of x = K + d rebuilt from the cost (recompute mode of the row stream).
template <int TG, int CH>
__device__ __forceinline__ void rebuild_row(Tile<float, TG, CH>& t, const DenseArgs<float>& A, int i) {
#pragma unroll
  for (int s = 0; s < CH; ++s) {
    const int64_t c = Tile<float, TG, CH>::col(s);
#pragma unroll
    for (int e = 0; e < 4; ++e)
      t.x[s][e] = c + e < A.ldk ? anchored_ff(A, i, c + e).hi + A.dv[c + e] : -__builtin_huge_valf();
  }
}

// Anchor build (float planes): E_ij = w_j - lam C_ij in float-float (error
// about 2^-46 |lam C_ij|, far below the float32 plane's rounding), row shift
// M_i = max_j hi(E_ij), K32 = fl32(E - M).  In the polish (Klo_out set) the
// lo plane Klo = fl32(K - K32) must carry float64 accuracy for every entry
// the float-float passes can keep, so those entries (K > -kFFLoBand) are
// re-evaluated in float64; the rest keep the float-float lo part.
template <int TG, int CH, int KIND>
__global__ void __launch_bounds__(TG) k_reanchor_ff(DenseArgs<float> A) {
  const CostRef cost = kind_ref<KIND>(A.cost);
  __shared__ float sht[TG / 32];
  constexpr int V = 4;
  const float csh = (float)A.cost.scale, csl = (float)(A.cost.scale - (double)csh);
  int r0, r1;
  row_range(A.m, A.rows_per_block, r0, r1);
  for (int i = r0; i < r1; ++i) {
    float eh[CH][V], el[CH][V];
    float mx = -__builtin_huge_valf();
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = Tile<float, TG, CH>::col(s);
#pragma unroll
      for (int e = 0; e < V; ++e) {
        if (c + e < A.n) {
          const float2 C = cost_ff(cost, i, c + e, csh, csl);
          const float p = A.lamh * C.x;  // lam C = p + pl (TwoProduct of the hi parts)
          const float pl = fmaf(A.lamh, C.x, -p) + fmaf(A.lamh, C.y, A.laml * C.x);
          const FF d = ff_add(FF{__ldg(A.wvh + c + e), __ldg(A.wvl + c + e)}, FF{-p, -pl});
          eh[s][e] = d.hi;
          el[s][e] = d.lo;
          mx = fmaxf(mx, d.hi);
        } else {
          eh[s][e] = -__builtin_huge_valf();
          el[s][e] = 0.f;
        }
      }
    }
    mx = block_max<TG>(mx, sht);
    if (A.rowMa != nullptr && threadIdx.x == 0) A.rowMa[i] = mx;
    if (A.Kout == nullptr) continue;  // recompute mode: the row shift is all the anchor keeps
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = Tile<float, TG, CH>::col(s);
      if (c < A.ldk) {
        float kv[V], lo[V];
#pragma unroll
        for (int e = 0; e < V; ++e) {
          if (c + e < A.n) {
            const FF k = ff_add(FF{eh[s][e], el[s][e]}, FF{-mx, 0.f});
            kv[e] = k.hi;
            lo[e] = k.lo;
            if (A.Klo_out != nullptr && k.hi > -kFFLoBand) {
              const double K64 = (A.wv[c + e] - A.lam * cost_at(cost, i, c + e)) - (double)mx;
              kv[e] = (float)K64;
              lo[e] = (float)(K64 - (double)kv[e]);
            }
          } else {
            kv[e] = -__builtin_huge_valf();
            lo[e] = 0.f;
          }
        }
        store_vec(A.Kout + (int64_t)i * A.ldk + c, kv);
        if (A.Klo_out != nullptr) store_vec(A.Klo_out + (int64_t)i * A.ldk + c, lo);
      }
    }
  }
}

// bit s * V + e set for each entry whose exponent exceeds the row shift mx by
// more than log_keep (the entries with exp(x - mx) > keep; no exp needed)
template <int TG, int CH>
__device__ __forceinline__ unsigned kept_mask_log(const Tile<float, TG, CH>& t, float mx, float log_keep) {
  static_assert(CH * 4 <= 32, "one bit per entry of the tile");
  const float thr = mx + log_keep;
  unsigned mk = 0u;
#pragma unroll
  for (int s = 0; s < CH; ++s)
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (t.x[s][e] > thr) mk |= 1u << (s * 4 + e);
  return mk;
}

// bit s * V + e set for each entry of the thread's tile above `keep`
template <int TG, int CH>
__device__ __forceinline__ unsigned kept_mask(const Tile<float, TG, CH>& t, float keep) {
  static_assert(CH * 4 <= 32, "one bit per entry of the tile");
  unsigned mk = 0u;
#pragma unroll
  for (int s = 0; s < CH; ++s)
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (t.x[s][e] > keep) mk |= 1u << (s * 4 + e);
  return mk;
}

// Up to four kept entries of a thread's row tile with their float-float exp,
// so the second sweep reuses them (entry position s * V + e; -1 = empty); a
// thread with more kept entries recomputes the rest.
struct KeptCache {
  int k0 = -1, k1 = -1, k2 = -1, k3 = -1;
  FF v0{0.f, 0.f}, v1{0.f, 0.f}, v2{0.f, 0.f}, v3{0.f, 0.f};
  int n = 0;
  __device__ __forceinline__ void put(int pos, FF v) {
    if (n == 0) { k0 = pos; v0 = v; }
    else if (n == 1) { k1 = pos; v1 = v; }
    else if (n == 2) { k2 = pos; v2 = v; }
    else if (n == 3) { k3 = pos; v3 = v; }
    ++n;
  }
  __device__ __forceinline__ bool get(int pos, FF& v) const {
    if (pos == k0) { v = v0; return true; }
    if (pos == k1) { v = v1; return true; }
    if (pos == k2) { v = v2; return true; }
    if (pos == k3) { v = v3; return true; }
    return false;
  }
};

// float-float exponent x_ij - mx of entry (s, e) of row i: K_hi + K_lo (K_lo
// absent in float32 mode) + d (hi + lo) - mx
__device__ __forceinline__ FF ff_x(const DenseArgs<float>& A, int i, int64_t c, int e, float mx) {
  FF k;
  if (A.recompute) {
    k = anchored_ff(A, i, c + e);
  } else {
    const int64_t off = (int64_t)i * A.ldk + c + e;
    k = FF{__ldg(A.K + off), A.Klo != nullptr ? __ldg(A.Klo + off) : 0.f};
  }
  const FF x = ff_add(k, FF{A.dv[c + e], A.dvlo[c + e]});
  return ff_add(x, FF{-mx, 0.f});
}

__device__ __forceinline__ FF ff_at(const float* h, const float* l, int64_t j) { return FF{h[j], l[j]}; }

// float64 value as a float-float pair (float64 instructions: kept entries only)
__device__ __forceinline__ FF ff_of(double v) {
  const float h = (float)v;
  return FF{h, (float)(v - (double)h)};
}

// plan pass: c_j = sum_i a_i P_ij (Eqs. 6-7).  Per-entry work in float-float
// (no float64 instruction on the per-row path); the pass stores S_i (float2)
// and the shift M_i (float) per row, and k_rows_ff forms lse_i = M_i + log S_i
// and sum_i a_i lse_i.  Column partials are float-float pairs.
template <int TG, int CH>
__global__ void __launch_bounds__(TG) k_plan_ff(DenseArgs<float> A) {
  extern __shared__ __align__(128) double dyn_sm[];
  __shared__ unsigned long long s_mbar[kMaxRowStages];
  __shared__ float shf[8 * (TG / 32)];
  __shared__ float sht[TG / 32];
  constexpr int V = 4;
  float2* acc = reinterpret_cast<float2*>(dyn_sm + A.ldk / 2);  // after the row buffer
  for (int64_t c = threadIdx.x; c < A.ldk; c += TG) acc[c] = make_float2(0.f, 0.f);
  __syncthreads();
  int r0, r1;
  row_range(A.m, A.rows_per_block, r0, r1);
  RowStream<float> rs;
  rs.start(A, dyn_sm, s_mbar, r0, r1);
  Tile<float, TG, CH> t;
  for (int i = r0; i < r1; ++i) {
    if (!rs.row(t, A, i, r1)) return;
    const float mx = block_max<TG>(t.local_max(), sht);
    const unsigned kept = kept_mask_log<TG, CH>(t, mx, kFFLogKeep);  // float32 filter
    // kept entries: one copy of the float-float code, looped over the mask
    KeptCache kc;
    FF S[1] = {FF{0.f, 0.f}};
    for (unsigned mk = kept; mk != 0u; mk &= mk - 1u) {
      const int pos = __ffs(mk) - 1;
      const int64_t c = Tile<float, TG, CH>::col(pos / V);
      const FF ev = ff_exp(ff_x(A, i, c, pos % V, mx));
      kc.put(pos, ev);
      S[0] = ff_add(S[0], ev);
    }
    block_sum_ffv<TG, 1>(S, shf);
    if (threadIdx.x == 0) {
      reinterpret_cast<float2*>(A.rowS0)[i] = make_float2(S[0].hi, S[0].lo);
      reinterpret_cast<float*>(A.rowM)[i] = mx;
    }
    if (kept == 0u) continue;  // no kept entry among this thread's columns
    const FF w = ff_div(FF{A.aT[i], A.alo[i]}, S[0]);
    for (unsigned mk = kept; mk != 0u; mk &= mk - 1u) {
      const int pos = __ffs(mk) - 1;
      const int64_t c = Tile<float, TG, CH>::col(pos / V) + pos % V;
      FF ev;
      if (!kc.get(pos, ev)) ev = ff_exp(ff_x(A, i, c - pos % V, pos % V, mx));
      const float2 a = acc[c];
      const FF r = ff_add(FF{a.x, a.y}, ff_mul(w, ev));
      acc[c] = make_float2(r.hi, r.lo);
    }
  }
  __syncthreads();
  for (int64_t c = threadIdx.x; c < A.ldk; c += TG)
    reinterpret_cast<float2*>(A.colpart)[(int64_t)blockIdx.x * A.ldk + c] = acc[c];
}

// Armijo trial in difference form (see k_armijo); v1 = em_j (hi, lo parts).
// Stores S0_i, S1_i (float2) and M_i per row for k_rows_ff; the row weight
// a_i / (S0 + S1) and the column contributions in float-float.
template <int TG, int CH>
__global__ void __launch_bounds__(TG) k_armijo_ff(DenseArgs<float> A) {
  extern __shared__ __align__(128) double dyn_sm[];
  __shared__ unsigned long long s_mbar[kMaxRowStages];
  __shared__ float shf[8 * (TG / 32)];
  __shared__ float sht[TG / 32];
  constexpr int V = 4;
  float2* acc = reinterpret_cast<float2*>(dyn_sm + A.ldk / 2);
  for (int64_t c = threadIdx.x; c < A.ldk; c += TG) acc[c] = make_float2(0.f, 0.f);
  __syncthreads();
  int r0, r1;
  row_range(A.m, A.rows_per_block, r0, r1);
  RowStream<float> rs;
  rs.start(A, dyn_sm, s_mbar, r0, r1);
  // an entry can grow by exp(t max|Delta|/eta) at the trial point: keep more
  const float log_keep = A.s2 > 0.0 ? kFFLogKeep + (float)log(A.s2) : -__builtin_huge_valf();
  Tile<float, TG, CH> t;
  for (int i = r0; i < r1; ++i) {
    if (!rs.row(t, A, i, r1)) return;
    const float mx = block_max<TG>(t.local_max(), sht);
    const unsigned kept = kept_mask_log<TG, CH>(t, mx, log_keep);
    KeptCache kc;
    FF S[2] = {FF{0.f, 0.f}, FF{0.f, 0.f}};
    for (unsigned mk = kept; mk != 0u; mk &= mk - 1u) {
      const int pos = __ffs(mk) - 1;
      const int64_t c = Tile<float, TG, CH>::col(pos / V);
      const FF ev = ff_exp(ff_x(A, i, c, pos % V, mx));
      kc.put(pos, ev);
      S[0] = ff_add(S[0], ev);
      S[1] = ff_add(S[1], ff_mul(ev, ff_at(A.v1, A.v1lo, c + pos % V)));
    }
    block_sum_ffv<TG, 2>(S, shf);
    if (threadIdx.x == 0) {
      reinterpret_cast<float2*>(A.rowS0)[i] = make_float2(S[0].hi, S[0].lo);
      reinterpret_cast<float2*>(A.rowS1)[i] = make_float2(S[1].hi, S[1].lo);
      reinterpret_cast<float*>(A.rowM)[i] = mx;
    }
    if (kept == 0u) continue;
    const FF w = ff_div(FF{A.aT[i], A.alo[i]}, ff_add(S[0], S[1]));
    for (unsigned mk = kept; mk != 0u; mk &= mk - 1u) {
      const int pos = __ffs(mk) - 1;
      const int64_t c = Tile<float, TG, CH>::col(pos / V) + pos % V;
      FF ev;
      if (!kc.get(pos, ev)) ev = ff_exp(ff_x(A, i, c - pos % V, pos % V, mx));
      const FF x = ff_add(ev, ff_mul(ev, ff_at(A.v1, A.v1lo, c)));  // ev (1 + em_j)
      const float2 a = acc[c];
      const FF r = ff_add(FF{a.x, a.y}, ff_mul(w, x));
      acc[c] = make_float2(r.hi, r.lo);
    }
  }
  __syncthreads();
  for (int64_t c = threadIdx.x; c < A.ldk; c += TG)
    reinterpret_cast<float2*>(A.colpart)[(int64_t)blockIdx.x * A.ldk + c] = acc[c];
}

// certificate (see k_certify): v1 = y, v2 = omega (hi, lo parts), v3 = e_c / S
// (hi, v3lo), v1d/v3d float64 copies for the plan export.  Per row: the kept
// entries' plan values in float-float (cached), zeta_i = min_j C_ij - gamma_j
// by a float32 scan whose candidates within the float32 error bound of the
// minimum are re-evaluated exactly in float64, and (dense costs only) the
// rank-one sum_j C_ij e_c,j / S in float-float; the sums over kept entries in
// float-float.  k_rows_cert forms the per-row float64 scalars (e_r, primal,
// dual and residual totals) from the stored per-row results; for the grid cost
// it forms sum_j C_ij e_c,j / S from four moments of e_c / S.
template <int TG, int CH, int KIND>
__global__ void __launch_bounds__(TG) k_certify_ff(DenseArgs<float> A) {
  const CostRef cost = kind_ref<KIND>(A.cost);  // the kind is a compile-time constant below
  extern __shared__ __align__(128) double dyn_sm[];
  __shared__ unsigned long long s_mbar[kMaxRowStages];
  __shared__ float shf[8 * (TG / 32)];
  __shared__ float sht[TG / 32];
  __shared__ long long shl[TG / 32];
  __shared__ double s_er;
  // |fl32(C) - fl32(gamma) - (C - gamma)| <= 2^-22 (max|C| + max|gamma|)
  const float zbound = 2.f * (float)ldexp(A.bounds[0] + A.bounds[1], -22);
  const float csh = (float)A.cost.scale, csl = (float)(A.cost.scale - (double)csh);
  constexpr bool rank1 = KIND != 2;  // grid: closed form in k_rows_cert
  constexpr int V = 4;
  float2* acc = reinterpret_cast<float2*>(dyn_sm + A.ldk / 2);
  for (int64_t c = threadIdx.x; c < A.ldk; c += TG) acc[c] = make_float2(0.f, 0.f);
  __syncthreads();
  int r0, r1;
  row_range(A.m, A.rows_per_block, r0, r1);
  RowStream<float> rs;
  rs.start(A, dyn_sm, s_mbar, r0, r1);
  Tile<float, TG, CH> t;
  for (int i = r0; i < r1; ++i) {
    if (!rs.row(t, A, i, r1)) return;
    const float mx = block_max<TG>(t.local_max(), sht);
    // sweep 1 (every entry, float32): c-transform scan (not for the grid cost,
    // whose c-transform comes in exactly from the separable computation) and,
    // for dense and point costs, the rank-one sum; the kept entries'
    // float-float work runs from the mask
    const unsigned kept = kept_mask_log<TG, CH>(t, mx, kFFLogKeep);
    float z32 = __builtin_huge_valf(), ceh = 0.f, cel = 0.f;
    int zpos = -1;  // the thread's scan minimum: always re-evaluated when the thread holds a candidate
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = Tile<float, TG, CH>::col(s);
#pragma unroll
      for (int e = 0; e < V; ++e) {
        if (c + e >= A.n) continue;
        if (KIND == 2) continue;  // grid: no scan and no rank-one sum here
        const float2 C = cost_ff(cost, i, c + e, csh, csl);
        const float zv = C.x - A.gam32[c + e];
        if (zv < z32) {
          z32 = zv;
          zpos = s * V + e;
        }
        if (rank1) {
          // C e_c / S in float-float: exact product of the hi parts plus the cross terms
          const float vh = A.v3[c + e];
          const float p = C.x * vh;
          cel += fmaf(C.x, A.v3lo[c + e], fmaf(C.y, vh, fmaf(C.x, vh, -p)));
          ff_acc(ceh, cel, p);
        }
      }
    }
    KeptCache kc;
    FF R[2] = {FF{0.f, 0.f}, ff_fast_two_sum(ceh, cel)};
    for (unsigned mk = kept; mk != 0u; mk &= mk - 1u) {
      const int pos = __ffs(mk) - 1;
      const FF ev = ff_exp(ff_x(A, i, Tile<float, TG, CH>::col(pos / V), pos % V, mx));
      kc.put(pos, ev);
      R[0] = ff_add(R[0], ev);
    }
    block_sum_ffv<TG, 2>(R, shf);
    double zeta;
    if constexpr (KIND == 2) {
      zeta = A.zeta_in[i];
    } else {
    const float m32 = -block_max<TG>(-z32, sht);
    double zc = kInf;
    if (z32 <= m32 + zbound) {  // only threads holding a candidate: mark, then re-evaluate in float64
      unsigned cand = zpos >= 0 ? 1u << zpos : 0u;
#pragma unroll
      for (int s = 0; s < CH; ++s) {
        const int64_t c = Tile<float, TG, CH>::col(s);
#pragma unroll
        for (int e = 0; e < V; ++e)
          if (c + e < A.n && cost_ff(cost, i, c + e, csh, csl).x - A.gam32[c + e] <= m32 + zbound)
            cand |= 1u << (s * V + e);
      }
      for (; cand != 0u; cand &= cand - 1u) {
        const int pos = __ffs(cand) - 1;
        const int64_t j = Tile<float, TG, CH>::col(pos / V) + pos % V;
        zc = fmin(zc, cost_at(cost, i, j) - A.gam[j]);
      }
    }
    zeta = block_min_exact<TG>(zc, shl);
    }
    // sweep 2 (kept entries): e_r, the plan part of the primal, complementarity, column sums
    FF Q[4] = {FF{0.f, 0.f}, FF{0.f, 0.f}, FF{0.f, 0.f}, FF{0.f, 0.f}};
    if (kept != 0u) {
      const FF inv = ff_div(FF{1.f, 0.f}, R[0]);
      const FF ai{A.aT[i], A.alo[i]};
      const FF zf = ff_of(zeta);
      for (unsigned mk = kept; mk != 0u; mk &= mk - 1u) {
        const int pos = __ffs(mk) - 1;
        const int64_t c = Tile<float, TG, CH>::col(pos / V) + pos % V;
        FF ev;
        if (!kc.get(pos, ev)) ev = ff_exp(ff_x(A, i, c - pos % V, pos % V, mx));
        const FF P = ff_mul(ev, inv);
        const float2 Cp = cost_ff(cost, i, c, csh, csl);
        const FF C{Cp.x, Cp.y};
        const FF aP = ff_mul(ai, P);
        const FF F = ff_mul(aP, ff_at(A.v1, A.v1lo, c));
        Q[0] = ff_add(Q[0], ff_mul(P, ff_at(A.v2, A.v2lo, c)));
        Q[1] = ff_add(Q[1], P);
        Q[2] = ff_add(Q[2], ff_mul(C, F));
        const FF red = ff_add(ff_add(C, ff_neg(zf)), ff_neg(ff_at(A.gam32, A.gamlo, c)));
        Q[3] = ff_add(Q[3], ff_mul(aP, red));
        const float2 a = acc[c];
        const FF r = ff_add(FF{a.x, a.y}, F);
        acc[c] = make_float2(r.hi, r.lo);
      }
    }
    block_sum_ffv<TG, 4>(Q, shf);
    if (threadIdx.x == 0) {
      float2* rb2 = reinterpret_cast<float2*>(A.rowbuf);
      const int64_t m = A.m;
#pragma unroll
      for (int q = 0; q < 4; ++q) rb2[q * m + i] = make_float2(Q[q].hi, Q[q].lo);
      A.rowbuf[4 * m + i] = zeta;
      rb2[5 * m + i] = make_float2(R[1].hi, R[1].lo);
    }
    if (A.plan_out != nullptr) {  // the final export: Xhat row by row (float64)
      if (threadIdx.x == 0) s_er = A.a[i] * ((double)Q[0].hi + (double)Q[0].lo);
      __syncthreads();
      const double er = s_er;
      const FF inv = ff_div(FF{1.f, 0.f}, R[0]);
      const double a_i = A.a[i];
#pragma unroll 1
      for (int pos = 0; pos < CH * V; ++pos) {
        const int64_t c = Tile<float, TG, CH>::col(pos / V) + pos % V;
        if (c >= A.n) continue;
        double P = 0.0;
        if ((kept >> pos) & 1u) {
          FF ev;
          if (!kc.get(pos, ev)) ev = ff_exp(ff_x(A, i, c - pos % V, pos % V, mx));
          const FF Pf = ff_mul(ev, inv);
          P = (double)Pf.hi + (double)Pf.lo;
        }
        A.plan_out[(int64_t)i * A.n + c] = a_i * P * A.v1d[c] + er * A.v3d[c];
      }
    }
  }
  __syncthreads();
  for (int64_t c = threadIdx.x; c < A.ldk; c += TG)
    reinterpret_cast<float2*>(A.colpart)[(int64_t)blockIdx.x * A.ldk + c] = acc[c];
}

// plan export for checks
template <int TG, int CH>
__global__ void __launch_bounds__(TG) k_export_ff(DenseArgs<float> A) {
  extern __shared__ __align__(128) double dyn_sm[];
  __shared__ unsigned long long s_mbar[kMaxRowStages];
  __shared__ float shf[8 * (TG / 32)];
  __shared__ float sht[TG / 32];
  constexpr int V = 4;
  int r0, r1;
  row_range(A.m, A.rows_per_block, r0, r1);
  RowStream<float> rs;
  rs.start(A, dyn_sm, s_mbar, r0, r1);
  Tile<float, TG, CH> t;
  for (int i = r0; i < r1; ++i) {
    if (!rs.row(t, A, i, r1)) return;
    const float mx = block_max<TG>(t.local_max(), sht);
    const double M = (double)mx;
    t.exp_shift(mx);
    double ps = 0.0;
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = Tile<float, TG, CH>::col(s);
#pragma unroll
      for (int e = 0; e < V; ++e)
        if (t.x[s][e] > kFFKeep) ps += exp(FFRow<TG, CH>::x64(A, i, c, e, M));
    }
    double S[1] = {ps};
    block_sum_ff<TG, 1>(S, shf);
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int64_t c = Tile<float, TG, CH>::col(s);
#pragma unroll
      for (int e = 0; e < V; ++e)
        if (c + e < A.n)
          A.plan_out[(int64_t)i * A.n + c + e] =
              t.x[s][e] > kFFKeep ? exp(FFRow<TG, CH>::x64(A, i, c, e, M)) / S[0] : 0.0;
    }
  }
}

}  // namespace ibsn
