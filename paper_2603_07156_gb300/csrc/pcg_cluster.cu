// Newton direction by PCG on one thread-block cluster (row a5 of the hot path,
// the shifted system (H_rho + ||g|| I) Delta = -g of Alg. 2; same float32
// Chronopoulos-Gear recurrence and float-float reductions as k_pcg32).
//
// Late in a solve the sparsified plan P_rho has a few nonzeros per row and
// the whole system fits in on-chip memory.  There the grid-wide kernel is
// bound by its two grid-wide waits per iteration (about 1.5 us each through
// L2 atomics).  This kernel runs the same iteration on one cluster of CS CTAs
// (CS = 16, one CTA of 1024 threads per SM): every CTA stages its rows' and
// columns' entries in shared memory once, with each entry's column (row)
// already translated to the distributed-shared-memory address of that
// column's state (row's t value) in its owner CTA, keeps the column state and
// t in shared memory, and synchronises with the cluster barrier.  Per
// iteration: row pass (t_i = a_i (P u)_i from remote column states), cluster
// barrier, column pass (update and six partial sums), cluster barrier, every
// CTA sums the CS partial records in rank order and forms alpha, beta
// identically.
//
// Ownership: CTA r owns rows [r rpc, (r+1) rpc) and columns [r cpc, (r+1) cpc);
// thread t owns local row t and local column t (rpc, cpc <= 1024).  When the
// staged entries of any CTA exceed its shared memory the kernel stores
// kDevCapacity in *err and every CTA returns; the host then uses the
// grid-wide kernel.  Control flow is uniform over the cluster (every CTA
// forms the same scalars from the same totals), so every CTA reaches every
// cluster barrier; a last cluster barrier keeps each CTA's shared memory alive
// until no other CTA reads it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace ibsn {

namespace {

constexpr int kClT = 1024;     // threads per CTA
constexpr int kClMax = 16;     // CTAs per cluster
constexpr size_t kClSmem = 200 * 1024;

struct PcgClArgs {
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
  int* err;
  double* scal;
  int m, n, istar;
  int rpc, cpc;
  float inv_eta, shift;
  double rtol;
  int maxit;
  uint32_t smem_bytes;
};

__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_map(const void* p, uint32_t rank) {
  uint32_t d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
  return d;
}
__device__ __forceinline__ float4 cl_ld4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a)
               : "memory");
  return v;
}
__device__ __forceinline__ int cl_ld_int(uint32_t a) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void cl_st(uint32_t a, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void cl_st2(uint32_t a, float x, float y) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(x), "f"(y) : "memory");
}
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// exclusive scan of one int per thread over the CTA; total on every thread
__device__ __forceinline__ int cta_scan_excl(int v, int* sh, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) sh[w] = x;
  __syncthreads();
  int base = 0, tot = 0;
  for (int q = 0; q < kClT / 32; ++q) {
    const int s = sh[q];
    if (q < w) base += s;
    tot += s;
  }
  *total = tot;
  return base + x - v;
}

// CTA sums of six floats, pushed into slot `rank` of every CTA's receive
// buffer.  Within a warp the six values (padded to eight) are reduced by
// recursive halving: at each of the first three exchange steps a lane sends
// half of the quantities it still holds and keeps the other half, so a warp
// issues 9 shuffles instead of 30 and lane l ends with the warp total of
// quantity l / 4 (float, as a plain warp sum).  Warps 0..5 then sum quantity
// q over the CTA's 32 warps in float-float, and lane r of warp q writes the
// (hi, lo) pair into CTA r's buffer.
__device__ __forceinline__ void cta_sum6_push(const float (&v)[6], float* sh, float* recv, uint32_t rank,
                                              uint32_t cs) {
  constexpr int NW = kClT / 32;
  static_assert(NW == 32, "one warp partial per lane");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float x[4];
  {
    const bool up = (lane & 16) != 0;  // keeps quantities 4..7 (0..3 otherwise; 6, 7 are zero)
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const float send = up ? v[p] : v[p + 4];
      const float keep = up ? v[p + 4] : v[p];
      x[p] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int p = 2; p < 4; ++p) {
      const float send = up ? v[p] : 0.f;
      const float keep = up ? 0.f : v[p];
      x[p] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
  }
  {
    const bool up = (lane & 8) != 0;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const float send = up ? x[p] : x[p + 2];
      const float keep = up ? x[p + 2] : x[p];
      x[p] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
  }
  {
    const bool up = (lane & 4) != 0;
    const float send = up ? x[0] : x[1];
    const float keep = up ? x[1] : x[0];
    x[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  x[0] += __shfl_xor_sync(0xffffffffu, x[0], 2);
  x[0] += __shfl_xor_sync(0xffffffffu, x[0], 1);
  const int qd = lane >> 2;  // quantity this lane now holds
  if ((lane & 3) == 0 && qd < 6) sh[qd * NW + w] = x[0];
  __syncthreads();
  if (w < 6) {
    const FF tq = warp_sum_ff(FF{sh[w * NW + lane], 0.f});
    if ((uint32_t)lane < cs) cl_st2(cl_map(recv + 12 * rank + 2 * w, (uint32_t)lane), tq.hi, tq.lo);
  }
}

// totals of the received records (warp 0): a fixed-order warp tree over the
// records in rank order, so every CTA forms bit-identical totals (lane 0)
__device__ __forceinline__ void cluster_totals(const float* recv, uint32_t cs, FF (&tot)[6]) {
  const uint32_t lane = threadIdx.x & 31;
  FF v[6];
#pragma unroll
  for (int q = 0; q < 6; ++q)
    v[q] = lane < cs ? FF{recv[12 * lane + 2 * q], recv[12 * lane + 2 * q + 1]} : FF{0.f, 0.f};
#pragma unroll
  for (int q = 0; q < 6; ++q) tot[q] = warp_sum_ff(v[q]);
}

__global__ void __launch_bounds__(kClT, 1) k_pcg_cluster(PcgClArgs A) {
  extern __shared__ __align__(16) unsigned char cl_sm[];
  __shared__ float s_red[6 * (kClT / 32)];
  __shared__ __align__(16) float s_recv[12 * kClMax];    // every CTA's record, pushed by its owner
  __shared__ int s_flag;                                 // staging overflow (read by every CTA)
  __shared__ int s_scan[kClT / 32];
  __shared__ float s_a32, s_b32, s_tstar, s_rtol2, s_astar, s_rr0, s_gam;
  __shared__ int s_done;
  const uint32_t rank = cl_rank(), cs = gridDim.x;
  const int t = threadIdx.x;
  // shared-memory layout (identical in every CTA, so a local address names
  // the same object in any CTA's window)
  float4* s_cs = reinterpret_cast<float4*>(cl_sm);      // cpc column states {r, w, s, 1/diag}
  float* s_p = reinterpret_cast<float*>(s_cs + A.cpc);  // cpc
  float* s_x = s_p + A.cpc;                             // cpc
  float* s_t = s_x + A.cpc;                             // m: replica of t, written by the rows' owners
  int* s_roff = reinterpret_cast<int*>(s_t + A.m);      // rpc + 1
  int* s_coff = s_roff + A.rpc + 1;                     // cpc + 1
  unsigned* s_rmask = reinterpret_cast<unsigned*>(s_coff + A.cpc + 1);  // rpc: CTAs owning a column of the row
  size_t used = (size_t)(reinterpret_cast<unsigned char*>(s_rmask + A.rpc) - cl_sm);
  used = (used + 15) & ~(size_t)15;
  uint2* s_ent = reinterpret_cast<uint2*>(cl_sm + used);
  const int64_t cap = ((int64_t)A.smem_bytes - (int64_t)used) / (int64_t)sizeof(uint2);

  const int row0 = (int)rank * A.rpc, col0 = (int)rank * A.cpc;
  const int nrow = max(0, min(A.rpc, A.m - row0)), ncol = max(0, min(A.cpc, A.n - col0));
  const int i = row0 + t, j = col0 + t;
  int rlen = 0, clen = 0;
  if (t < nrow && i != A.istar) rlen = A.row_len[i];
  if (t < ncol) clen = (int)(A.colptr[j + 1] - A.colptr[j]);
  int rtot = 0, ctot = 0;
  const int roff = cta_scan_excl(rlen, s_scan, &rtot);
  const int coff = cta_scan_excl(clen, s_scan, &ctot);
  if (t == 0) s_flag = (used > A.smem_bytes || (int64_t)rtot + ctot > cap) ? 1 : 0;
  __syncthreads();
  cl_sync();
  int bad = 0;
  for (uint32_t r = 0; r < cs; ++r) bad |= cl_ld_int(cl_map(&s_flag, r));
  if (bad) {
    if (rank == 0 && t == 0) atomicExch(A.err, (int)kDevCapacity);
    cl_sync();
    return;
  }

  // stage the entries: a row entry carries the distributed-shared-memory
  // address of its column's state in the owner CTA, a column entry the
  // local index of its row in the t replica
  if (t < nrow) s_roff[t] = roff;
  if (t == 0) s_roff[nrow] = rtot;
  if (t < ncol) s_coff[t] = coff;
  if (t == 0) s_coff[ncol] = ctot;
  unsigned mask = 0;
  if (rlen > 0) {
    const int64_t st = A.row_start[i];
    for (int k = 0; k < rlen; ++k) {
      const int c = A.col[st + k];
      const int owner = c / A.cpc;
      mask |= 1u << owner;
      s_ent[roff + k] = make_uint2(cl_map(s_cs + (c - owner * A.cpc), (uint32_t)owner), __float_as_uint(A.val[st + k]));
    }
  }
  if (t < nrow) s_rmask[t] = mask;
  float q = 0.f, crho = 0.f, r0 = 0.f, dinv = 0.f;
  if (t < ncol) {
    const int64_t k0 = A.colptr[j];
    for (int k = 0; k < clen; ++k)
      s_ent[rtot + coff + k] = make_uint2((unsigned)A.crow[k0 + k], __float_as_uint(A.cval[k0 + k]));
    dinv = (float)(1.0 / A.diag[j]);
    r0 = (float)A.rhs[j];
    q = A.prow[j];
    crho = (float)A.crho[j];
    s_cs[t] = make_float4(r0, 0.f, 0.f, dinv);
    s_p[t] = 0.f;
    s_x[t] = 0.f;
  }
  const float ai = (t < nrow) ? A.a32[i] : 0.f;
  {
    const float red[6] = {0.f, 0.f, 0.f, q * dinv * r0, 0.f, 0.f};
    cta_sum6_push(red, s_red, s_recv, rank, cs);
  }
  __syncthreads();
  cl_sync();  // states, entries and records of every CTA are in place

  FF Qr{0.f, 0.f}, Qw{0.f, 0.f}, Qs{0.f, 0.f};
  float rr = 0.f;
  // thread 0's scalars live in shared memory (1024 threads leave 64 registers each)
  if (t == 0) {
    s_rtol2 = (float)(A.rtol * A.rtol);
    s_astar = A.a32[A.istar];
    s_rr0 = 0.f;
    s_gam = 0.f;
  }
  bool warm = true;
  int it = 0;
  if (t < 32) {
    FF tot[6];
    cluster_totals(s_recv, cs, tot);
    Qr = tot[3];
  }
  if (t == 0) {
    s_a32 = 0.f;
    s_b32 = 0.f;
    s_tstar = s_astar * Qr.hi;
  }
  __syncthreads();
  const int re0 = (t < nrow) ? s_roff[t] : 0, re1 = (t < nrow) ? s_roff[t + 1] : 0;
  const int ce0 = (t < ncol) ? rtot + s_coff[t] : 0, ce1 = (t < ncol) ? rtot + s_coff[t + 1] : 0;
  const unsigned rmask = (t < nrow) ? s_rmask[t] : 0u;
  for (;;) {
    const float a32 = s_a32, b32 = s_b32, tstar = s_tstar;
    // ---- row pass: t_i = a_i (P_rho u)_i, u from the owners' column states;
    // t_i goes to every CTA that owns a column of row i
    if (rmask != 0u) {
      float acc = 0.f;
#pragma unroll 4
      for (int k = re0; k < re1; ++k) {
        const uint2 e = s_ent[k];
        const float4 c = cl_ld4(e.x);
        acc += __uint_as_float(e.y) * ((c.x - a32 * (c.y + b32 * c.z)) * c.w);
      }
      const float ti = ai * acc;
      for (unsigned mk = rmask; mk != 0u; mk &= mk - 1u) cl_st(cl_map(s_t + i, (uint32_t)(__ffs(mk) - 1)), ti);
    }
    cl_sync();
    // ---- column pass (t from the local replica)
    float dsum[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (t < ncol) {
      float acc = 0.f;
#pragma unroll 2
      for (int k = ce0; k < ce1; ++k) {
        const uint2 e = s_ent[k];
        acc += __uint_as_float(e.y) * s_t[e.x];
      }
      const float4 c = s_cs[t];
      const float s_new = c.y + b32 * c.z;
      const float p_new = c.x * c.w + b32 * s_p[t];
      const float r_new = c.x - a32 * s_new;
      const float u_new = r_new * c.w;
      const float v = acc + q * tstar;
      const float w_new = (crho * u_new - v) * A.inv_eta + A.shift * u_new;
      s_x[t] += a32 * p_new;
      s_p[t] = p_new;
      s_cs[t] = make_float4(r_new, w_new, s_new, c.w);
      const float qd = q * c.w;
      dsum[0] = r_new * u_new;
      dsum[1] = w_new * u_new;
      dsum[2] = r_new * r_new;
      dsum[3] = qd * r_new;
      dsum[4] = qd * w_new;
      dsum[5] = qd * s_new;
    }
    cta_sum6_push(dsum, s_red, s_recv, rank, cs);
    cl_sync();  // every record has arrived everywhere
    FF tot[6];
    if (t < 32) cluster_totals(s_recv, cs, tot);
    if (t == 0) {
      // Chronopoulos-Gear update, identical in every CTA; alpha and beta
      // start from this iteration's values (the loop-top copies a32, b32)
      float alpha = a32, beta = b32, rr0 = s_rr0, gam = s_gam;
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
        if (rr <= s_rtol2 * rr0 || it >= A.maxit) {
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
      s_rr0 = rr0;
      s_gam = gam;
      s_done = done;
      s_a32 = alpha;
      s_b32 = beta;
      const FF qu = ff_add(Qr, ff_neg(ff_mul_f(ff_add(Qw, ff_mul_f(Qs, beta)), alpha)));
      s_tstar = s_astar * qu.hi;
    }
    __syncthreads();
    if (s_done) break;
  }
  if (t < ncol) A.x_out[j] = (double)s_x[t];
  if (rank == 0 && t == 0) {
    A.scal[S_CG_ITERS] = (double)it;
    A.scal[S_CG_RES] = s_rr0 > 0.f ? sqrt((double)rr / (double)s_rr0) : 0.0;
  }
  cl_sync();  // no CTA leaves while another may still write or read its shared memory
}

// cluster size this device schedules (0: none), found once per process
int cluster_size_for_device() {
  static std::once_flag once;
  static int size = 0;
  std::call_once(once, [] {
    if (cudaFuncSetAttribute(k_pcg_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClSmem) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    if (cudaFuncSetAttribute(k_pcg_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
      cudaGetLastError();
    for (int csz : {kClMax, 8}) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = (unsigned)csz;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3((unsigned)csz);
      cfg.blockDim = dim3(kClT);
      cfg.dynamicSmemBytes = kClSmem;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int ncl = 0;
      if (cudaOccupancyMaxActiveClusters(&ncl, k_pcg_cluster, &cfg) == cudaSuccess && ncl >= 1) {
        size = csz;
        return;
      }
      cudaGetLastError();
    }
  });
  return size;
}

}  // namespace

cudaError_t launch_pcg_cluster(const SparseBufs& S, const PcgBufs& B, int m, int64_t n, int istar, const float* a32,
                               double eta, double shift, double rtol, int maxit, double* scal, cudaStream_t st,
                               bool* launched) {
  *launched = false;
  const int csz = cluster_size_for_device();
  if (csz <= 0) return cudaSuccess;
  const int64_t lim = (int64_t)csz * kClT;
  if ((int64_t)m > lim || n > lim) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(B.err, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  PcgClArgs A;
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
  A.err = B.err;
  A.scal = scal;
  A.m = m;
  A.n = (int)n;
  A.istar = istar;
  A.rpc = (int)((m + csz - 1) / csz);
  A.cpc = (int)((n + csz - 1) / csz);
  A.inv_eta = (float)(1.0 / eta);
  A.shift = (float)shift;
  A.rtol = rtol;
  A.maxit = maxit;
  A.smem_bytes = (uint32_t)kClSmem;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)csz;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)csz);
  cfg.blockDim = dim3(kClT);
  cfg.dynamicSmemBytes = kClSmem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_pcg_cluster, A);
  note_launch();
  if (e == cudaSuccess) *launched = true;
  return e;
}

}  // namespace ibsn
