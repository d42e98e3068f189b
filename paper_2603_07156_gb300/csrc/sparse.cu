// Sparsified Hessian H_rho of Alg. 1 in CSR/CSC form and the Newton-direction
// solve of Alg. 2 by Jacobi-preconditioned CG in one persistent kernel.
//
// H_rho v = (c_rho o v - P_rho^T (a o (P_rho v))) / eta, with c_rho = P_rho^T a,
// is applied matrix-free: a row phase (u = P_rho v over CSR rows, row i* dense)
// and a column phase (P_rho^T w over CSC columns).  The CSC copy is built
// deterministically: block b of the sparsify pass owns rows [b*rpb, (b+1)*rpb),
// its per-column counts are prefix-summed over blocks, and each block scatters
// its rows in row order.
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
// Persistent PCG.  Three bounded grid barriers per iteration:
//   A rows:  u_i = sum_j P_ij p_j with p = z + beta p_old formed on the fly,
//            w_i = a_i u_i; row i* (dense) as per-block partial dots
//   B cols:  p_j <- z_j + beta p_j; v_j = sum_i P_ij w_i + P_i*j w_i*;
//            q_j = (c_rho_j p_j - v_j)/eta + shift p_j; partial p.q
//   C upd:   alpha = rz / pq; x += alpha p; r -= alpha q; z = r / diag;
//            partials r.z and r.r
// Every block reduces the per-block partials itself in a fixed order, so all
// blocks take the same branch.
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
  double *x, *r, *z, *p, *q, *w;
  double* part;  // [4][nb]
  unsigned int* bar;
  int* err;
  double* scal;
  int m, istar;
  int64_t n;
  double inv_eta, shift, rtol;
  int maxit;
  unsigned long long deadline_ns;
};

__device__ __forceinline__ double reduce_parts(const double* part, int nb) {
  // fixed-order reduction of nb partials by warp 0, broadcast through smem
  __shared__ double s_val;
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int q = threadIdx.x; q < nb; q += 32) s += __ldcg(part + q);
    s = warp_sum(s);
    if (threadIdx.x == 0) s_val = s;
  }
  __syncthreads();
  const double v = s_val;
  __syncthreads();
  return v;
}

template <int NT>
__device__ __forceinline__ double block_total(double v, double* sh) {
  double t[1] = {v};
  block_sum<NT, 1>(t, sh);
  return t[0];
}

template <typename T>
__global__ void __launch_bounds__(kPcgThreads) k_pcg(PcgArgs<T> A) {
  __shared__ double sh[2 * (kPcgThreads / 32)];
  const int nb = gridDim.x;
  const int lane = threadIdx.x & 31;
  const int nwb = kPcgThreads / 32;
  const int gwarp = blockIdx.x * nwb + (threadIdx.x >> 5);
  const int nwarps = nb * nwb;
  const int64_t gtid = (int64_t)blockIdx.x * kPcgThreads + threadIdx.x;
  const int64_t nthr = (int64_t)nb * kPcgThreads;
  double* partRZ = A.part;
  double* partRR = A.part + nb;
  double* partPQ = A.part + 2 * nb;
  double* partD = A.part + 3 * nb;
  unsigned int* bcount = A.bar;
  unsigned int* bgen = A.bar + 1;

  // init: x = 0, r = rhs, z = r / diag
  double lrz = 0.0, lrr = 0.0;
  for (int64_t j = gtid; j < A.n; j += nthr) {
    const double rj = A.rhs[j];
    const double zj = rj / A.diag[j];
    __stcg(A.x + j, 0.0);
    __stcg(A.r + j, rj);
    __stcg(A.z + j, zj);
    __stcg(A.p + j, 0.0);
    lrz += rj * zj;
    lrr += rj * rj;
  }
  {
    double t[2] = {lrz, lrr};
    block_sum<kPcgThreads, 2>(t, sh);
    if (threadIdx.x == 0) {
      __stcg(partRZ + blockIdx.x, t[0]);
      __stcg(partRR + blockIdx.x, t[1]);
    }
  }
  if (!grid_barrier(bcount, bgen, A.err, A.deadline_ns)) return;

  double rz_old = 0.0, bnorm = 0.0, rr = 0.0;
  int it = 0;
  // column slice of row i* owned by this block
  const int64_t dchunk = (A.n + nb - 1) / nb;
  const int64_t d0 = (int64_t)blockIdx.x * dchunk;
  const int64_t d1 = d0 + dchunk < A.n ? d0 + dchunk : A.n;
  for (;;) {
    const double rz = reduce_parts(partRZ, nb);
    rr = reduce_parts(partRR, nb);
    if (it == 0) bnorm = sqrt(rr);
    if (bnorm == 0.0 || sqrt(rr) <= A.rtol * bnorm || it >= A.maxit) break;
    const double beta = (it == 0) ? 0.0 : rz / rz_old;
    rz_old = rz;
    // ---- A: rows
    for (int i = gwarp; i < A.m; i += nwarps) {
      if (i == A.istar) continue;
      const int64_t s = A.row_start[i];
      const int len = A.row_len[i];
      double acc = 0.0;
      for (int k = lane; k < len; k += 32) {
        const int32_t j = A.col[s + k];
        acc += (double)A.val[s + k] * (__ldcg(A.z + j) + beta * __ldcg(A.p + j));
      }
      acc = warp_sum(acc);
      if (lane == 0) __stcg(A.w + i, A.a[i] * acc);
    }
    {
      double ld = 0.0;
      for (int64_t j = d0 + threadIdx.x; j < d1; j += kPcgThreads)
        ld += (double)A.prow[j] * (__ldcg(A.z + j) + beta * __ldcg(A.p + j));
      ld = block_total<kPcgThreads>(ld, sh);
      if (threadIdx.x == 0) __stcg(partD + blockIdx.x, ld);
    }
    if (!grid_barrier(bcount, bgen, A.err, A.deadline_ns)) return;
    // ---- B: columns
    const double wstar = A.a[A.istar] * reduce_parts(partD, nb);
    double lpq = 0.0;
    for (int64_t j = gwarp; j < A.n; j += nwarps) {
      double acc = 0.0;
      const int64_t k1 = A.colptr[j + 1];
      for (int64_t k = A.colptr[j] + lane; k < k1; k += 32) acc += (double)A.cval[k] * __ldcg(A.w + A.crow[k]);
      acc = warp_sum(acc);
      if (lane == 0) {
        const double pj = __ldcg(A.z + j) + beta * __ldcg(A.p + j);
        __stcg(A.p + j, pj);
        const double v = acc + (double)A.prow[j] * wstar;
        const double qj = (A.crho[j] * pj - v) * A.inv_eta + A.shift * pj;
        __stcg(A.q + j, qj);
        lpq += pj * qj;
      }
    }
    lpq = block_total<kPcgThreads>(lpq, sh);
    if (threadIdx.x == 0) __stcg(partPQ + blockIdx.x, lpq);
    if (!grid_barrier(bcount, bgen, A.err, A.deadline_ns)) return;
    // ---- C: update
    const double pq = reduce_parts(partPQ, nb);
    const double alpha = pq > 0.0 ? rz_old / pq : 0.0;
    lrz = 0.0;
    lrr = 0.0;
    for (int64_t j = gtid; j < A.n; j += nthr) {
      const double pj = __ldcg(A.p + j);
      __stcg(A.x + j, __ldcg(A.x + j) + alpha * pj);
      const double rj = __ldcg(A.r + j) - alpha * __ldcg(A.q + j);
      __stcg(A.r + j, rj);
      const double zj = rj / A.diag[j];
      __stcg(A.z + j, zj);
      lrz += rj * zj;
      lrr += rj * rj;
    }
    {
      double t[2] = {lrz, lrr};
      block_sum<kPcgThreads, 2>(t, sh);
      if (threadIdx.x == 0) {
        __stcg(partRZ + blockIdx.x, t[0]);
        __stcg(partRR + blockIdx.x, t[1]);
      }
    }
    if (!grid_barrier(bcount, bgen, A.err, A.deadline_ns)) return;
    ++it;
    if (pq <= 0.0) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.scal[S_CG_ITERS] = (double)it;
    A.scal[S_CG_RES] = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
  }
}

}  // namespace

int pcg_max_blocks(int nsm) { return nsm * 4; }

cudaError_t launch_csc_build(const SparseBufs& S, int m, int64_t n, int64_t ldk, int nb, int rpb, bool fp64,
                             const double* a, int istar, double eta, cudaStream_t st) {
  k_colscan<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S.blkcnt, S.blkpre, nb, ldk, n, S.colptr);
  k_scan_colptr<<<1, 1024, 0, st>>>(n, S.colptr);
  note_launch(4);
  const size_t smem = (size_t)n * sizeof(int32_t);
  static bool attr_set[2] = {false, false};
  if (fp64) {
    if (!attr_set[1]) {
      cudaFuncSetAttribute(k_scatter<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      attr_set[1] = true;
    }
    k_scatter<double><<<nb, 256, smem, st>>>(S.pool_col, (const double*)S.pool_val, S.row_start, S.row_len,
                                             S.blkpre, S.colptr, S.csc_row, (double*)S.csc_val, m, n, ldk, rpb);
    k_colstats<double><<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(
        S.colptr, S.csc_row, (const double*)S.csc_val, (const double*)S.prow, a, istar, n, eta, S.crho, S.diag);
  } else {
    if (!attr_set[0]) {
      cudaFuncSetAttribute(k_scatter<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      attr_set[0] = true;
    }
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

template <typename T>
static cudaError_t launch_pcg_t(const SparseBufs& S, const PcgBufs& B, int m, int64_t n, int istar,
                                const double* a, double eta, double shift, double rtol, int maxit, double timeout_s,
                                int nsm, double* scal, cudaStream_t st) {
  static int occ = 0;
  if (occ == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg<T>, kPcgThreads, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorCooperativeLaunchTooLarge;
  }
  // one block per SM keeps the barrier short; never more than fit co-resident
  int nb = nsm;
  if (nb > nsm * occ) nb = nsm * occ;
  if (nb > pcg_max_blocks(nsm)) nb = pcg_max_blocks(nsm);
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
  A.x = B.x; A.r = B.r; A.z = B.z; A.p = B.p; A.q = B.q; A.w = B.w;
  A.part = B.part;
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
  // bound on each barrier wait, in nanoseconds of the GPU global timer
  A.deadline_ns = (unsigned long long)(timeout_s * 1e9);
  void* args[] = {(void*)&A};
  note_launch();
  return cudaLaunchCooperativeKernel((const void*)k_pcg<T>, dim3(nb), dim3(kPcgThreads), args, 0, st);
}

cudaError_t launch_pcg(const SparseBufs& S, const PcgBufs& B, int m, int64_t n, int istar, bool fp64,
                       const double* a, double eta, double shift, double rtol, int maxit, double timeout_s, int nsm,
                       double* scal, cudaStream_t st) {
  if (fp64) return launch_pcg_t<double>(S, B, m, n, istar, a, eta, shift, rtol, maxit, timeout_s, nsm, scal, st);
  return launch_pcg_t<float>(S, B, m, n, istar, a, eta, shift, rtol, maxit, timeout_s, nsm, scal, st);
}

}  // namespace ibsn
