// Launch-configuration choice and dispatch for the dense passes.  Included by
// one translation unit per pass precision.
#pragma once

#include <mutex>
#include <type_traits>

#include "dense.cuh"

namespace ibsn {

template <typename T, int TG, int CH>
static const void* dense_kernel(Pass p) {
  switch (p) {
    case Pass::Plan: return (const void*)k_plan<T, TG, CH>;
    case Pass::Armijo: return (const void*)k_armijo<T, TG, CH>;
    case Pass::Stop: return (const void*)k_stop<T, TG, CH>;
    case Pass::Sparsify: return (const void*)k_sparsify<T, TG, CH>;
    case Pass::Certify: return (const void*)k_certify<T, TG, CH>;
    case Pass::Reanchor: return (const void*)k_reanchor<T, TG, CH>;
    case Pass::Export: return (const void*)k_export<T, TG, CH>;
    default: return nullptr;
  }
}

static bool pass_uses_colacc(Pass p) {
  return p == Pass::Plan || p == Pass::Armijo || p == Pass::Certify;
}

// Register-tile configurations, smallest first: capacity TG * CH * V columns.
template <typename T>
struct TileTable;
template <>
struct TileTable<float> {
  static constexpr int count = 6;
  static constexpr int tg[count] = {64, 128, 128, 256, 256, 512};
  static constexpr int ch[count] = {1, 2, 4, 4, 8, 8};
};
template <>
struct TileTable<double> {
  static constexpr int count = 6;
  static constexpr int tg[count] = {64, 128, 256, 256, 512, 1024};
  static constexpr int ch[count] = {2, 4, 4, 8, 8, 8};
};

// Shared memory a float pass may give its ring of row buffers.  A 16384-wide
// float row is 64 KiB; two buffers (two copies in flight) measured fastest:
// a third (192 KiB) left too little L1 for the per-column vectors the passes
// read with every row (plan pass 3966 against 4674 GB/s).
constexpr size_t kRowRingSmemMax = 160 * 1024;

// The stop-test pass holds no column accumulators, so its float tiles take
// twice the threads (half the chunks per thread) from the third configuration
// on: same row capacity, twice the warps to hide its latency.
struct StopTileTable {
  static constexpr int count = 6;
  static constexpr int tg[count] = {64, 128, 256, 512, 512, 1024};
  static constexpr int ch[count] = {1, 2, 2, 2, 4, 4};
};

template <typename T>
static int pick_tile(int64_t n) {
  for (int q = 0; q < TileTable<T>::count; ++q)
    if ((int64_t)TileTable<T>::tg[q] * TileTable<T>::ch[q] * VecT<T>::N >= n) return q;
  return -1;
}

template <typename T>
static const void* kernel_for(int q, Pass p) {
  if (std::is_same<T, float>::value && p == Pass::Stop) {
    using ST = StopTileTable;
    switch (q) {
      case 0: return (const void*)k_stop<T, ST::tg[0], ST::ch[0]>;
      case 1: return (const void*)k_stop<T, ST::tg[1], ST::ch[1]>;
      case 2: return (const void*)k_stop<T, ST::tg[2], ST::ch[2]>;
      case 3: return (const void*)k_stop<T, ST::tg[3], ST::ch[3]>;
      case 4: return (const void*)k_stop<T, ST::tg[4], ST::ch[4]>;
      case 5: return (const void*)k_stop<T, ST::tg[5], ST::ch[5]>;
      default: return nullptr;
    }
  }
  switch (q) {
    case 0: return dense_kernel<T, TileTable<T>::tg[0], TileTable<T>::ch[0]>(p);
    case 1: return dense_kernel<T, TileTable<T>::tg[1], TileTable<T>::ch[1]>(p);
    case 2: return dense_kernel<T, TileTable<T>::tg[2], TileTable<T>::ch[2]>(p);
    case 3: return dense_kernel<T, TileTable<T>::tg[3], TileTable<T>::ch[3]>(p);
    case 4: return dense_kernel<T, TileTable<T>::tg[4], TileTable<T>::ch[4]>(p);
    case 5: return dense_kernel<T, TileTable<T>::tg[5], TileTable<T>::ch[5]>(p);
    default: return nullptr;
  }
}

template <typename T>
int dense_max_blocks_t(int64_t n, int nsm) {
  const int q = pick_tile<T>(n);
  if (q < 0) return 0;
  return nsm * (2048 / TileTable<T>::tg[q]);
}

template <typename T>
cudaError_t launch_dense_t(Pass p, DenseArgs<T>& A, int nsm, cudaStream_t st, PassGeom* geom) {
  const int q = pick_tile<T>(A.n);
  if (q < 0) return cudaErrorInvalidValue;
  const void* fn = kernel_for<T>(q, p);
  const bool stop_tile = std::is_same<T, float>::value && p == Pass::Stop;
  const int tg = stop_tile ? StopTileTable::tg[q] : TileTable<T>::tg[q];
  // float64 passes: column accumulator; float passes: the row buffer of the row stream
  size_t smem = 0;
  if (std::is_same<T, double>::value) {
    if (pass_uses_colacc(p)) smem = (size_t)A.ldk * sizeof(double);
  } else if (p != Pass::Reanchor) {
    // as many row copies in flight per block (up to three) as the ring's budget holds
    const size_t row = (size_t)A.ldk * sizeof(float);
    A.stages = 3 * row <= kRowRingSmemMax ? 3 : (2 * row <= kRowRingSmemMax ? 2 : 1);
    smem = (size_t)A.stages * (size_t)A.ldk * sizeof(float);
  }
  // one-time opt-in to large dynamic shared memory, and cached occupancy
  static std::mutex mu;
  static int occ_cache[TileTable<T>::count][(int)Pass::kCount] = {};
  static size_t smem_set[TileTable<T>::count][(int)Pass::kCount] = {};
  int occ;
  {
    std::lock_guard<std::mutex> lk(mu);
    cudaError_t e;
    if (smem > smem_set[q][(int)p]) {
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      smem_set[q][(int)p] = smem;
      occ_cache[q][(int)p] = 0;
    }
    occ = occ_cache[q][(int)p];
    if (occ == 0) {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, tg, smem);
      if (e != cudaSuccess) return e;
      if (occ < 1) occ = 1;
      occ_cache[q][(int)p] = occ;
    }
  }
  int nb = nsm * occ;
  const int cap = dense_max_blocks_t<T>(A.n, nsm);
  if (nb > cap) nb = cap;
  if (nb > A.m) nb = A.m;
  int rpb = (A.m + nb - 1) / nb;
  nb = (A.m + rpb - 1) / rpb;
  A.rows_per_block = rpb;
  void* args[] = {(void*)&A};
  cudaError_t e = cudaLaunchKernel(fn, dim3(nb), dim3(tg), args, smem, st);
  note_launch();
  if (geom) {
    geom->tg = tg;
    geom->ch = stop_tile ? StopTileTable::ch[q] : TileTable<T>::ch[q];
    geom->nb = nb;
    geom->rpb = rpb;
    geom->smem = smem;
  }
  return e;
}


// ---- float-float passes (float tile table; instantiated in one translation unit) ----
#ifdef IBSN_FF_PASSES
template <int TG, int CH, int KIND>
static const void* ff_kernel_k(Pass p) {
  switch (p) {
    case Pass::Certify: return (const void*)k_certify_ff<TG, CH, KIND>;
    case Pass::Reanchor: return (const void*)k_reanchor_ff<TG, CH, KIND>;
    default: return nullptr;
  }
}

template <int TG, int CH>
static const void* ff_kernel(Pass p, int kind) {
  switch (p) {
    case Pass::Plan: return (const void*)k_plan_ff<TG, CH>;
    case Pass::Armijo: return (const void*)k_armijo_ff<TG, CH>;
    case Pass::Export: return (const void*)k_export_ff<TG, CH>;
    default:
      if (kind == 0) return ff_kernel_k<TG, CH, 0>(p);
      if (kind == 1) return ff_kernel_k<TG, CH, 1>(p);
      if (kind == 3) return ff_kernel_k<TG, CH, 3>(p);
      return ff_kernel_k<TG, CH, 2>(p);
  }
}

static const void* ff_kernel_for(int q, Pass p, int kind) {
  using TT = TileTable<float>;
  switch (q) {
    case 0: return ff_kernel<TT::tg[0], TT::ch[0]>(p, kind);
    case 1: return ff_kernel<TT::tg[1], TT::ch[1]>(p, kind);
    case 2: return ff_kernel<TT::tg[2], TT::ch[2]>(p, kind);
    case 3: return ff_kernel<TT::tg[3], TT::ch[3]>(p, kind);
    case 4: return ff_kernel<TT::tg[4], TT::ch[4]>(p, kind);
    case 5: return ff_kernel<TT::tg[5], TT::ch[5]>(p, kind);
    default: return nullptr;
  }
}

inline cudaError_t launch_dense_ff_t(Pass p, DenseArgs<float>& A, int nsm, cudaStream_t st, PassGeom* geom) {
  A.stages = 1;  // the float64 column accumulator follows the single row buffer
  const int q = pick_tile<float>(A.n);
  if (q < 0) return cudaErrorInvalidValue;
  const void* fn = ff_kernel_for(q, p, A.cost.kind);
  if (fn == nullptr) return cudaErrorInvalidValue;
  const int tg = TileTable<float>::tg[q];
  // row buffer of the row stream, then the float64 column accumulator
  const size_t smem = p == Pass::Reanchor ? 0
                      : (size_t)A.ldk * sizeof(float) + (p == Pass::Export ? 0 : (size_t)A.ldk * sizeof(double));
  static std::mutex mu;
  const int kk = (A.cost.kind >= 0 && A.cost.kind <= 3) ? A.cost.kind : 2;
  static int occ_cache[TileTable<float>::count][(int)Pass::kCount][4] = {};
  static size_t smem_set[TileTable<float>::count][(int)Pass::kCount][4] = {};
  int occ;
  {
    std::lock_guard<std::mutex> lk(mu);
    cudaError_t e;
    if (smem > smem_set[q][(int)p][kk]) {
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      smem_set[q][(int)p][kk] = smem;
      occ_cache[q][(int)p][kk] = 0;
    }
    occ = occ_cache[q][(int)p][kk];
    if (occ == 0) {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, tg, smem);
      if (e != cudaSuccess) return e;
      if (occ < 1) occ = 1;
      occ_cache[q][(int)p][kk] = occ;
    }
  }
  int nb = nsm * occ;
  const int cap = dense_max_blocks_t<float>(A.n, nsm);
  if (nb > cap) nb = cap;
  if (nb > A.m) nb = A.m;
  int rpb = (A.m + nb - 1) / nb;
  nb = (A.m + rpb - 1) / rpb;
  A.rows_per_block = rpb;
  void* args[] = {(void*)&A};
  cudaError_t e = cudaLaunchKernel(fn, dim3(nb), dim3(tg), args, smem, st);
  note_launch();
  if (geom) {
    geom->tg = tg;
    geom->ch = TileTable<float>::ch[q];
    geom->nb = nb;
    geom->rpb = rpb;
    geom->smem = smem;
  }
  return e;
}

#endif  // IBSN_FF_PASSES

}  // namespace ibsn
