// Internal interfaces between the host control code and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace ibsn {

// Kernels launched by this library (all threads, all contexts).
inline std::atomic<long long> g_launches{0};
inline void note_launch(int k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

constexpr int kRowParts = 8;        // per-block row-partial slots of a dense pass
constexpr int kMaxN = 16384;        // widest row the register tiles cover

// Cost access for the passes that read C (anchor build, certificate).
struct CostRef {
  const void* C;
  int64_t ldc;
  int kind;      // ibsn_cost_kind
  int gw;        // grid width (GRID2D)
  double scale;  // GRID2D / SQEUCLID_POINTS scale
  const int* rc; // GRID2D: bin coordinates packed as row | col << 16 (n entries), or null
  // SQEUCLID_POINTS: C_ij = scale * ||x_i - y_j||^2 with x (m x dim) and y (n x dim)
  // row-major float64; xs / ys hold every coordinate as a float pair (hi, lo)
  // with hi + lo = the float64 value to 2^-48 (null: not set up)
  const double* px;
  const double* py;
  const float2* xs;
  const float2* ys;
  int dim;
};

constexpr int kMaxPointDim = 16;    // coordinates per point of the on-the-fly point cost

enum class Pass : int { Plan = 0, Armijo, Stop, Sparsify, Certify, Reanchor, Export, kCount };

template <typename T>
struct DenseArgs;

// Geometry of one dense-pass launch.
struct PassGeom {
  int tg = 0, ch = 0;   // threads per block, chunks per thread
  int nb = 0;           // blocks
  int rpb = 0;          // rows per block
  size_t smem = 0;      // dynamic shared memory
  bool ffpart = false;  // column partials are float-float pairs (float passes)
};

// Leading dimension of the anchored matrix: n rounded up to 32 elements.
inline int64_t ldk_for(int64_t n) { return (n + 31) / 32 * 32; }

// Upper bound on the blocks of any dense pass for this n and type (sizes the
// per-block partial buffers); 0 when n is outside the tile table.
int dense_max_blocks_f32(int64_t n, int nsm);
int dense_max_blocks_f64(int64_t n, int nsm);

template <typename T>
cudaError_t launch_dense(Pass p, DenseArgs<T>& A, int nsm, cudaStream_t st, PassGeom* geom);
template <>
cudaError_t launch_dense<float>(Pass p, DenseArgs<float>& A, int nsm, cudaStream_t st, PassGeom* geom);
template <>
cudaError_t launch_dense<double>(Pass p, DenseArgs<double>& A, int nsm, cudaStream_t st, PassGeom* geom);
// float-float passes (Plan, Armijo, Certify, Export) over the hi/lo float planes
cudaError_t launch_dense_ff(Pass p, DenseArgs<float>& A, int nsm, cudaStream_t st, PassGeom* geom);

}  // namespace ibsn

namespace ibsn {

// Scalar slots (float64) written by kernels and read back by the host.
enum Slot : int {
  S_GN2 = 0,       // ||g||^2
  S_ROW0 = 1,      // .. S_ROW0 + kRowParts - 1: totals of a dense pass's row partials
  S_DMAX = 12,     // max_j |d_j|
  S_MEAN = 13,     // mean removed by a centring
  S_SLOPE = 14,    // g^T Delta
  S_DELTAMAX = 15, // max_j |Delta_j| / eta
  S_PHI = 16,      // sum_j c_j phi(t Delta_j / eta)
  S_ECSUM = 17,    // S = ||e_c||_1
  S_COLVIOL = 18,  // sum_j |Xhat^T 1 - b|_j
  S_BGAM = 19,     // b^T gamma
  S_AMIN = 20, S_ASUM = 21, S_BMIN = 22, S_BSUM = 23, S_ABAD = 24,
  S_CBAD = 25,     // C check: count of negative or non-finite entries
  S_CG_ITERS = 26, S_CG_RES = 27,
  S_NNZ = 28,
  S_MAXROW = 29, S_MAXCOL = 30,  // longest row / column of P_rho (diagnostics)
  S_CMAX = 31, S_GMAX = 32,      // max C_ij, max_j |gamma_j| (adjacent: certificate bounds)
  S_TMP = 33,                    // scratch total between two kernels of one step
  S_DEVERR = 34,                 // nonzero: a bounded device wait of a dense pass ran out
  S_W0 = 40,                     // .. S_W0 + 3: moments of w = e_c / S over the grid (sum w, sum r w, sum c w, sum (r^2 + c^2) w)
  S_C2SUM = 44,                  // sum_ij C_ij^2 (once per context)
  S_NSLOTS = 64
};

// Counter slots (unsigned) for last-block reductions and barriers.
enum Counter : int { C_FINISH = 0, C_BAR_COUNT = 1, C_BAR_GEN = 2, C_POOL_LO = 4, C_NCOUNTERS = 16 };

// Scratch of the multi-block O(n) reductions: a counter (zero between kernels)
// and room for K block results per block.
struct RedBuf {
  unsigned int* counter;
  double* blockbuf;
};
cudaError_t launch_finish_cols(const double* colpart, bool ffpart, int nb, int64_t ldk, int64_t n, const double* b,
                               double* c_out, double* g_out, const double* rowpart, int nrp, double* scal,
                               const RedBuf& rb, cudaStream_t st);

// single-block vector kernels; `dT` is float or double per `fp64`
cudaError_t launch_rows_ff(int64_t m, bool armijo, const double* a, const double* S0, const double* S1,
                           const double* M, double* rowout, double* scal, const RedBuf& rb, cudaStream_t st);
cudaError_t launch_set_anchor(int64_t n, int64_t ldk, double eta, const double* Gam, double* gam, double* ganc,
                              const double* logb, double* wv, float* wvh, float* wvl, double* dd, float* d32,
                              float* dlo, double* d64, cudaStream_t st);
cudaError_t launch_sinkhorn_update(int64_t n, double eta, const double* b, const double* c, double* gam,
                                   const double* ganc, double* dd, float* d32, float* dlo, double* d64, bool fp64,
                                   double* scal, const RedBuf& rb, cudaStream_t st);
cudaError_t launch_center(int64_t n, double eta, double* gam, const double* ganc, double* dd, float* d32,
                          float* dlo, double* d64, double* scal, const RedBuf& rb, cudaStream_t st);
cudaError_t launch_dir_post(int64_t n, double eta, double* delta, const double* g, double* scal, const RedBuf& rb,
                            cudaStream_t st);
cudaError_t launch_armijo_prep(int64_t n, int64_t ldk, double eta, double t, const double* delta, const double* c,
                               float* em32, float* emlo, double* em64, double* scal, const RedBuf& rb,
                               cudaStream_t st);
cudaError_t launch_armijo_accept(int64_t n, double eta, double t, const double* delta, double* gam,
                                 const double* ganc, double* dd, float* d32, float* dlo, double* d64,
                                 const double* cnew, const double* b, double* g, double* scal, const RedBuf& rb,
                                 cudaStream_t st);
// per-column rounding inputs, written in float and float64: y, omega, e_c, e_c / S
struct RoundVecs {
  float *y32, *om32, *ec32, *ecs32, *lec32;
  float* ecsl32;  // e_c / S - fl32(e_c / S): the float-float lo part
  float *ylo32, *omlo32;  // lo parts of y and omega
  float* hom32;   // (1 - omega) log(1 - omega) + omega
  double* hom64;
  double *y64, *om64, *ec64, *ecs64, *lec64;  // lec = log e_c (-inf where e_c = 0)
};
cudaError_t launch_round_prep(int64_t n, const double* b, const double* c, const double* g, const RoundVecs& R,
                              const int* grid_rc, double* scal, const RedBuf& rb, cudaStream_t st);
cudaError_t launch_grid_rc(int64_t n, int gw, int* rc, cudaStream_t st);
cudaError_t launch_rows_cert(int64_t m, const double* a, const double* rowbuf, const int* grid_rc, double scale,
                             double* zeta_out, double* er_out, double* scal, const RedBuf& rb, cudaStream_t st);
cudaError_t launch_certify_cols(int64_t n, const double* b, const double* colF, const double* c, const double* gam,
                                double ersum, double* scal, const RedBuf& rb, cudaStream_t st);
cudaError_t launch_validate_marginals(int64_t m, int64_t n, const double* a, const double* b, double* scal,
                                      cudaStream_t st);
cudaError_t launch_split_coords(int64_t count, const double* x, float2* out, cudaStream_t st);
// zeta_i = min_j C_ij - gamma_j for the h x w grid cost C = s * squared bin distance
// (hmin: h*w doubles of scratch)
cudaError_t launch_ctransform_grid(int h, int w, double s, const double* gam, double* hmin, double* zeta,
                                   cudaStream_t st);
cudaError_t launch_validate_cost(int64_t m, int64_t n, const void* C, int64_t ldc, int kind, const double* px,
                                 const double* py, int dim, double scale, double* scal,
                                 cudaStream_t st);
cudaError_t launch_certify_prep(int64_t n, const double* gam, float* gam32, float* gamlo, double* scal,
                                const RedBuf& rb, cudaStream_t st);
cudaError_t launch_set_slot(double* scal, int slot, double v, cudaStream_t st);
cudaError_t launch_fill_pad(void* v, int64_t n, int64_t ldk, bool fp64, double value, cudaStream_t st);
cudaError_t launch_neg(int64_t n, const double* x, double* y, cudaStream_t st);

// sparse side
struct SparseBufs {
  int32_t* pool_col;
  void* pool_val;
  int64_t* row_start;
  int32_t* row_len;
  int32_t* blkcnt;      // nb x ldk
  int32_t* blkpre;      // nb x ldk
  int64_t* colptr;      // n + 1
  int32_t* csc_row;
  void* csc_val;
  void* prow;           // row i* (n)
  double* crho;         // n
  double* diag;         // n (without shift)
  int64_t cap;
};

cudaError_t launch_csc_build(const SparseBufs& S, int m, int64_t n, int64_t ldk, int nb, int rpb, bool fp64,
                             const double* a, int istar, double eta, cudaStream_t st);
cudaError_t launch_export_sparse(const SparseBufs& S, int m, int64_t n, int istar, bool fp64, double* out,
                                 cudaStream_t st);

struct PcgBufs {
  double *x, *p, *rhs;  // n
  double* cs;           // 4n: packed column state {r, w, s, 1/diag}
  float* cs32;          // 4n floats: float copy of the packed state
  double* t;            // m (float or double values)
  double* part;         // 8 x maxblocks (float-float partials of 6 sums)
  unsigned int* bar;    // [count, gen]
  int* err;
};

// PCG on one thread-block cluster (float32 Hessian, m, n <= 16 x 1024): sets
// *launched when it ran; *err = kDevCapacity afterwards means the staged
// entries did not fit and nothing was computed.
cudaError_t launch_pcg_cluster(const SparseBufs& S, const PcgBufs& B, int m, int64_t n, int istar, const float* a32,
                               double eta, double shift, double rtol, int maxit, double* scal, cudaStream_t st,
                               bool* launched);
cudaError_t launch_pcg(const SparseBufs& S, const PcgBufs& B, int m, int64_t n, int istar, bool fp64,
                       const double* a, const float* a32, double eta, double shift, double rtol, int maxit,
                       double timeout_s, int nsm, int64_t nnz, double* scal, cudaStream_t st);
int pcg_max_blocks(int nsm);
cudaError_t launch_len_stats(const SparseBufs& S, int m, int64_t n, double* scal, cudaStream_t st);

// Semi-dual objective at k = 0 (Eq. 5 with X^0 = a b^T):
//   L^0(gamma) = -b^T gamma + eta sum_i a_i log sum_j a_i b_j exp((gamma_j - C_ij)/eta),
// float64 throughout; gamma nullable (zero).  rowval: m doubles of scratch;
// the value is written to *out (device).
cudaError_t launch_semidual0(const CostRef& cost, int m, int64_t n, double eta, const double* a, const double* b,
                             const double* logb, const double* gamma, double* rowval, double* out, cudaStream_t st);

}  // namespace ibsn
