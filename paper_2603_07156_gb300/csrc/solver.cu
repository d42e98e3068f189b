// Host control of IBSN (Alg. 2) and the C ABI declared in include/ibsn.h.
//
// State of one run (the "context"): outer index k, cumulative potential
// Gamma^k, current potential gamma, anchor potential gamma^anc and the
// anchored exponent matrix K (float32 or float64).  By induction on the outer
// update X^{k+1} = diag(a) P^k(gamma^{k,fin}) from X^0 = a b^T,
//   log X^k_ij + (gamma_j - C_ij)/eta = s_i + log b_j + (Gamma^k_j + gamma_j - (k+1) C_ij)/eta
// for row constants s_i that P^k does not see, so the outer update is the
// vector add Gamma^{k+1} = Gamma^k + gamma^{k,fin} followed by one anchor pass.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ibsn.h"
#include "dense.cuh"
#include "internal.h"

using namespace ibsn;

namespace {

thread_local std::string g_last_cuda_error;

constexpr double kReanchorF32 = 16.0;   // max |d_j| before a float32 anchor is rebuilt
constexpr double kReanchorF64 = 1e6;
// nonzeros up to which a direction is first tried on one thread-block cluster
constexpr int64_t kClusterPcgMaxNnz = 160000;

struct Carver {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) / 256 * 256;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += std::max<size_t>(count, 1) * sizeof(T);
    return p;
  }
};

__global__ void k_log(int64_t n, const double* x, double* y) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) y[j] = log(x[j]);
}
__global__ void k_to_float(int64_t n, const double* x, float* y) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) y[j] = (float)x[j];
}
__global__ void k_lo_float(int64_t n, const double* x, float* y) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) y[j] = (float)(x[j] - (double)(float)x[j]);
}
__global__ void k_axpy(int64_t n, double alpha, const double* x, double* y) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) y[j] += alpha * x[j];
}

__global__ void k_add_const(int64_t n, double v, double* x) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) x[j] += v;
}

cudaError_t launch_add_const(int64_t n, double v, double* x, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_add_const<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, v, x);
  note_launch();
  return cudaGetLastError();
}

int device_sm_count() {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm > 0 ? nsm : 1;
}

}  // namespace

// Optional per-step device timing with CUDA events on the solve's stream.
struct Profiler {
  bool on = false;
  struct Pending {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> pool;
  std::vector<Pending> pend;
  double ms[16] = {};
  long long calls[16] = {};
  double bytes[16] = {};
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  // events of completed steps are read after a stream synchronisation
  void harvest() {
    for (const Pending& p : pend) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) ms[p.kind] += t;
      calls[p.kind] += 1;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pend.clear();
  }
  ~Profiler() {
    for (const Pending& p : pend) {
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

struct ibsn_ctx {
  Profiler prof;
  // problem
  int m = 0;
  int64_t n = 0, ldk = 0;
  CostRef cost{};
  const double *a = nullptr, *b = nullptr;
  double eta = 0;
  ibsn_params prm{};
  cudaStream_t st = nullptr;
  int nsm = 1;
  int istar = 0;
  bool have_f32 = false, have_f64 = false, have_ff = false;
  bool recompute = false;  // no stored anchored matrix (params.recompute)
  double lam = 0.0;        // (k+1)/eta of the current anchor
  // state
  int64_t k = 0;
  int prec = 0;            // 0 float64 passes, 1 float32 passes, 2 float-float polish
  bool have_dir = false;
  int sp_nb = 0, sp_rpb = 0;
  bool sp_f64 = false;     // value type of the current sparsified Hessian
  double anorm = 0.0, bnorm = 0.0;
  int64_t nnz = 0;
  double gn = 0.0;         // ||g|| at the current gamma
  int64_t dense_passes = 0;
  int reanchors = 0;
  int64_t cl_fail_nnz = INT64_MAX;  // smallest nnz whose cluster PCG did not fit
  int64_t cl_runs = 0;              // directions solved by the cluster PCG
  // device buffers
  float* K32 = nullptr;     // float anchored matrix (hi plane in the polish)
  float* Klo = nullptr;     // lo plane of the float-float anchored matrix
  double* K64 = nullptr;    // float64 anchored matrix (plain float64 mode)
  double *Gam, *gam, *ganc, *dd, *c, *c2, *g, *delta, *logb, *wv, *colF;
  double *lse, *lse2, *er, *zeta, *zgrid;
  double *rowS0, *rowS1, *rowM;  // per-row results of the float-float passes
  double* rowbuf;                // 6 x m per-row results of the float-float certificate
  int* gridrc;                   // grid cost: bin coordinates per column (null otherwise)
  float2 *xs, *ys;               // point cost: coordinates as float pairs (null otherwise)
  float* alo32;                  // a - fl32(a)
  float* rowMa;                  // anchor row shifts (recompute mode)
  float *d32, *em32, *a32, *gam32, *wvh, *wvl;
  float *dlo32, *emlo32, *gamlo32;  // float-float lo parts
  double *d64, *em64;
  RoundVecs rv{};
  double *colpart, *rowpart, *blockbuf;
  SparseBufs sp{};
  PcgBufs pc{};
  double* scal = nullptr;
  unsigned int* ctr = nullptr;
  int* err = nullptr;
  unsigned long long* pool_top = nullptr;
  double* h_scal = nullptr;  // pinned copy of scal (slots), then one int for the PCG error flag
  int* h_perr = nullptr;
  int nbcap = 0;
};

namespace {

int set_cuda_error(cudaError_t e) {
  g_last_cuda_error = cudaGetErrorString(e);
  return IBSN_ERR_CUDA;
}

#define CK(expr)                                    \
  do {                                              \
    cudaError_t e_ = (expr);                        \
    if (e_ != cudaSuccess) return set_cuda_error(e_); \
  } while (0)
#define RT(expr)                     \
  do {                               \
    int r_ = (expr);                 \
    if (r_ != IBSN_OK) return r_;    \
  } while (0)

bool fp32_capable(const ibsn_params* p) { return p->precision == IBSN_PREC_MIXED; }
bool fp64_needed(const ibsn_params* p) { return p->precision == IBSN_PREC_FP64; }
bool ff_needed(const ibsn_params* p) { return p->precision == IBSN_PREC_MIXED && p->polish; }

int check_problem(const ibsn_problem* pr) {
  if (!pr) return IBSN_ERR_INVALID_ARG;
  if (pr->m < 1 || pr->n < 1 || !(pr->eta > 0.0) || !std::isfinite(pr->eta)) return IBSN_ERR_INVALID_ARG;
  if (!pr->a || !pr->b) return IBSN_ERR_INVALID_ARG;
  if (pr->m > (int64_t)0x7fffffff) return IBSN_ERR_UNSUPPORTED;
  if (pr->n > kMaxN) return IBSN_ERR_UNSUPPORTED;
  switch (pr->cost_kind) {
    case IBSN_COST_DENSE_F64:
    case IBSN_COST_DENSE_F32:
      if (!pr->C || pr->ldc < pr->n) return IBSN_ERR_INVALID_ARG;
      break;
    case IBSN_COST_GRID2D:
      if (pr->grid_h < 1 || pr->grid_w < 1 || (int64_t)pr->grid_h * pr->grid_w != pr->m || pr->m != pr->n)
        return IBSN_ERR_INVALID_ARG;
      if (!(pr->cost_scale >= 0.0) || !std::isfinite(pr->cost_scale)) return IBSN_ERR_NONFINITE;
      break;
    case IBSN_COST_SQEUCLID_POINTS:
      if (!pr->x || !pr->y || pr->dim < 1) return IBSN_ERR_INVALID_ARG;
      if (pr->dim > kMaxPointDim) return IBSN_ERR_UNSUPPORTED;
      if (!(pr->cost_scale >= 0.0) || !std::isfinite(pr->cost_scale)) return IBSN_ERR_NONFINITE;
      break;
    default:
      return IBSN_ERR_INVALID_ARG;
  }
  return IBSN_OK;
}

// Lay out (or size, when base == nullptr) every device buffer of a context.
void carve(ibsn_ctx* X, Carver& cv, const ibsn_problem* pr, const ibsn_params* pp, int nsm) {
  const int64_t m = pr->m, n = pr->n, ldk = ldk_for(n);
  X->have_f32 = fp32_capable(pp);
  X->have_f64 = fp64_needed(pp);
  X->nbcap = std::max(fp32_capable(pp) ? dense_max_blocks_f32(n, nsm) : 0,
                      fp64_needed(pp) ? dense_max_blocks_f64(n, nsm) : 0);
  const int nbcap = X->nbcap;
  const int64_t cap = pp->nnz_cap > 0 ? pp->nnz_cap : m * n;
  X->have_ff = ff_needed(pp);
  X->recompute = pp->recompute != 0 && X->have_f32;
  X->K32 = X->have_f32 && !X->recompute ? cv.take<float>((size_t)m * ldk) : nullptr;
  X->Klo = X->have_ff && !X->recompute ? cv.take<float>((size_t)m * ldk) : nullptr;
  X->rowMa = cv.take<float>(m);
  X->K64 = X->have_f64 ? cv.take<double>((size_t)m * ldk) : nullptr;
  double** nvec[] = {&X->Gam, &X->gam, &X->ganc, &X->dd, &X->c, &X->c2, &X->g, &X->delta, &X->logb, &X->wv, &X->colF};
  for (double** v : nvec) *v = cv.take<double>(n);
  double** mvec[] = {&X->lse, &X->lse2, &X->er, &X->zeta, &X->zgrid, &X->rowS0, &X->rowS1, &X->rowM};
  for (double** v : mvec) *v = cv.take<double>(m);
  X->a32 = cv.take<float>(m);
  X->alo32 = cv.take<float>(m);
  X->rowbuf = cv.take<double>(6 * (size_t)m);
  X->gridrc = pr->cost_kind == IBSN_COST_GRID2D ? cv.take<int>(n) : nullptr;
  const bool pts = pr->cost_kind == IBSN_COST_SQEUCLID_POINTS;
  X->xs = pts ? cv.take<float2>((size_t)m * pr->dim) : nullptr;
  X->ys = pts ? cv.take<float2>((size_t)n * pr->dim) : nullptr;
  float** fvec[] = {&X->d32,      &X->em32,      &X->gam32,      &X->rv.y32,   &X->rv.om32, &X->rv.ec32,
                    &X->rv.ecs32, &X->rv.ecsl32, &X->rv.lec32, &X->wvh,      &X->wvl, &X->rv.hom32,
                    &X->dlo32,    &X->emlo32,    &X->gamlo32,    &X->rv.ylo32, &X->rv.omlo32};
  for (float** v : fvec) *v = cv.take<float>(ldk);
  double** dvec[] = {&X->d64,       &X->em64,       &X->rv.y64,     &X->rv.om64,
                     &X->rv.ec64,   &X->rv.ecs64,   &X->rv.lec64,   &X->rv.hom64};
  for (double** v : dvec) *v = cv.take<double>(ldk);
  X->colpart = cv.take<double>((size_t)nbcap * ldk);
  X->rowpart = cv.take<double>((size_t)nbcap * kRowParts);
  X->blockbuf = cv.take<double>(8 * std::max((n + 31) / 32, (m + 255) / 256) + 8);
  X->sp.pool_col = cv.take<int32_t>(cap);
  X->sp.pool_val = cv.take<double>(cap);
  X->sp.row_start = cv.take<int64_t>(m);
  X->sp.row_len = cv.take<int32_t>(m);
  X->sp.blkcnt = cv.take<int32_t>((size_t)nbcap * ldk);
  X->sp.blkpre = cv.take<int32_t>((size_t)nbcap * ldk);
  X->sp.colptr = cv.take<int64_t>(n + 1);
  X->sp.csc_row = cv.take<int32_t>(cap);
  X->sp.csc_val = cv.take<double>(cap);
  X->sp.prow = cv.take<double>(n);
  X->sp.crho = cv.take<double>(n);
  X->sp.diag = cv.take<double>(n);
  X->sp.cap = cap;
  double** pvec[] = {&X->pc.x, &X->pc.p, &X->pc.rhs};
  for (double** v : pvec) *v = cv.take<double>(n);
  X->pc.cs = cv.take<double>(4 * (size_t)n);
  X->pc.cs32 = cv.take<float>(4 * (size_t)n);
  X->pc.t = cv.take<double>(m);
  X->pc.part = cv.take<double>(8 * (size_t)pcg_max_blocks(nsm));
  X->pc.bar = cv.take<unsigned int>(4);
  X->pc.err = cv.take<int>(4);
  X->scal = cv.take<double>(S_NSLOTS);
  X->ctr = cv.take<unsigned int>(C_NCOUNTERS);
  X->err = cv.take<int>(4);
  X->pool_top = cv.take<unsigned long long>(2);
}

RedBuf rb(ibsn_ctx* X) { return RedBuf{X->ctr + C_FINISH, X->blockbuf}; }

int read_scal(ibsn_ctx* X) {
  CK(cudaMemcpyAsync(X->h_scal, X->scal, sizeof(double) * S_NSLOTS, cudaMemcpyDeviceToHost, X->st));
  CK(cudaStreamSynchronize(X->st));
  if (X->prof.on) X->prof.harvest();
  if (X->h_scal[S_DEVERR] != 0.0) return IBSN_ERR_TIMEOUT;  // a dense pass's bounded wait ran out
  return IBSN_OK;
}

// Brackets one step of kind `kind` with CUDA events when profiling is on.
struct ProfScope {
  ibsn_ctx* X;
  int kind;
  cudaEvent_t a = nullptr;
  ProfScope(ibsn_ctx* x, int k, double bytes, bool hi) : X(x), kind(k + (hi ? 8 : 0)) {
    if (X->prof.on) {
      X->prof.bytes[kind] += bytes;
      a = X->prof.get();
      cudaEventRecord(a, X->st);
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = X->prof.get();
      cudaEventRecord(b, X->st);
      X->prof.pend.push_back({kind, a, b});
    }
  }
};

int pass_kind(Pass p) {
  switch (p) {
    case Pass::Plan: return 0;
    case Pass::Armijo: return 1;
    case Pass::Stop: return 2;
    case Pass::Sparsify: return 3;
    case Pass::Certify: return 4;
    case Pass::Reanchor: return 5;
    default: return 7;
  }
}

// How a dense pass is evaluated under the context's precision.
enum class Mode { F32, F64, FF };

Mode mode_for(const ibsn_ctx* X, Pass p) {
  if (X->prec == 0) return Mode::F64;
  // the certificate uses the float-float kernel in both float modes (without
  // a lo plane in float32 mode: the entries are then those of float32 K)
  if (X->prec == 1) return p == Pass::Certify ? Mode::FF : Mode::F32;
  // float-float polish: the passes that produce the gradient, the Armijo
  // decrease and the certificate are float64-accurate; the Hessian model
  // (sparsify) and the stop test read the float hi plane
  if (p == Pass::Plan || p == Pass::Armijo || p == Pass::Certify || p == Pass::Export) return Mode::FF;
  return Mode::F32;
}

// Inputs of one dense pass beyond the common ones.
struct PassIn {
  const float *v1f = nullptr, *v2f = nullptr, *v3f = nullptr, *v4f = nullptr;
  const float *v1lo = nullptr, *v2lo = nullptr;
  const double *v1d = nullptr, *v2d = nullptr, *v3d = nullptr, *v4d = nullptr;
  double s1 = 0.0, s2 = 0.0;
  double *rowout = nullptr, *rowout2 = nullptr, *plan_out = nullptr;
  const double* gam = nullptr;
  const double* zeta_in = nullptr;
  bool sparsify = false, reanchor = false;
  double lam = 0.0;
};

template <typename T>
DenseArgs<T> make_args(ibsn_ctx* X, const PassIn& in) {
  DenseArgs<T> A;
  memset(&A, 0, sizeof(A));
  constexpr bool F = std::is_same<T, float>::value;
  if constexpr (F) {
    A.K = X->K32;
    A.dv = X->d32;
    A.v1 = in.v1f;
    A.v2 = in.v2f;
    A.v3 = in.v3f;
    A.v4 = in.v4f;
  } else {
    A.K = X->K64;
    A.dv = X->d64;
    A.v1 = in.v1d;
    A.v2 = in.v2d;
    A.v3 = in.v3d;
    A.v4 = in.v4d;
  }
  if constexpr (F) {
    A.aT = X->a32;
  } else {
    A.aT = X->a;
  }
  A.Klo = X->prec == 2 ? X->Klo : nullptr;  // the lo plane is maintained in the polish only
  A.dv64 = X->d64;
  A.v1d = in.v1d;
  A.v2d = in.v2d;
  A.v3d = in.v3d;
  A.ldk = X->ldk;
  A.m = X->m;
  A.n = (int)X->n;
  A.istar = X->istar;
  A.a = X->a;
  A.colpart = X->colpart;
  A.rowpart = X->rowpart;
  A.cost = X->cost;
  A.s1 = in.s1;
  A.s2 = in.s2;
  A.scal = X->scal;
  A.rowS0 = X->rowS0;
  A.rowS1 = X->rowS1;
  A.rowM = X->rowM;
  A.alo = X->alo32;
  A.rowbuf = X->rowbuf;
  A.dvlo = X->dlo32;
  A.v1lo = in.v1lo;
  A.v2lo = in.v2lo;
  A.gamlo = X->gamlo32;
  A.gam32 = X->gam32;
  A.v3lo = X->rv.ecsl32;
  A.bounds = X->scal + S_CMAX;
  A.rowout = in.rowout;
  A.rowout2 = in.rowout2;
  A.plan_out = in.plan_out;
  A.gam = in.gam;
  A.zeta_in = in.zeta_in;
  if (in.sparsify) {
    A.pool_col = X->sp.pool_col;
    A.pool_val = (T*)X->sp.pool_val;
    A.row_start = X->sp.row_start;
    A.row_len = X->sp.row_len;
    A.blkcnt = X->sp.blkcnt;
    A.prow = (T*)X->sp.prow;
    A.pool_top = X->pool_top;
    A.cap = X->sp.cap;
    A.err = X->err;
  }
  if (in.reanchor || X->recompute) {
    // the anchor-time w and lam: inputs of the anchor pass, and in recompute
    // mode of every pass (they rebuild K from them)
    const double lam = in.reanchor ? in.lam : X->lam;
    A.wv = X->wv;
    A.wvh = X->wvh;
    A.wvl = X->wvl;
    A.lam = lam;
    A.lamh = (float)lam;
    A.laml = (float)(lam - (double)A.lamh);
  }
  if (X->recompute) {
    A.recompute = 1;
    A.rc_lo = X->prec == 2 ? 1 : 0;
    A.rowMa = X->rowMa;
  }
  if (in.reanchor && !X->recompute) {
    if constexpr (F) {
      A.Kout = X->K32;
      A.Klo_out = X->prec == 2 ? X->Klo : nullptr;
    } else {
      A.Kout = X->K64;
    }
  }
  return A;
}

// algorithmic bytes of one dense pass (see ibsn_result.pass_bytes)
double pass_bytes(ibsn_ctx* X, Pass p, Mode md) {
  const double mn = (double)X->m * (double)X->n;
  // bytes of C read per entry: dense kinds only (grid and point costs are rebuilt on the fly)
  const double sc = X->cost.kind == 0 ? 8.0 : (X->cost.kind == 1 ? 4.0 : 0.0);
  const double sk = md == Mode::F64 ? 8.0 : (X->recompute ? 0.0 : 4.0);
  switch (p) {
    case Pass::Reanchor:
      return mn * ((X->recompute ? 0.0 : (X->prec == 2 ? 8.0 : (md == Mode::F64 ? 8.0 : 4.0))) + sc);
    case Pass::Certify: return mn * (sk + sc);
    default: return mn * sk;
  }
}

// Launch one dense pass in the mode the context's precision selects.
int run_pass(ibsn_ctx* X, Pass p, const PassIn& in, PassGeom* g = nullptr) {
  // the float anchor is built in float-float arithmetic (K32, and Klo in the polish)
  const Mode md = p == Pass::Reanchor ? (X->prec == 0 ? Mode::F64 : Mode::FF) : mode_for(X, p);
  if (g) g->ffpart = md != Mode::F64;  // float passes write float-float column partials
  ProfScope ps(X, pass_kind(p), pass_bytes(X, p, md), md != Mode::F32);
  if (md == Mode::F64) {
    DenseArgs<double> A = make_args<double>(X, in);
    CK(launch_dense<double>(p, A, X->nsm, X->st, g));
  } else {
    DenseArgs<float> A = make_args<float>(X, in);
    if (md == Mode::FF) CK(launch_dense_ff(p, A, X->nsm, X->st, g));
    else CK(launch_dense<float>(p, A, X->nsm, X->st, g));
  }
  X->dense_passes++;
  return IBSN_OK;
}

// finish a pass that wrote column partials: c_out = sum of partials, g = c - b
int finish(ibsn_ctx* X, const PassGeom& g, double* c_out, bool grad, int nrp) {
  CK(launch_finish_cols(X->colpart, g.ffpart, g.nb, X->ldk, X->n, grad ? X->b : nullptr, c_out, grad ? X->g : nullptr,
                        X->rowpart, nrp, X->scal, rb(X), X->st));
  return IBSN_OK;
}

// ---------------------------------------------------------------- steps ----

// a1: anchor build for the current (k, Gamma, gamma) in precision X->prec
int do_reanchor(ibsn_ctx* X) {
  CK(launch_set_anchor(X->n, X->ldk, X->eta, X->Gam, X->gam, X->ganc, X->logb, X->wv, X->wvh, X->wvl, X->dd,
                       X->d32, X->dlo32, X->d64, X->st));
  PassIn in;
  in.reanchor = true;
  in.lam = (double)(X->k + 1) / X->eta;
  X->lam = in.lam;
  RT(run_pass(X, Pass::Reanchor, in));
  X->reanchors++;
  return IBSN_OK;
}

int maybe_reanchor(ibsn_ctx* X, double dmax) {
  const double lim = X->prec == 0 ? kReanchorF64 : kReanchorF32;
  if (dmax > lim) return do_reanchor(X);
  return IBSN_OK;
}

// a2: plan pass; leaves c, g, ||g|| for the current gamma
int do_plan(ibsn_ctx* X) {
  PassGeom g;
  PassIn in;
  in.rowout = X->lse;
  RT(run_pass(X, Pass::Plan, in, &g));
  if (mode_for(X, Pass::Plan) == Mode::FF) {
    CK(launch_rows_ff(X->m, false, X->a, X->rowS0, nullptr, X->rowM, X->lse, X->scal, rb(X), X->st));
    RT(finish(X, g, X->c, true, 0));
  } else {
    RT(finish(X, g, X->c, true, 1));
  }
  RT(read_scal(X));
  X->gn = std::sqrt(X->h_scal[S_GN2]);
  return IBSN_OK;
}

int do_center(ibsn_ctx* X) {
  CK(launch_center(X->n, X->eta, X->gam, X->ganc, X->dd, X->d32, X->dlo32, X->d64, X->scal, rb(X), X->st));
  return IBSN_OK;
}

// a3: Sinkhorn warm-up in semi-dual form, then centring (Alg. 2)
int do_sinkhorn(ibsn_ctx* X, double tol, int max_iter, int* iters) {
  RT(do_plan(X));
  int it = 0;
  while (X->gn >= tol && it < max_iter) {
    CK(launch_sinkhorn_update(X->n, X->eta, X->b, X->c, X->gam, X->ganc, X->dd, X->d32, X->dlo32, X->d64, X->prec == 0,
                              X->scal, rb(X), X->st));
    RT(read_scal(X));
    RT(maybe_reanchor(X, X->h_scal[S_DMAX]));
    RT(do_plan(X));
    ++it;
  }
  RT(do_center(X));
  RT(read_scal(X));
  RT(maybe_reanchor(X, X->h_scal[S_DMAX]));
  if (iters) *iters = it;
  return IBSN_OK;
}

// a4: sparsification (Alg. 1) + CSC build + c_rho and Jacobi diagonal
int do_sparsify(ibsn_ctx* X, double rho) {
  CK(cudaMemsetAsync(X->pool_top, 0, sizeof(unsigned long long), X->st));
  CK(cudaMemsetAsync(X->err, 0, sizeof(int), X->st));
  PassGeom g;
  PassIn in;
  in.sparsify = true;
  in.s1 = rho;
  RT(run_pass(X, Pass::Sparsify, in, &g));
  const bool f64 = mode_for(X, Pass::Sparsify) == Mode::F64;
  X->sp_nb = g.nb;
  X->sp_rpb = g.rpb;
  X->sp_f64 = f64;
  {
    ProfScope ps(X, 3, 0.0, false);
    CK(launch_csc_build(X->sp, X->m, X->n, X->ldk, g.nb, g.rpb, f64, X->a, X->istar, X->eta, X->st));
  }
  unsigned long long top = 0;
  int err = 0;
  CK(cudaMemcpyAsync(&top, X->pool_top, sizeof(top), cudaMemcpyDeviceToHost, X->st));
  CK(cudaMemcpyAsync(&err, X->err, sizeof(int), cudaMemcpyDeviceToHost, X->st));
  CK(cudaStreamSynchronize(X->st));
  if (err == kDevCapacity || (int64_t)top > X->sp.cap) return IBSN_ERR_CAPACITY;
  X->nnz = (int64_t)top;
  return IBSN_OK;
}

// a5: Newton direction by persistent PCG
int do_direction(ibsn_ctx* X, double shift, double rtol, int max_cg, int* iters, double* resid) {
  CK(launch_neg(X->n, X->g, X->pc.rhs, X->st));
  // Jacobi diagonal of H_rho + shift I; c2 is free until the next Armijo trial
  CK(cudaMemcpyAsync(X->c2, X->sp.diag, sizeof(double) * X->n, cudaMemcpyDeviceToDevice, X->st));
  CK(launch_add_const(X->n, shift, X->c2, X->st));
  SparseBufs S = X->sp;
  S.diag = X->c2;
  const bool prof0 = X->prof.on;
  int perr = 0;
  // small float32 systems: one thread-block cluster (no grid-wide waits);
  // if its shared memory cannot hold the entries, the grid-wide kernel
  // the direction's post-processing (copy, centring, slope) is queued right
  // behind the solve; one read-back serves both
  auto post = [&]() -> int {
    CK(cudaMemcpyAsync(X->delta, X->pc.x, sizeof(double) * X->n, cudaMemcpyDeviceToDevice, X->st));
    CK(launch_dir_post(X->n, X->eta, X->delta, X->g, X->scal, rb(X), X->st));
    CK(cudaMemcpyAsync(X->h_perr, X->pc.err, sizeof(int), cudaMemcpyDeviceToHost, X->st));
    RT(read_scal(X));
    perr = *X->h_perr;
    return IBSN_OK;
  };
  bool done = false;
  if (!X->sp_f64 && X->nnz <= kClusterPcgMaxNnz && X->nnz < X->cl_fail_nnz) {
    bool launched = false;
    {
      ProfScope ps(X, 6, 0.0, false);
      CK(launch_pcg_cluster(S, X->pc, X->m, X->n, X->istar, X->a32, X->eta, shift, rtol, max_cg, X->scal, X->st,
                            &launched));
    }
    if (launched) {
      RT(post());
      if (perr == kDevCapacity) {
        X->cl_fail_nnz = X->nnz;  // the entries did not fit: nothing was computed
      } else {
        done = true;
        X->cl_runs++;
      }
    }
  }
  if (!done) {
    {
      ProfScope ps(X, 6, 0.0, X->sp_f64);
      CK(launch_pcg(S, X->pc, X->m, X->n, X->istar, X->sp_f64, X->a, X->a32, X->eta, shift, rtol, max_cg,
                    X->prm.wait_timeout_s, X->nsm, X->nnz, X->scal, X->st));
    }
    RT(post());
  }
  if (perr == kDevTimeout) return IBSN_ERR_TIMEOUT;
  if (iters) *iters = (int)X->h_scal[S_CG_ITERS];
  if (resid) *resid = X->h_scal[S_CG_RES];
  if (prof0) {
    const double sk = X->sp_f64 ? 8.0 : 4.0;
    const double per_it = 2.0 * (double)X->nnz * (4.0 + sk) + 2.0 * (double)X->n * sk +
                          8.0 * (6.0 * (double)X->n + 2.0 * (double)X->m);
    X->prof.bytes[6 + (X->sp_f64 ? 8 : 0)] += per_it * X->h_scal[S_CG_ITERS];
  }
  X->have_dir = true;
  return IBSN_OK;
}

// a6: one Armijo trial; dL = t g^T Delta + eta sum_j c_j phi_j + eta sum_i a_i psi(s_i)
int do_armijo_trial(ibsn_ctx* X, double t, double* dL, double* slope) {
  CK(launch_armijo_prep(X->n, X->ldk, X->eta, t, X->delta, X->c, X->em32, X->emlo32, X->em64, X->scal, rb(X),
                        X->st));
  PassGeom g;
  PassIn in;
  in.v1f = X->em32;
  in.v1d = X->em64;
  in.v1lo = X->emlo32;
  in.rowout = X->lse2;
  // entry j moves by t Delta_j / eta at the trial point, so its ratio to the
  // row maximum can grow by exp(2 t max|Delta| / eta): the float-float filter
  // keeps entries above 2^-64 exp(-2 t max|Delta| / eta) of the anchor maximum
  in.s2 = std::exp(-2.0 * t * X->h_scal[S_DELTAMAX]);
  RT(run_pass(X, Pass::Armijo, in, &g));
  if (mode_for(X, Pass::Armijo) == Mode::FF) {
    CK(launch_rows_ff(X->m, true, X->a, X->rowS0, X->rowS1, X->rowM, X->lse2, X->scal, rb(X), X->st));
    RT(finish(X, g, X->c2, false, 0));
  } else {
    RT(finish(X, g, X->c2, false, 2));
  }
  RT(read_scal(X));
  const double sl = X->h_scal[S_SLOPE];
  *slope = sl;
  *dL = t * sl + X->eta * X->h_scal[S_PHI] + X->eta * X->h_scal[S_ROW0 + 0];
  return IBSN_OK;
}

int do_accept(ibsn_ctx* X, double t) {
  CK(launch_armijo_accept(X->n, X->eta, t, X->delta, X->gam, X->ganc, X->dd, X->d32, X->dlo32, X->d64, X->c2, X->b,
                          X->g, X->scal, rb(X), X->st));
  std::swap(X->c, X->c2);
  std::swap(X->lse, X->lse2);
  RT(read_scal(X));
  X->gn = std::sqrt(X->h_scal[S_GN2]);
  RT(maybe_reanchor(X, X->h_scal[S_DMAX]));
  return IBSN_OK;
}

// a7: D_phi(Proj(X), X) (Eq. 8) at the current gamma (uses c, g of the current plan)
int do_stop(ibsn_ctx* X, double* dphi) {
  CK(launch_round_prep(X->n, X->b, X->c, X->g, X->rv, X->gridrc, X->scal, rb(X), X->st));
  PassGeom g;
  PassIn in;
  in.v1f = X->rv.om32;
  in.v1d = X->rv.om64;
  in.v2f = X->rv.ec32;
  in.v2d = X->rv.ec64;
  in.v3f = X->rv.lec32;
  in.v3d = X->rv.lec64;
  in.v4f = X->rv.hom32;
  in.v4d = X->rv.hom64;
  in.rowout = X->er;
  RT(run_pass(X, Pass::Stop, in, &g));
  // D_phi total: sum of row partials (no column work)
  RT(finish(X, g, nullptr, false, 1));
  RT(read_scal(X));
  *dphi = X->h_scal[S_ROW0 + 0];
  return IBSN_OK;
}

struct Cert {
  double p, d, gap, viol, kkt;
};

// a8: certificate at X = diag(a) P^k(gamma): primal of the Alg. 3 rounding,
// c-transform dual, relative gap, marginal violation, Delta_kkt
int do_certify(ibsn_ctx* X, Cert* out, double* plan, double* zeta) {
  CK(launch_round_prep(X->n, X->b, X->c, X->g, X->rv, X->gridrc, X->scal, rb(X), X->st));
  PassGeom g;
  PassIn in;
  in.v1f = X->rv.y32;
  in.v1d = X->rv.y64;
  in.v1lo = X->rv.ylo32;
  in.v2f = X->rv.om32;
  in.v2d = X->rv.om64;
  in.v2lo = X->rv.omlo32;
  in.v3f = X->rv.ecs32;
  in.v3d = X->rv.ecs64;
  in.gam = X->gam;
  in.rowout = zeta ? zeta : X->zeta;
  in.rowout2 = X->er;
  in.plan_out = plan;
  if (mode_for(X, Pass::Certify) == Mode::FF) {
    CK(launch_certify_prep(X->n, X->gam, X->gam32, X->gamlo32, X->scal, rb(X), X->st));
    if (X->cost.kind == IBSN_COST_GRID2D) {
      // exact c-transform of the grid cost by separability (colF is free until the pass's finish)
      CK(launch_ctransform_grid((int)(X->m / X->cost.gw), X->cost.gw, X->cost.scale, X->gam, X->colF, X->zgrid,
                                X->st));
      in.zeta_in = X->zgrid;
    }
  }
  RT(run_pass(X, Pass::Certify, in, &g));
  if (mode_for(X, Pass::Certify) == Mode::FF) {
    CK(launch_rows_cert(X->m, X->a, X->rowbuf, X->gridrc, X->cost.scale, in.rowout, in.rowout2, X->scal, rb(X),
                        X->st));
    RT(finish(X, g, X->colF, false, 0));
  } else {
    RT(finish(X, g, X->colF, false, 7));
  }
  RT(read_scal(X));
  const double ersum = X->h_scal[S_ROW0 + 3];
  const double primal = X->h_scal[S_ROW0 + 0];
  const double azeta = X->h_scal[S_ROW0 + 1];
  const double rowviol = X->h_scal[S_ROW0 + 2];
  const double comp = X->h_scal[S_ROW0 + 4];
  const double c2sum = X->h_scal[S_ROW0 + 5];
  const double rv2 = X->h_scal[S_ROW0 + 6];
  CK(launch_certify_cols(X->n, X->b, X->colF, X->c, X->gam, ersum, X->scal, rb(X), X->st));
  RT(read_scal(X));
  const double dual = azeta + X->h_scal[S_BGAM];
  out->p = primal;
  out->d = dual;
  const double den = std::max(std::fabs(primal), std::fabs(dual));
  out->gap = den > 0 ? (primal - dual) / den : std::fabs(primal - dual);
  out->viol = rowviol + X->h_scal[S_COLVIOL];
  // Delta_kkt (App. C.1) with the c-transform zeta (Delta_d = 0):
  // max(||X1 - a|| / (1 + ||a||), ||X^T 1 - b|| / (1 + ||b||), |<X, U>| / (1 + ||C||_F))
  const double cf = 1.0 + std::sqrt(c2sum);
  out->kkt = std::max(std::max(std::sqrt(rv2) / (1.0 + X->anorm), X->gn / (1.0 + X->bnorm)),
                      std::fabs(comp) / cf);
  return IBSN_OK;
}

struct NewtonStats {
  int newton = 0, cg = 0, armijo = 0;
  int fallbacks = 0;  // steps taken along -g because the Newton direction gave none
  int64_t max_nnz = 0;
};

// One Newton step of Alg. 2 at the current gamma: threshold rho = eta ||g|| / (m n)
// and sparsified Hessian (Alg. 1), Newton direction by PCG, Armijo backtracking
// in difference form, and the move gamma += t Delta (with its plan pass).
int newton_step(ibsn_ctx* X, const ibsn_params& P, double gate, int k, int v, NewtonStats* ns) {
  const double mn = (double)X->m * (double)X->n;
  const double gn = X->gn;
  const double rho = P.sparsify ? X->eta * gn / mn : 0.0;
  RT(do_sparsify(X, rho));
  ns->max_nnz = std::max(ns->max_nnz, X->nnz);
  // forcing term ||g||, relaxed to the accuracy at which the linear model
  // predicts the next gradient below the gate (reading R3)
  double rtol = gn > 0.0 ? std::min(P.cg_rtol, std::max(gn, 0.25 * gate / gn)) : P.cg_rtol;
  if (X->prec != 0) rtol = std::max(rtol, P.cg_rtol_floor_mixed);  // float32 Hessian values
  int cgit = 0;
  double cgres = 0.0;
  if (P.verbose > 1) CK(launch_len_stats(X->sp, X->m, X->n, X->scal, X->st));
  RT(do_direction(X, gn, rtol, P.max_cg, &cgit, &cgres));
  ns->cg += cgit;
  if (P.verbose > 1)
    fprintf(stderr, "[ibsn]   newton k=%d v=%d |g|=%.3e nnz=%lld maxrow=%d maxcol=%d cg=%d rtol=%.1e\n", k, v, gn,
            (long long)X->nnz, (int)X->h_scal[S_MAXROW], (int)X->h_scal[S_MAXCOL], cgit, rtol);
  // Backtracking along the stored direction.  Trials whose largest exponent
  // change t max|Delta|/eta exceeds the pass range are rejected unevaluated
  // (exp would overflow in that precision).  Returns 0 when a step met the
  // Armijo condition, 1 when only the last trial gave a finite decrease
  // (taken, reading R4: near the solution rounding can make every trial's
  // decrease slightly positive), 2 when no trial gave a finite value.
  const double range = X->prec == 0 ? 600.0 : (X->prec == 1 ? 60.0 : 30.0);
  double t = 1.0, dL = 0.0, slope = 0.0;
  auto backtrack = [&](int* outcome) -> int {
    const double dmax = X->h_scal[S_DELTAMAX];
    t = 1.0;
    bool evaluated = false;
    for (int tr = 0; tr < P.max_armijo; ++tr) {
      const bool last = tr + 1 == P.max_armijo;
      if (t * dmax <= range || last) {
        RT(do_armijo_trial(X, t, &dL, &slope));
        evaluated = true;
        ++ns->armijo;
        if (std::isfinite(dL) && dL <= P.sigma * t * slope) {
          *outcome = 0;
          return IBSN_OK;
        }
      }
      if (!last) t *= P.beta;
    }
    *outcome = (evaluated && std::isfinite(dL)) ? 1 : 2;
    return IBSN_OK;
  };
  int outcome = 2;
  RT(backtrack(&outcome));
  if (outcome == 2) {
    if (!(gn > 0.0) || !std::isfinite(gn)) return IBSN_ERR_NUMERICAL;
    // no finite trial along the Newton direction (a non-finite direction, or
    // one whose smallest trial still overflows): fall back to the
    // steepest-descent direction -g, scaled to an
    // exponent change of at most 1 at t = 1, and backtrack again
    CK(cudaMemsetAsync(X->delta, 0, sizeof(double) * X->n, X->st));
    k_axpy<<<(unsigned)((X->n + 255) / 256), 256, 0, X->st>>>(X->n, -X->eta / gn, X->g, X->delta);
    note_launch();
    CK(cudaGetLastError());
    CK(launch_dir_post(X->n, X->eta, X->delta, X->g, X->scal, rb(X), X->st));
    RT(read_scal(X));
    ++ns->fallbacks;
    RT(backtrack(&outcome));
    if (outcome == 2) return IBSN_ERR_NUMERICAL;
  }
  RT(do_accept(X, t));
  if (!std::isfinite(X->gn)) return IBSN_ERR_NUMERICAL;
  ++ns->newton;
  return IBSN_OK;
}

int outer_advance(ibsn_ctx* X, int new_prec) {
  // Gamma^{k+1} = Gamma^k + gamma^{k,fin}; k += 1; rebuild the anchor
  k_axpy<<<(unsigned)((X->n + 255) / 256), 256, 0, X->st>>>(X->n, 1.0, X->gam, X->Gam);
  note_launch();
  CK(cudaGetLastError());
  X->k += 1;
  X->prec = new_prec;
  return do_reanchor(X);
}

int ctx_create_impl(const ibsn_problem* pr, const ibsn_params* pp, void* ws, size_t bytes, cudaStream_t st,
                    ibsn_ctx** out) {
  RT(check_problem(pr));
  if (!pp || !out) return IBSN_ERR_INVALID_ARG;
  if (pp->precision != IBSN_PREC_FP64 && pp->precision != IBSN_PREC_MIXED) return IBSN_ERR_INVALID_ARG;
  if (pp->recompute && pp->precision != IBSN_PREC_MIXED) return IBSN_ERR_INVALID_ARG;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) return IBSN_ERR_WORKSPACE;
  const int nsm = device_sm_count();
  ibsn_ctx* X = new ibsn_ctx();
  Carver dry{nullptr};
  carve(X, dry, pr, pp, nsm);
  if (dry.off > bytes) {
    delete X;
    return IBSN_ERR_WORKSPACE;
  }
  Carver cv{static_cast<char*>(ws)};
  carve(X, cv, pr, pp, nsm);
  X->m = (int)pr->m;
  X->n = pr->n;
  X->ldk = ldk_for(pr->n);
  X->cost.C = pr->C;
  X->cost.ldc = pr->ldc;
  X->cost.kind = pr->cost_kind;
  X->cost.gw = pr->grid_w;
  X->cost.scale = pr->cost_scale;
  X->cost.rc = X->gridrc;
  X->cost.px = pr->x;
  X->cost.py = pr->y;
  X->cost.xs = X->xs;
  X->cost.ys = X->ys;
  X->cost.dim = pr->cost_kind == IBSN_COST_SQEUCLID_POINTS ? pr->dim : 0;
  X->a = pr->a;
  X->b = pr->b;
  X->eta = pr->eta;
  X->prm = *pp;
  X->st = st;
  X->nsm = nsm;
  X->prec = pp->precision == IBSN_PREC_MIXED ? 1 : 0;
  cudaError_t e = cudaMallocHost(&X->h_scal, sizeof(double) * (S_NSLOTS + 1));
  if (e == cudaSuccess) X->h_perr = reinterpret_cast<int*>(X->h_scal + S_NSLOTS);
  if (e != cudaSuccess) {
    delete X;
    return set_cuda_error(e);
  }
  auto fail = [&](int code) {
    cudaFreeHost(X->h_scal);
    delete X;
    return code;
  };
  if (cudaMemsetAsync(X->scal, 0, sizeof(double) * S_NSLOTS, st) != cudaSuccess) return fail(IBSN_ERR_CUDA);
  // validation (Eq. 1): a, b > 0, finite, sums 1; C finite and >= 0
  if (launch_validate_marginals(pr->m, pr->n, pr->a, pr->b, X->scal, st) != cudaSuccess) return fail(IBSN_ERR_CUDA);
  if (pr->cost_kind != IBSN_COST_GRID2D &&
      launch_validate_cost(pr->m, pr->n, pr->C, pr->ldc, pr->cost_kind, pr->x, pr->y, X->cost.dim, pr->cost_scale,
                           X->scal, st) != cudaSuccess)
    return fail(IBSN_ERR_CUDA);
  if (pr->cost_kind == IBSN_COST_SQEUCLID_POINTS &&
      (launch_split_coords(pr->m * pr->dim, pr->x, X->xs, st) != cudaSuccess ||
       launch_split_coords(pr->n * pr->dim, pr->y, X->ys, st) != cudaSuccess))
    return fail(IBSN_ERR_CUDA);
  if (pr->cost_kind == IBSN_COST_GRID2D) {
    // max C of the grid cost (two opposite corners) and sum C^2 over all pairs
    // of bins, sum over offsets (dr, dc) of (h - |dr|)(w - |dc|)(dr^2 + dc^2)^2
    const double dh = (double)(pr->grid_h - 1), dw = (double)(pr->grid_w - 1);
    double c2 = 0.0;
    for (int dr = -(pr->grid_h - 1); dr < pr->grid_h; ++dr)
      for (int dc = -(pr->grid_w - 1); dc < pr->grid_w; ++dc) {
        const double q = (double)dr * dr + (double)dc * dc;
        c2 += (double)(pr->grid_h - std::abs(dr)) * (double)(pr->grid_w - std::abs(dc)) * q * q;
      }
    c2 *= pr->cost_scale * pr->cost_scale;
    if (cudaMemsetAsync(&X->scal[S_CBAD], 0, sizeof(double), st) != cudaSuccess ||
        launch_set_slot(X->scal, S_CMAX, pr->cost_scale * (dh * dh + dw * dw), st) != cudaSuccess ||
        launch_set_slot(X->scal, S_C2SUM, c2, st) != cudaSuccess ||
        launch_grid_rc(pr->n, pr->grid_w, X->gridrc, st) != cudaSuccess)
      return fail(IBSN_ERR_CUDA);
  }
  if (read_scal(X) != IBSN_OK) return fail(IBSN_ERR_CUDA);
  const double* h = X->h_scal;
  if (h[S_ABAD] > 0 || h[S_CBAD] > 0) return fail(IBSN_ERR_NONFINITE);
  if (!(h[S_AMIN] > 0) || !(h[S_BMIN] > 0) || std::fabs(h[S_ASUM] - 1.0) > 1e-12 || std::fabs(h[S_BSUM] - 1.0) > 1e-12)
    return fail(IBSN_ERR_MARGINALS);
  // i* = argmax a (lowest index on ties)
  std::vector<double> ha(pr->m);
  if (cudaMemcpyAsync(ha.data(), pr->a, sizeof(double) * pr->m, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(IBSN_ERR_CUDA);
  X->istar = (int)(std::max_element(ha.begin(), ha.end()) - ha.begin());
  std::vector<double> hb(pr->n);
  if (cudaMemcpyAsync(hb.data(), pr->b, sizeof(double) * pr->n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(IBSN_ERR_CUDA);
  for (double v : ha) X->anorm += v * v;
  for (double v : hb) X->bnorm += v * v;
  X->anorm = std::sqrt(X->anorm);
  X->bnorm = std::sqrt(X->bnorm);
  k_log<<<(unsigned)((X->n + 255) / 256), 256, 0, st>>>(X->n, pr->b, X->logb);
  k_to_float<<<(unsigned)((X->m + 255) / 256), 256, 0, st>>>(X->m, pr->a, X->a32);
  k_lo_float<<<(unsigned)((X->m + 255) / 256), 256, 0, st>>>(X->m, pr->a, X->alo32);
  note_launch(3);
  // zero state, pad the float/double per-column vectors
  cudaMemsetAsync(X->Gam, 0, sizeof(double) * X->n, st);
  cudaMemsetAsync(X->gam, 0, sizeof(double) * X->n, st);
  cudaMemsetAsync(X->ctr, 0, sizeof(unsigned int) * C_NCOUNTERS, st);
  float* tf[] = {X->d32,      X->em32,       X->gam32,    X->rv.y32,  X->rv.om32,   X->rv.ec32,
                 X->rv.ecs32, X->rv.ecsl32, X->rv.lec32, X->rv.hom32, X->dlo32,    X->emlo32,
                 X->gamlo32,  X->rv.ylo32,  X->rv.omlo32};
  for (float* v : tf) cudaMemsetAsync(v, 0, sizeof(float) * X->ldk, st);
  double* td[] = {X->d64, X->em64, X->rv.y64, X->rv.om64, X->rv.ec64, X->rv.ecs64, X->rv.lec64, X->rv.hom64};
  for (double* v : td) cudaMemsetAsync(v, 0, sizeof(double) * X->ldk, st);
  if (cudaGetLastError() != cudaSuccess) return fail(IBSN_ERR_CUDA);
  *out = X;
  return IBSN_OK;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

const char* ibsn_status_string(int s) {
  switch (s) {
    case IBSN_OK: return "ok";
    case IBSN_ERR_INVALID_ARG: return "invalid argument";
    case IBSN_ERR_MARGINALS: return "marginals not positive or not summing to 1";
    case IBSN_ERR_NONFINITE: return "non-finite or negative input";
    case IBSN_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case IBSN_ERR_CUDA: return "CUDA error";
    case IBSN_ERR_TIMEOUT: return "device wait timed out";
    case IBSN_ERR_CAPACITY: return "sparsified Hessian exceeds the reserved nonzeros";
    case IBSN_ERR_UNSUPPORTED: return "size not supported by this build";
    case IBSN_NOT_CONVERGED: return "not converged";
    case IBSN_ERR_NUMERICAL: return "non-finite intermediate (numerical breakdown)";
    default: return "unknown status";
  }
}

const char* ibsn_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

void ibsn_params_default(ibsn_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->sigma = 1e-4;
  p->beta = 0.8;
  p->sinkhorn_tol = 1e-3;
  p->mu0 = 1e-4;
  p->mu_min = 1e-11;
  p->gap_tol = 1e-8;
  p->cg_rtol = 0.1;
  p->cg_rtol_floor_mixed = 1e-6;
  p->polish_gap = 1e-6;
  p->wait_timeout_s = 2.0;
  p->gamma0 = nullptr;
  p->nnz_cap = 0;
  p->max_outer = 5000;
  p->max_newton = 50;
  p->max_cg = 1000;
  p->max_sinkhorn = 10000;
  p->max_armijo = 60;
  p->precision = IBSN_PREC_FP64;
  p->polish = 1;
  p->sparsify = 1;
  p->verbose = 0;
  p->eot = 0;
  p->eot_gtol = 1e-9;
  p->recompute = 0;
}

int ibsn_workspace_size(const ibsn_problem* prob, const ibsn_params* params, size_t* bytes) {
  if (!bytes || !params) return IBSN_ERR_INVALID_ARG;
  RT(check_problem(prob));
  ibsn_ctx X;
  Carver dry{nullptr};
  carve(&X, dry, prob, params, device_sm_count());
  *bytes = dry.off + 256;
  return IBSN_OK;
}

int ibsn_ctx_create(const ibsn_problem* prob, const ibsn_params* params, void* ws, size_t bytes, void* stream,
                    ibsn_ctx** out) {
  return ctx_create_impl(prob, params, ws, bytes, (cudaStream_t)stream, out);
}

int ibsn_ctx_destroy(ibsn_ctx* X) {
  if (!X) return IBSN_ERR_INVALID_ARG;
  if (X->st) cudaStreamSynchronize(X->st);
  cudaFreeHost(X->h_scal);
  delete X;
  return IBSN_OK;
}

int ibsn_ctx_set_state(ibsn_ctx* X, int64_t k, const double* Gamma, const double* gamma, int precision) {
  if (!X || k < 0) return IBSN_ERR_INVALID_ARG;
  if (precision == 1 && !X->have_f32) return IBSN_ERR_INVALID_ARG;
  if (precision == 0 && !X->have_f64) return IBSN_ERR_INVALID_ARG;
  if (precision == 2 && !X->have_ff) return IBSN_ERR_INVALID_ARG;
  if (precision < 0 || precision > 2) return IBSN_ERR_INVALID_ARG;
  if (Gamma) CK(cudaMemcpyAsync(X->Gam, Gamma, sizeof(double) * X->n, cudaMemcpyDeviceToDevice, X->st));
  else CK(cudaMemsetAsync(X->Gam, 0, sizeof(double) * X->n, X->st));
  if (gamma) CK(cudaMemcpyAsync(X->gam, gamma, sizeof(double) * X->n, cudaMemcpyDeviceToDevice, X->st));
  else CK(cudaMemsetAsync(X->gam, 0, sizeof(double) * X->n, X->st));
  X->k = k;
  X->prec = precision;
  X->have_dir = false;
  RT(do_reanchor(X));
  CK(cudaStreamSynchronize(X->st));
  return IBSN_OK;
}

int ibsn_ctx_plan(ibsn_ctx* X, double* colsum, double* grad_norm) {
  if (!X) return IBSN_ERR_INVALID_ARG;
  RT(do_plan(X));
  if (colsum) CK(cudaMemcpyAsync(colsum, X->c, sizeof(double) * X->n, cudaMemcpyDeviceToDevice, X->st));
  CK(cudaStreamSynchronize(X->st));
  if (grad_norm) *grad_norm = X->gn;
  return IBSN_OK;
}

int ibsn_ctx_export_plan(ibsn_ctx* X, double* P) {
  if (!X || !P) return IBSN_ERR_INVALID_ARG;
  PassIn in;
  in.plan_out = P;
  RT(run_pass(X, Pass::Export, in));
  CK(cudaStreamSynchronize(X->st));
  return IBSN_OK;
}

int ibsn_ctx_get_gamma(ibsn_ctx* X, double* gamma) {
  if (!X || !gamma) return IBSN_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(gamma, X->gam, sizeof(double) * X->n, cudaMemcpyDeviceToDevice, X->st));
  CK(cudaStreamSynchronize(X->st));
  return IBSN_OK;
}

int ibsn_ctx_sinkhorn(ibsn_ctx* X, double tol, int32_t max_iter, int32_t* iters, double* grad_norm) {
  if (!X) return IBSN_ERR_INVALID_ARG;
  int it = 0;
  RT(do_sinkhorn(X, tol, max_iter, &it));
  if (iters) *iters = it;
  if (grad_norm) *grad_norm = X->gn;
  return IBSN_OK;
}

int ibsn_ctx_sparsify(ibsn_ctx* X, double rho, int64_t* nnz) {
  if (!X || !(rho >= 0.0)) return IBSN_ERR_INVALID_ARG;
  RT(do_plan(X));
  RT(do_sparsify(X, rho));
  if (nnz) *nnz = X->nnz;
  return IBSN_OK;
}

int ibsn_ctx_export_sparse(ibsn_ctx* X, double* P_rho) {
  if (!X || !P_rho) return IBSN_ERR_INVALID_ARG;
  CK(launch_export_sparse(X->sp, X->m, X->n, X->istar, X->prec == 0, P_rho, X->st));
  CK(cudaStreamSynchronize(X->st));
  return IBSN_OK;
}

int ibsn_ctx_newton_direction(ibsn_ctx* X, double shift, double rtol, int32_t max_cg, double* delta,
                              int32_t* cg_iters, double* resid) {
  if (!X || max_cg < 0 || !(rtol >= 0.0)) return IBSN_ERR_INVALID_ARG;
  if (shift < 0.0) shift = X->gn;
  int it = 0;
  double rs = 0.0;
  RT(do_direction(X, shift, rtol, max_cg, &it, &rs));
  if (delta) CK(cudaMemcpyAsync(delta, X->delta, sizeof(double) * X->n, cudaMemcpyDeviceToDevice, X->st));
  CK(cudaStreamSynchronize(X->st));
  if (cg_iters) *cg_iters = it;
  if (resid) *resid = rs;
  return IBSN_OK;
}

int ibsn_ctx_armijo_trial(ibsn_ctx* X, double t, int32_t accept, double* dL, double* slope, int32_t* accepted) {
  if (!X || !X->have_dir || !(t > 0.0)) return IBSN_ERR_INVALID_ARG;
  double d = 0.0, s = 0.0;
  RT(do_armijo_trial(X, t, &d, &s));
  const bool ok = d <= X->prm.sigma * t * s;
  if (accept && ok) RT(do_accept(X, t));
  if (dL) *dL = d;
  if (slope) *slope = s;
  if (accepted) *accepted = (accept && ok) ? 1 : 0;
  return IBSN_OK;
}

int ibsn_ctx_stop_check(ibsn_ctx* X, double* dphi) {
  if (!X) return IBSN_ERR_INVALID_ARG;
  RT(do_plan(X));
  double d = 0.0;
  RT(do_stop(X, &d));
  if (dphi) *dphi = d;
  return IBSN_OK;
}

int ibsn_ctx_certify(ibsn_ctx* X, double* primal, double* dual, double* rel_gap, double* marg_viol, double* plan,
                     double* zeta) {
  if (!X) return IBSN_ERR_INVALID_ARG;
  RT(do_plan(X));
  Cert c{};
  RT(do_certify(X, &c, plan, zeta));
  CK(cudaStreamSynchronize(X->st));
  if (primal) *primal = c.p;
  if (dual) *dual = c.d;
  if (rel_gap) *rel_gap = c.gap;
  if (marg_viol) *marg_viol = c.viol;
  return IBSN_OK;
}

int ibsn_solve_batch(int count, const ibsn_problem* probs, const ibsn_params* params, void* const* workspaces,
                     const size_t* workspace_bytes, ibsn_result* results, void* const* streams, int threads) {
  if (count < 0) return IBSN_ERR_INVALID_ARG;
  if (count == 0) return IBSN_OK;
  if (!probs || !params || !workspaces || !workspace_bytes || !results) return IBSN_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IBSN_ERR_CUDA;
  const int nt = std::max(1, std::min(threads > 0 ? threads : 8, count));
  std::atomic<int> next{0};
  std::vector<int> codes((size_t)count, IBSN_OK);
  // largest problems first (by m n), so that no large solve starts last and
  // leaves the other threads idle; each problem's result does not depend on
  // the order
  std::vector<int> order((size_t)count);
  for (int q = 0; q < count; ++q) order[(size_t)q] = q;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return (double)probs[x].m * (double)probs[x].n > (double)probs[y].m * (double)probs[y].n;
  });
  auto worker = [&]() {
    if (cudaSetDevice(dev) != cudaSuccess) return;
    cudaStream_t own = nullptr;
    if (!streams && cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess) own = nullptr;
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= count) break;
      const int q = order[(size_t)k];
      void* st = streams ? streams[q] : (void*)own;
      codes[(size_t)q] = ibsn_solve(&probs[q], params, workspaces[q], workspace_bytes[q], &results[q], st);
    }
    if (own) {
      cudaStreamSynchronize(own);
      cudaStreamDestroy(own);
    }
  };
  std::vector<std::thread> pool;
  pool.reserve((size_t)nt);
  for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
  for (std::thread& t : pool) t.join();
  int ret = IBSN_OK;
  for (int q = 0; q < count; ++q) {
    const int c = codes[(size_t)q];
    if (c != IBSN_OK && c != IBSN_NOT_CONVERGED) return c;
    if (c == IBSN_NOT_CONVERGED) ret = IBSN_NOT_CONVERGED;
  }
  return ret;
}

int ibsn_solve(const ibsn_problem* prob, const ibsn_params* params, void* ws, size_t bytes, ibsn_result* res,
               void* stream) {
  if (!res || !params) return IBSN_ERR_INVALID_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  ibsn_ctx* X = nullptr;
  RT(ibsn_ctx_create(prob, params, ws, bytes, stream, &X));
  X->prof.on = params->profile != 0;
  const long long launches0 = g_launches.load();
  struct Guard {
    ibsn_ctx* X;
    ~Guard() { ibsn_ctx_destroy(X); }
  } guard{X};
  const ibsn_params& P = *params;
  const int64_t m = X->m, n = X->n;
  const double floor32 = 32.0 * std::ldexp(1.0, -24);  // relative float32 noise of a column sum
  // (E)IBSN: the single entropic subproblem with X^0 = 1 1^T instead of a b^T;
  // the row factor a_i does not change the plan, the column factor b_j is
  // dropped from the anchored exponent
  if (P.eot) CK(cudaMemsetAsync(X->logb, 0, sizeof(double) * n, X->st));
  // initial state: k = 0, Gamma = 0, gamma = gamma0 or 0
  RT(ibsn_ctx_set_state(X, 0, nullptr, P.gamma0, X->prec));
  NewtonStats ns;
  int tot_sk = 0, polish_outer = 0;
  Cert cert{1e300, -1e300, 1e300, 0, 0};
  double best_gap = 1e300;
  int stall = 0;
  int status = IBSN_NOT_CONVERGED;
  int k = 0;
  double bnorm = 0.0;
  {
    std::vector<double> hb(n);
    CK(cudaMemcpyAsync(hb.data(), X->b, sizeof(double) * n, cudaMemcpyDeviceToHost, X->st));
    CK(cudaStreamSynchronize(X->st));
    for (double v : hb) bnorm += v * v;
    bnorm = std::sqrt(bnorm);  // ||b||_2 for the float32 gradient floor
  }
  if (P.eot) {
    // Sinkhorn warm-up, then Newton steps until ||g|| < eot_gtol or max_newton
    // steps (App. C.4).  Float32 passes cannot resolve ||g|| below their noise
    // floor: there (or once a step no longer halves ||g||) a mixed solve with
    // polish continues in float-float passes.
    int sk = 0;
    RT(do_sinkhorn(X, P.sinkhorn_tol, P.max_sinkhorn, &sk));
    tot_sk += sk;
    if (!std::isfinite(X->gn)) return IBSN_ERR_NUMERICAL;
    double gn_before = 1e300;
    for (int v = 0; v < P.max_newton; ++v) {
      if (X->gn < P.eot_gtol) {
        status = IBSN_OK;
        break;
      }
      if (X->prec == 1 && X->have_ff && (X->gn < floor32 * bnorm || X->gn > 0.5 * gn_before)) {
        X->prec = 2;
        RT(do_reanchor(X));
        RT(do_plan(X));
        if (X->gn < P.eot_gtol) {
          status = IBSN_OK;
          break;
        }
      }
      gn_before = X->gn;
      RT(newton_step(X, P, P.eot_gtol, 0, v, &ns));
      if (P.verbose)
        fprintf(stderr, "[ibsn] eot v=%d prec=%s |g|=%.3e nnz=%lld\n", v,
                X->prec == 0 ? "f64" : (X->prec == 1 ? "f32" : "ff"), X->gn, (long long)X->nnz);
    }
    if (status != IBSN_OK && X->gn < P.eot_gtol) status = IBSN_OK;
    if (X->prec == 2) polish_outer = 1;
    RT(do_certify(X, &cert, nullptr, nullptr));
    k = 1;
  }
  for (k = P.eot ? 1 : 0; !P.eot && k < P.max_outer; ++k) {
    const double mu = std::max(P.mu0 / ((double)(k + 1) * (double)(k + 1)), P.mu_min);
    int sk = 0;
    RT(do_sinkhorn(X, P.sinkhorn_tol, P.max_sinkhorn, &sk));
    tot_sk += sk;
    if (!std::isfinite(X->gn)) return IBSN_ERR_NUMERICAL;
    const double gate = X->prec == 1 ? std::max(mu, floor32 * bnorm) : mu;
    int v = 0;
    for (v = 0; v < P.max_newton; ++v) {
      const double gn = X->gn;
      RT(newton_step(X, P, gate, k, v, &ns));
      if (X->gn < gate) {
        double dphi = 0.0;
        RT(do_stop(X, &dphi));
        if (dphi <= (double)std::min(m, n) * mu) {
          ++v;
          break;
        }
        // float32 passes: below the gate the gradient is at the float32 noise
        // floor; once a Newton step no longer halves it, more steps cannot
        // pass Eq. 8 in this precision, so the outer loop proceeds
        if (X->prec == 1 && X->gn > 0.5 * gn) {
          ++v;
          break;
        }
      }
    }
    // certificate at X^{k+1} = diag(a) P^k(gamma^{k,fin}); with float32 passes
    // it only steers the switch to the polish, so it is taken every 4th step
    const bool certify_now = X->prec != 1 || (k % 4) == 0 || k + 1 == P.max_outer;
    if (certify_now) RT(do_certify(X, &cert, nullptr, nullptr));
    if (!std::isfinite(cert.gap)) return IBSN_ERR_NUMERICAL;
    if (X->prec == 2) ++polish_outer;
    if (P.verbose)
      fprintf(stderr, "[ibsn] k=%d prec=%s sk=%d newton=%d |g|=%.3e nnz=%lld p=%.12e d=%.12e gap=%.3e\n", k,
              X->prec == 0 ? "f64" : (X->prec == 1 ? "f32" : "ff"), sk, v, X->gn, (long long)X->nnz, cert.p,
              cert.d, cert.gap);
    if (cert.gap <= P.gap_tol && X->prec != 1) {
      status = IBSN_OK;
      ++k;
      break;
    }
    if (cert.gap <= P.gap_tol && X->prec == 1 && !P.polish) {
      status = IBSN_OK;
      ++k;
      break;
    }
    // mixed precision: float32 passes until the (float32-plan) certificate
    // reaches polish_gap, or makes no 2x progress over 12 outer steps (the
    // float32 noise floor of the certificate); then float-float passes
    int next_prec = X->prec;
    if (X->prec == 1 && P.polish && certify_now) {
      if (cert.gap < 0.5 * best_gap) {
        best_gap = cert.gap;
        stall = 0;
      } else {
        stall += 4;
      }
      if (cert.gap <= P.polish_gap || stall >= 12) next_prec = 2;
    }
    if (k + 1 < P.max_outer) RT(outer_advance(X, next_prec));
  }
  // outputs
  if (res->gamma) CK(cudaMemcpyAsync(res->gamma, X->gam, sizeof(double) * n, cudaMemcpyDeviceToDevice, X->st));
  if (res->plan || res->zeta) {
    Cert c2{};
    RT(do_certify(X, &c2, res->plan, res->zeta));
  }
  CK(cudaStreamSynchronize(X->st));
  res->primal = cert.p;
  res->dual = cert.d;
  res->rel_gap = cert.gap;
  res->kkt = cert.kkt;
  res->marg_viol = cert.viol;
  res->grad_norm = X->gn;
  res->outer_iters = k;
  res->newton_iters = ns.newton;
  res->cg_iters = ns.cg;
  res->sinkhorn_iters = tot_sk;
  res->armijo_trials = ns.armijo;
  res->polish_outer = polish_outer;
  res->reanchors = X->reanchors;
  res->status = status;
  res->max_nnz = ns.max_nnz;
  res->dense_passes = X->dense_passes;
  res->kernel_launches = g_launches.load() - launches0;
  X->prof.harvest();
  for (int q = 0; q < 16; ++q) {
    res->pass_ms[q] = X->prof.ms[q];
    res->pass_calls[q] = X->prof.calls[q];
    res->pass_bytes[q] = X->prof.bytes[q];
  }
  res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return status;
}

// Warm start or fallback start (Alg. 2 starts from gamma = 0; the fallback is
// that zero start or a given potential): the start with the smaller
// semi-dual objective L^0 (Eq. 5 at k = 0) wins; a non-finite value never
// wins.  The plan-pass gradient norms (Eq. 7) from both starts are reported
// alongside.
int ibsn_judge_warm_start(const ibsn_problem* prob, const ibsn_params* params, const double* gamma_hat,
                          const double* gamma_fallback, void* workspace, size_t workspace_bytes,
                          double* objective_warm, double* objective_fallback, double* grad_norm_warm,
                          double* grad_norm_fallback, int32_t* use_warm, void* stream) {
  if (!prob || !params || !gamma_hat || !use_warm) return IBSN_ERR_INVALID_ARG;
  ibsn_ctx* X = nullptr;
  RT(ctx_create_impl(prob, params, workspace, workspace_bytes, (cudaStream_t)stream, &X));
  struct Guard {
    ibsn_ctx* X;
    ~Guard() { ibsn_ctx_destroy(X); }
  } guard{X};
  const int prec = X->prec;
  double gw = 0.0, gz = 0.0;
  RT(ibsn_ctx_set_state(X, 0, nullptr, gamma_hat, prec));
  RT(ibsn_ctx_plan(X, nullptr, &gw));
  CK(launch_semidual0(X->cost, X->m, X->n, X->eta, X->a, X->b, X->logb, gamma_hat, X->er, X->scal + S_TMP, X->st));
  RT(read_scal(X));
  const double Lw = X->h_scal[S_TMP];
  RT(ibsn_ctx_set_state(X, 0, nullptr, gamma_fallback, prec));
  RT(ibsn_ctx_plan(X, nullptr, &gz));
  CK(launch_semidual0(X->cost, X->m, X->n, X->eta, X->a, X->b, X->logb, gamma_fallback, X->er, X->scal + S_TMP,
                      X->st));
  RT(read_scal(X));
  const double Lz = X->h_scal[S_TMP];
  if (objective_warm) *objective_warm = Lw;
  if (objective_fallback) *objective_fallback = Lz;
  if (grad_norm_warm) *grad_norm_warm = gw;
  if (grad_norm_fallback) *grad_norm_fallback = gz;
  *use_warm = (std::isfinite(Lw) && Lw < Lz) ? 1 : 0;
  return IBSN_OK;
}

}  // extern "C"
