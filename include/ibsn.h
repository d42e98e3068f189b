/*
 * ibsn.h -- C ABI of the GB300 (sm_103a) IBSN solver for exact discrete optimal
 * transport (Inexact Bregman Sparse Newton, arXiv 2603.07156).
 *
 * Problem (Eq. 1, Sec. 1):  min <C, X>  s.t.  X 1 = a,  X^T 1 = b,  X >= 0,
 * with C >= 0 (m x n), a > 0, b > 0, 1^T a = 1^T b = 1.  The solver runs the
 * Bregman proximal point method of Alg. 2 with proximal weight eta > 0 (Eq. 2),
 * solving each semi-dual subproblem (Eq. 5) by the sparsified-Hessian Newton
 * method (Alg. 1, Alg. 2), and certifies the result with the rounding of
 * Alg. 3 and the c-transform dual of App. C.1.
 *
 * Conventions for every entry point:
 *  - Pointers marked "device" are CUDA device pointers on the current device;
 *    "host" pointers are ordinary host memory.  The caller owns all of them;
 *    the library never frees caller memory and allocates no device memory of
 *    its own: all device scratch comes from the caller's workspace.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Calls enqueue their kernels on it and synchronise it before
 *    returning host-visible scalars.
 *  - Every function returns an ibsn_status; nothing aborts the process.  A
 *    device-side wait that exceeds params.wait_timeout_s ends the kernel and
 *    returns IBSN_ERR_TIMEOUT with the CUDA context still usable.
 *  - Not thread-safe per context; distinct contexts may be used from distinct
 *    host threads.
 */
#ifndef IBSN_H
#define IBSN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ibsn_status {
  IBSN_OK = 0,
  IBSN_ERR_INVALID_ARG = 1,  /* null pointer, m or n < 1, eta <= 0, bad enum */
  IBSN_ERR_MARGINALS = 2,    /* a or b not > 0, or |sum - 1| > 1e-12 (Eq. 1) */
  IBSN_ERR_NONFINITE = 3,    /* NaN/Inf in C, a or b, or C < 0 */
  IBSN_ERR_WORKSPACE = 4,    /* workspace null, too small, or misaligned (256 B) */
  IBSN_ERR_CUDA = 5,         /* a CUDA runtime call failed; see ibsn_last_cuda_error */
  IBSN_ERR_TIMEOUT = 6,      /* a bounded device wait (grid barrier) expired */
  IBSN_ERR_CAPACITY = 7,     /* sparsified Hessian needs more nonzeros than reserved */
  IBSN_ERR_UNSUPPORTED = 8,  /* size outside this build's kernels (n > 16384) */
  IBSN_NOT_CONVERGED = 9,    /* result valid but rel_gap > gap_tol after max_outer */
  IBSN_ERR_NUMERICAL = 10    /* a gradient, objective change or certificate became non-finite */
} ibsn_status;

typedef enum ibsn_cost_kind {
  IBSN_COST_DENSE_F64 = 0,   /* C given as a dense row-major float64 matrix */
  IBSN_COST_DENSE_F32 = 1,   /* C given as a dense row-major float32 matrix (exact values) */
  IBSN_COST_GRID2D = 2,      /* bins of one h x w grid (row-major), m = n = h*w:
                                C_ij = cost_scale * ((r_i - r_j)^2 + (c_i - c_j)^2),
                                rebuilt on the fly from the integer coordinates */
  IBSN_COST_SQEUCLID_POINTS = 3  /* point clouds x (m x dim) and y (n x dim), float64
                                row-major device arrays, 1 <= dim <= 16:
                                C_ij = cost_scale * ||x_i - y_j||^2, rebuilt on the fly
                                (in float-float arithmetic, ~2^-46 relative) wherever
                                the solver reads C; no m x n cost matrix is stored */
} ibsn_cost_kind;

typedef enum ibsn_precision {
  IBSN_PREC_FP64 = 0,        /* every pass in float64 */
  IBSN_PREC_MIXED = 1        /* float32 plan / exp / SpMV passes, float64 potentials,
                                gradient and residual accumulation, CG inner
                                products and certificate; optional float64 polish */
} ibsn_precision;

/* One OT instance (Eq. 1).  All pointers are device pointers. */
typedef struct ibsn_problem {
  int64_t m, n;              /* sizes, >= 1 */
  int64_t ldc;               /* row stride of C in elements (>= n), dense kinds */
  const void* C;             /* dense kinds: m x ldc, float64 or float32 */
  const double* a;           /* m, source marginal */
  const double* b;           /* n, target marginal */
  double eta;                /* proximal weight eta > 0 (Eq. 2) */
  double cost_scale;         /* GRID2D: C = cost_scale * integer squared distance;
                                SQEUCLID_POINTS: C = cost_scale * squared distance */
  int32_t cost_kind;         /* ibsn_cost_kind */
  int32_t grid_h, grid_w;    /* GRID2D */
  int32_t dim;               /* SQEUCLID_POINTS: coordinates per point */
  const double* x;           /* SQEUCLID_POINTS: m x dim source points (device) */
  const double* y;           /* SQEUCLID_POINTS: n x dim target points (device) */
} ibsn_problem;

/* Parameters.  ibsn_params_default() fills the paper's constants. */
typedef struct ibsn_params {
  double sigma;              /* Armijo parameter, 1e-4 (Alg. 2) */
  double beta;               /* backtracking factor, 0.8 (Alg. 2) */
  double sinkhorn_tol;       /* warm-up stops when ||g|| < 1e-3 (Sec. 5) */
  double mu0, mu_min;        /* mu_k = max(mu0/(k+1)^2, mu_min): 1e-4, 1e-11 (Eq. 8) */
  double gap_tol;            /* outer stop: relative duality gap, 1e-8 */
  double cg_rtol;            /* CG stops at ||r|| <= min(cg_rtol, ||g||) ||g||; 0.1 */
  double cg_rtol_floor_mixed;/* mixed passes: relative CG tolerance floor, 1e-6 */
  double polish_gap;         /* mixed: switch to float64 once the certified gap < this (1e-6) */
  double wait_timeout_s;     /* bound on any device-side wait, seconds (default 2) */
  const double* gamma0;      /* nullable device n-vector: warm-start potential */
  int64_t nnz_cap;           /* nonzeros reserved for P_rho; 0 = m*n (never overflows) */
  int32_t max_outer;         /* 5000 */
  int32_t max_newton;        /* 50 per outer step */
  int32_t max_cg;            /* 1000 per Newton direction */
  int32_t max_sinkhorn;      /* 10000 per warm-up */
  int32_t max_armijo;        /* 60 trials */
  int32_t precision;         /* ibsn_precision */
  int32_t polish;            /* mixed: finish in float64 (1) or not (0) */
  int32_t sparsify;          /* 1 = IBSN (Alg. 1); 0 = IBN, dense Hessian (App. C.3) */
  int32_t verbose;           /* per-outer log lines on stderr */
  int32_t profile;           /* 1: time every pass kind with CUDA events (ibsn_result.pass_ms) */
  double eot_gtol;           /* eot mode: stop once ||g|| < eot_gtol (1e-9, App. C.4) */
  int32_t eot;               /* 1 = (E)IBSN (App. C.4): one entropic subproblem with
                                X^0 = 1 1^T (not a b^T), Sinkhorn warm-up, then at most
                                max_newton Newton steps until ||g|| < eot_gtol; no
                                outer update.  The result's gamma is the semi-dual
                                solution of that subproblem; primal/dual/rel_gap
                                certify its rounded plan for the LP of Eq. 1; status
                                IBSN_OK when the gradient test passed.  0 = IBSN. */
  int32_t recompute;         /* mixed precision only: 1 = store no anchored exponent
                                matrix; every pass rebuilds K_ij from the cost with the
                                arithmetic of the anchor build (identical values, no
                                m x n workspace; ALU instead of HBM traffic).  0 = stored K */
} ibsn_params;

/* Result of ibsn_solve.  Output vectors are optional caller buffers. */
typedef struct ibsn_result {
  double* gamma;             /* nullable device n: final potential gamma (semi-dual) */
  double* zeta;              /* nullable device m: c-transform zeta_i = min_j C_ij - gamma_j */
  double* plan;              /* nullable device m*n float64: rounded feasible plan (Alg. 3) */
  double primal;             /* p = <C, Proj(X)>                    (App. A, Sec. 5) */
  double dual;               /* d = a^T zeta + b^T gamma             (App. C.1) */
  double rel_gap;            /* (p - d) / max(|p|, |d|) */
  double kkt;                /* Delta_kkt of App. C.1 at the unrounded plan */
  double marg_viol;          /* ||Xhat 1 - a||_1 + ||Xhat^T 1 - b||_1 of the rounded plan */
  double grad_norm;          /* final ||g|| */
  double seconds;            /* wall time inside ibsn_solve */
  int32_t outer_iters, newton_iters, cg_iters, sinkhorn_iters;
  int32_t armijo_trials, polish_outer, reanchors, status;
  int64_t max_nnz;           /* largest nnz(P_rho) seen */
  int64_t dense_passes;      /* dense m x n passes launched */
  int64_t kernel_launches;   /* kernels this library launched during the solve */
  /* with params.profile: device time (CUDA events on the solve's stream),
   * launch count and algorithmic bytes per step kind, index kind + 8 * (1 if
   * the step ran in float64 passes else 0); kinds: 0 plan pass, 1 Armijo
   * pass, 2 stop-test pass, 3 sparsify pass + CSC build, 4 certificate pass,
   * 5 anchor pass, 6 persistent PCG, 7 other.  Algorithmic bytes: m*n*s_K
   * per dense pass that reads the anchored matrix (s_K = 4 or 8), plus m*n*s_K
   * written by the anchor pass, plus the cost matrix when it is read; for PCG,
   * per iteration 2*nnz*(4 + s_K) + 2*n*s_K + 8*(6n + 2m). */
  double pass_ms[16];
  int64_t pass_calls[16];
  double pass_bytes[16];
} ibsn_result;

/* Human-readable name of a status code. */
const char* ibsn_status_string(int status);
/* Text of the last CUDA error seen by this thread, or "". */
const char* ibsn_last_cuda_error(void);

/* Fill *p with the defaults listed above.  Never fails. */
void ibsn_params_default(ibsn_params* p);

/* Bytes of device workspace needed by a context for this problem and params.
 * The workspace must be 256-byte aligned.  Returns IBSN_ERR_INVALID_ARG or
 * IBSN_ERR_UNSUPPORTED for sizes the kernels do not cover. */
int ibsn_workspace_size(const ibsn_problem* prob, const ibsn_params* params, size_t* bytes);

/* Solve one problem: Alg. 2 with the stopping rules above.  The workspace is
 * device memory of at least ibsn_workspace_size bytes.  Returns IBSN_OK,
 * IBSN_NOT_CONVERGED (result still filled) or an error. */
int ibsn_solve(const ibsn_problem* prob, const ibsn_params* params, void* workspace,
               size_t workspace_bytes, ibsn_result* result, void* stream);

/* Solve `count` independent problems (the batched workload: many uneven OT
 * problems at once).  Problem q uses workspaces[q] (workspace_bytes[q] bytes,
 * from ibsn_workspace_size for probs[q]) and fills results[q] (its status in
 * results[q].status), exactly as ibsn_solve(&probs[q], params, ...) would:
 * the results are identical to solving the problems one by one.  The solves
 * run concurrently: `threads` host threads (<= 0: 8) take problems largest
 * first (by m n; ties in index order), each issuing its problems' kernels on
 * its own stream (streams[q]
 * when `streams` is not null, otherwise a stream the thread creates and
 * destroys), so passes of different problems overlap on the GPU.  Runs on the
 * calling thread's current device.  Returns IBSN_OK when every problem
 * converged, IBSN_NOT_CONVERGED when some did not, otherwise the first error
 * in problem order (the other problems are still solved). */
int ibsn_solve_batch(int count, const ibsn_problem* probs, const ibsn_params* params, void* const* workspaces,
                     const size_t* workspace_bytes, ibsn_result* results, void* const* streams, int threads);

/* ---------------------------------------------------------------------------
 * Step-level interface.  A context holds the state of one run of Alg. 2:
 * outer index k, cumulative potential Gamma^k (so that log X^k_ij equals
 * s_i + log b_j + (Gamma^k_j - k C_ij)/eta for some row constants s_i), the
 * current potential gamma, the anchored exponent matrix, and the sparsified
 * Hessian.  Each call below is one row of the hot path and is what ibsn_solve
 * runs internally.
 * ------------------------------------------------------------------------- */
typedef struct ibsn_ctx ibsn_ctx;

/* Create a context over a caller workspace; validates the problem (Eq. 1). */
int ibsn_ctx_create(const ibsn_problem* prob, const ibsn_params* params, void* workspace,
                    size_t workspace_bytes, void* stream, ibsn_ctx** out);
int ibsn_ctx_destroy(ibsn_ctx* ctx);

/* Outer update / anchor build (Alg. 2 outer update; Eq. 6): set k, Gamma
 * (device n) and gamma (device n), choose the working precision (0: float64
 * passes; 1: float32 passes; 2: float-float passes, K held as two float
 * planes, float64 arithmetic on every entry that does not underflow in
 * float32 -- needs a mixed context with polish) and rebuild the anchored
 * exponent matrix K_ij = log b_j + (Gamma_j + gamma_j - (k+1) C_ij)/eta - R_i.
 * Gamma may be NULL (zero). */
int ibsn_ctx_set_state(ibsn_ctx* ctx, int64_t k, const double* Gamma, const double* gamma,
                       int precision);

/* Plan pass (Eqs. 6-7): at the current gamma, writes the column sums
 * c = P^T a (device n, nullable) and the gradient norm ||c - b|| (host,
 * nullable). */
int ibsn_ctx_plan(ibsn_ctx* ctx, double* colsum, double* grad_norm);

/* Dense plan export for checks: P^k(gamma) as float64 m x n (device). */
int ibsn_ctx_export_plan(ibsn_ctx* ctx, double* P);

/* Current potential gamma (device n) copied out. */
int ibsn_ctx_get_gamma(ibsn_ctx* ctx, double* gamma);

/* Sinkhorn warm-up (Alg. 2, Eq. 3-4 alternating minimisation in semi-dual
 * form): repeat gamma_j += eta (log b_j - log c_j) until ||g|| < tol or
 * max_iter steps; then centre gamma.  Host outputs may be NULL. */
int ibsn_ctx_sinkhorn(ibsn_ctx* ctx, double tol, int32_t max_iter, int32_t* iters, double* grad_norm);

/* Hessian sparsification (Alg. 1) at the current gamma with threshold rho:
 * builds P_rho in CSR and CSC form plus c_rho = P_rho^T a.  nnz (host) is the
 * number of stored entries outside row i* (row i* is kept dense). */
int ibsn_ctx_sparsify(ibsn_ctx* ctx, double rho, int64_t* nnz);

/* Export P_rho as a dense float64 m x n matrix (device) for checks. */
int ibsn_ctx_export_sparse(ibsn_ctx* ctx, double* P_rho);

/* Newton direction (Alg. 2): solve (H_rho + shift I) Delta = -g by Jacobi-
 * preconditioned CG in one persistent kernel, H_rho applied matrix-free as
 * (c_rho o v - P_rho^T (a o (P_rho v)))/eta.  shift < 0 means ||g||.  The
 * direction is centred and kept in the context; delta (device n) nullable. */
int ibsn_ctx_newton_direction(ibsn_ctx* ctx, double shift, double rtol, int32_t max_cg,
                              double* delta, int32_t* cg_iters, double* resid);

/* Armijo trial (Alg. 2): for step t along the stored direction, returns
 * dL = L^k(gamma + t Delta) - L^k(gamma) (host) evaluated in a cancellation-
 * free form, and g^T Delta (host).  If accept != 0 and the Armijo inequality
 * holds, gamma moves to gamma + t Delta. *accepted reports that. */
int ibsn_ctx_armijo_trial(ibsn_ctx* ctx, double t, int32_t accept, double* dL, double* slope,
                          int32_t* accepted);

/* Inexact stopping test (Eq. 8): D_phi(Proj(X), X) for X = diag(a) P^k(gamma),
 * Proj by Alg. 3 (host out). */
int ibsn_ctx_stop_check(ibsn_ctx* ctx, double* dphi);

/* Certificate (App. A, App. C.1): primal of the rounded plan, c-transform dual,
 * relative gap, and marginal violation (host outs, nullable); the rounded plan
 * is written to plan (device m*n float64, nullable) and zeta (device m, nullable). */
int ibsn_ctx_certify(ibsn_ctx* ctx, double* primal, double* dual, double* rel_gap,
                     double* marg_viol, double* plan, double* zeta);

/* ---------------------------------------------------------------------------
 * Workspace-free plan pass.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory or pass a workspace
 * (for example code running where another runtime owns all allocations, or a
 * process that must keep its device footprint fixed after start-up).
 *
 * Computes, for the outer iterate given by (k, Gamma, gamma) exactly as
 * ibsn_ctx_set_state does, the column sums colsum = P^T a (device float64, n)
 * of that iterate's row-normalised plan P, whose entry (i, j) is proportional
 * to b_j exp((Gamma_j + gamma_j - (k+1) C_ij)/eta), and, if grad_norm is
 * non-NULL, ||colsum - b|| (host; the call then synchronises the stream).
 * Arithmetic is float64; the exponent is rebuilt from the cost for every
 * entry.  Gamma and gamma are device n-vectors, either may be NULL (zero).
 *
 * Unlike ibsn_ctx_create, this call does not validate the problem's values:
 * the caller must pass a, b > 0 summing to 1 and a finite C >= 0 (a
 * non-positive b_j, for instance, yields NaN results with status IBSN_OK).
 *
 * Scratch lives in one fixed array inside the library (about 4.1 MiB on every
 * GPU that loads it, held until the process exits); the call allocates
 * nothing.  Limits: n <= 4096 columns (larger n returns IBSN_ERR_UNSUPPORTED),
 * any m.  All calls share that array: calls whose kernels overlap on the GPU
 * race, so serialise them on one stream.  The first call on each device looks
 * up the array's device address and caches it for the life of the process;
 * make it before any CUDA stream capture, and do not use this call after a
 * cudaDeviceReset (or any teardown of the device's primary context): the
 * cached address would belong to the old context. */
int ibsn_plan_pass_noalloc(const ibsn_problem* prob, int64_t k, const double* Gamma, const double* gamma,
                           double* colsum, double* grad_norm, void* stream);

/* ---------------------------------------------------------------------------
 * Check of the bounded device waits.  The paper has no counterpart: the
 * persistent PCG kernels (Newton direction of Alg. 2) synchronise their blocks
 * with grid-wide barriers whose waits are bounded by params.wait_timeout_s;
 * this call runs that same barrier on its own so that a caller can check, on
 * its GPU, that a wait which can never complete ends with an error instead of
 * a hang.
 *
 * Launches `blocks` co-resident blocks (2 <= blocks <= the device's SM count)
 * that meet at one grid barrier.  With withhold = 0 all arrive and the call
 * returns IBSN_OK; with withhold != 0 block 0 leaves without arriving, the
 * others wait timeout_s seconds (0 < timeout_s <= 10), record the time-out and
 * return, and the call returns IBSN_ERR_TIMEOUT; the CUDA context stays
 * usable.  scratch: caller device memory of at least 8 bytes, 8-byte aligned
 * (overwritten).  Synchronises the stream.  IBSN_ERR_INVALID_ARG for bad
 * arguments, IBSN_ERR_CUDA when the launch fails. */
int ibsn_wait_probe(int blocks, int withhold, double timeout_s, void* scratch, void* stream);

/* ---------------------------------------------------------------------------
 * Learned warm start.  The paper starts every solve from gamma^{0,0} = 0
 * (Alg. 2).  These calls train and run a small network that predicts the
 * optimal dual potential gamma (cost units, centred) of a point-cloud problem
 * with squared-Euclidean cost, to be passed as params.gamma0; the zero start
 * stays as the fallback and ibsn_judge_warm_start picks the start with the
 * smaller semi-dual objective (Eq. 5).
 *
 * Network (three layers, width 128, bfloat16 weights, float32 arithmetic):
 *   source point i: e_i = relu(W_s [x_i1, x_i2, m a_i] + b_s)
 *   target point j: h_j = relu(W_t [y_j1, y_j2, n b_j] + b_t)
 *   p_s = mean_i e_i, p_t = mean_j h_j
 *   z_j = W_h [h_j; p_s; p_t] + b_h,  o_j = w_o . relu(z_j) + b_o
 *   gamma_hat_j = o_j - mean_l o_l
 * Parameters: one float32 vector of IBSN_WS_PARAM_COUNT values (the master
 * copy that Adam updates), laid out row-major as W_s 128x3, b_s 128, W_t 128x3,
 * b_t 128, W_h 128x384, b_h 128, w_o 128, b_o 1.  Every forward and backward
 * pass rounds them to bfloat16 (nearest, ties to even) and computes with the
 * rounded values; gradients are taken with respect to those rounded weights.
 * Loss of a batch of Q problems: (1/Q) sum_q (1/n_q) ||gamma_hat_q - centred
 * gamma*_q||^2.
 * ------------------------------------------------------------------------- */
#define IBSN_WS_HIDDEN 128
#define IBSN_WS_PARAM_COUNT 50433
#define IBSN_WS_MAX_POINTS 16384  /* per cloud and problem */

/* A batch of point-cloud problems.  Problem q has m[q] source and n[q] target
 * points (1 <= m[q], n[q] <= IBSN_WS_MAX_POINTS); its rows follow those of
 * problems 0..q-1 in the concatenated device arrays.  1 <= Q <= 65535.
 *
 * Errors of every call taking a batch: IBSN_ERR_INVALID_ARG for Q outside
 * [1, 65535], null m or n arrays, an empty cloud, or a null pointer argument;
 * IBSN_ERR_UNSUPPORTED for a cloud above IBSN_WS_MAX_POINTS; IBSN_ERR_WORKSPACE
 * for a null, misaligned (256 B) or too small workspace; IBSN_ERR_CUDA when a
 * copy or launch fails.  All of these are detected before any device work
 * except the last.  The caller owns every buffer; the calls allocate nothing. */
typedef struct ibsn_ws_batch {
  int32_t count;             /* Q >= 1 */
  int32_t reserved_;
  const int64_t* m;          /* host [Q] */
  const int64_t* n;          /* host [Q] */
  const double* x;           /* device, (sum m) x 2 row-major source coordinates */
  const double* y;           /* device, (sum n) x 2 target coordinates */
  const double* a;           /* device, sum m: source weights (each problem's sum 1) */
  const double* b;           /* device, sum n: target weights */
} ibsn_ws_batch;

/* Adam hyper-parameters (Kingma & Ba 2015, Algorithm 1). */
typedef struct ibsn_ws_adam {
  double lr;                 /* default 1e-3 */
  double beta1;              /* default 0.9 */
  double beta2;              /* default 0.999 */
  double eps;                /* default 1e-8 */
} ibsn_ws_adam;

/* Number of parameters (IBSN_WS_PARAM_COUNT). */
int64_t ibsn_ws_param_count(void);
/* Fill *hp with the defaults above.  Never fails. */
void ibsn_ws_adam_default(ibsn_ws_adam* hp);

/* Bytes of device workspace (256-byte aligned) for a batch of these sizes
 * (host only: reads batch->count, m and n). */
int ibsn_ws_workspace_size(const ibsn_ws_batch* batch, size_t* bytes);

/* Forward pass: gamma_hat (device, sum n float64, centred per problem).
 * Synchronises the stream once (the row offsets are copied from host). */
int ibsn_ws_predict(const ibsn_ws_batch* batch, const float* params, double* gamma_hat, void* workspace,
                    size_t workspace_bytes, void* stream);

/* Forward and backward pass against targets gamma_star (device, sum n; each
 * problem's target is centred inside): the batch loss (host, nullable; the
 * stream is synchronised for it, as it is once for the row offsets in every
 * call) and its gradient grad (device float32,
 * IBSN_WS_PARAM_COUNT, overwritten).  gamma_hat (device, nullable) receives
 * the prediction.  Reductions run in a fixed order: the result does not
 * depend on the launch or on timing. */
int ibsn_ws_loss_grad(const ibsn_ws_batch* batch, const float* params, const double* gamma_star, double* loss,
                      float* grad, double* gamma_hat, void* workspace, size_t workspace_bytes, void* stream);

/* One Adam step t >= 1 on `count` float32 parameters (device arrays params,
 * first and second moments m1, m2, updated in place; gradient grad).  Returns
 * IBSN_ERR_INVALID_ARG for count < 1, a null pointer, t < 1, lr <= 0, beta1 or
 * beta2 outside [0, 1) or eps <= 0; IBSN_ERR_CUDA when the launch fails. */
int ibsn_ws_adam_step(int64_t count, float* params, float* m1, float* m2, const float* grad, int64_t t,
                      const ibsn_ws_adam* hp, void* stream);

/* Judge a warm start for one problem against a fallback start (Alg. 2
 * starts from gamma = 0): the semi-dual objective of Eq. 5 at k = 0
 * (X^0 = a b^T),
 *   L^0(gamma) = -b^T gamma + eta sum_i a_i log sum_j a_i b_j exp((gamma_j - C_ij)/eta),
 * evaluated in float64 at gamma_hat (device n) and at the fallback
 * gamma_fallback (device n; NULL means the zero start), reported in
 * objective_warm / objective_fallback (host outs, nullable); *use_warm = 1 when
 * the warm start's value is finite and smaller than the fallback's.
 * Also reports the gradient norms of Eq. 7 from both starts (plan passes in
 * the working precision of `params`; host outs, nullable).  Uses the solver
 * workspace of ibsn_workspace_size.  Errors: IBSN_ERR_INVALID_ARG for a null
 * prob, params, gamma_hat or use_warm; otherwise those of ibsn_ctx_create
 * (problem validation, workspace), ibsn_ctx_set_state and ibsn_ctx_plan. */
int ibsn_judge_warm_start(const ibsn_problem* prob, const ibsn_params* params, const double* gamma_hat,
                          const double* gamma_fallback, void* workspace, size_t workspace_bytes,
                          double* objective_warm, double* objective_fallback, double* grad_norm_warm,
                          double* grad_norm_fallback, int32_t* use_warm, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* IBSN_H */
