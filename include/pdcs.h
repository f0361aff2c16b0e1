/*
 * pdcs.h -- C ABI of a restarted-PDHG conic solver for one NVIDIA B300 (sm_103a).
 *
 * Problem (PDCS technical note, Sec. 1.1, eq. prob_cp):
 *     min  c^T x   s.t.   G x - h  in  K_r,   l <= x[0:nb] <= u,   x[nb:n] in K_p
 * K_r (written K_d^* in the paper; the cone G x - h belongs to) and K_p are
 * ordered products of blocks from pdcs_cone_type.  The dual variable y lies in
 * the dual cone K_r^* (eq. dual_conic).
 *
 * Method: Algorithm 2 (diagonal rescaling, Sec. 2.6) around Algorithm 1 (restarted
 * PDHG with the adaptive step of Function 1, the adaptive reflected Halpern
 * iteration of Sec. 2.2, weighted averaging, the normalized-duality-gap restarts
 * of Sec. 2.3 computed by the bisection of Algorithm 3, and the primal-weight
 * rule of Sec. 2.5).  Termination uses the relative infinity-norm KKT errors of
 * Sec. 3.2.3 (eq. PDCS_terminate_tolerance_rel); exit codes follow Table 1.
 *
 * Every step after the host-to-device copy runs in this library's CUDA kernels on
 * the device that is current when pdcs_setup is called.
 *
 * Conventions for every entry point:
 *   - Return value: PDCS_OK (0) or a negative pdcs_error.  Solver outcomes are
 *     reported in pdcs_result.exit_code, never in the return value.
 *   - pdcs_last_error() returns a NUL-terminated message for the calling
 *     thread's most recent failure (valid until the next call from that thread).
 *   - Array arguments may be host or device pointers (cudaMemcpyDefault
 *     semantics); device arrays must live on the handle's device.
 *   - Inputs are copied: the caller may free or reuse them after the call.
 *   - Indices are 0-based; CSR column indices must be strictly increasing
 *     within each row.
 */
#ifndef PDCS_H
#define PDCS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Cone block types (Sec. 1.1 list of blocks; Sec. 3.2.3 row ordering).
 *   ZERO      {0}^d
 *   NONNEG    R_+^d
 *   SOC       {(t, w) : ||w||_2 <= t}, dim >= 1 (head first)
 *   RSOC      {(p, q, w) : 2 p q >= ||w||^2, p, q >= 0}, dim >= 2; handled by the
 *             orthogonal reformulation ((p+q)/sqrt2, (p-q)/sqrt2, w) -> SOC (Sec. 3)
 *   EXP       cl{(x, y, z) : y > 0, y exp(x / y) <= z}, dim == 3
 *   DUAL_EXP  cl{(u, v, w) : u < 0, -u exp(v / u) <= e w}, dim == 3            */
typedef enum {
  PDCS_CONE_ZERO = 0,
  PDCS_CONE_NONNEG = 1,
  PDCS_CONE_SOC = 2,
  PDCS_CONE_RSOC = 3,
  PDCS_CONE_EXP = 4,
  PDCS_CONE_DUAL_EXP = 5
} pdcs_cone_type;

typedef struct {
  int32_t type; /* pdcs_cone_type */
  int32_t pad;
  int64_t dim;
} pdcs_cone;

typedef enum {
  PDCS_OK = 0,
  PDCS_ERR_INVALID = -1,  /* bad argument: sizes, cone dims, CSR structure, NaN data */
  PDCS_ERR_CUDA = -2,     /* a CUDA runtime call failed */
  PDCS_ERR_NOMEM = -3,    /* device allocation failed */
  PDCS_ERR_TIMEOUT = -4,  /* a bounded device-side wait gave up */
  PDCS_ERR_UNSUPPORTED = -5
} pdcs_error;

/* Exit codes of Table 1. */
typedef enum {
  PDCS_EXIT_OPTIMAL = 0,
  PDCS_EXIT_MAX_ITER = 1,
  PDCS_EXIT_PRIMAL_INFEASIBLE_LOW_ACC = 2,
  PDCS_EXIT_PRIMAL_INFEASIBLE_HIGH_ACC = 3,
  PDCS_EXIT_DUAL_INFEASIBLE_LOW_ACC = 4,
  PDCS_EXIT_DUAL_INFEASIBLE_HIGH_ACC = 5,
  PDCS_EXIT_TIME_LIMIT = 6,
  PDCS_EXIT_CONTINUE = 7,
  PDCS_EXIT_NUMERICAL_ERROR = 8
} pdcs_exit_code;

/* Options; names and defaults follow the direct API of Sec. 3.2.3 where the
 * paper gives them.  Extra fields are this library's. */
typedef struct {
  double rel_tol;            /* 1e-6: max relative inf-norm KKT error to stop */
  double abs_tol;            /* 1e-6: used only when require_abs != 0 */
  double time_limit;         /* 1000 s (wall clock, checked between check periods) */
  int64_t max_iter;          /* accepted PDHG iterations; default INT64_MAX */
  int32_t use_preconditioner;/* 1: Ruiz + Pock-Chambolle rescaling (Sec. 2.6) */
  int32_t ruiz_iters;        /* 10 */
  double pc_alpha;           /* 1.0; negative skips the Pock-Chambolle pass */
  int32_t method;            /* 0 = average (compare both candidates), 1 = halpern */
  int32_t use_adaptive_restart; /* 1 */
  int64_t check_freq;        /* restart / termination check period: 64 */
  int32_t precision;         /* 0 = FP64 throughout, 1 = FP32 bulk with FP64
                                residuals, decisions, averages and exp Newton */
  int32_t require_abs;       /* 0: relative criterion only; 1: also abs_tol */
  double bisect_rel_tol;     /* 1e-3: Algorithm 3 stops when t_r - t_l <= tol * t_r
                                (the paper leaves the tolerance open) */
  int32_t verbose;           /* 0 silent, 1 one line per check period on stderr */
  int32_t trace_capacity;    /* >0: record one trace row per accepted iteration */
  int32_t profile;           /* 1: time every kernel launch on the device (see
                                pdcs_get_profile and pdcs_get_kernel_times) */
  int32_t eager;             /* 1: launch the kernels one by one from the host
                                instead of replaying captured graphs (slower; for
                                per-kernel profilers) */
  int32_t use_adaptive_step_size_weight; /* 1: the line search of Function 1 (Sec.
                                2.1); 0: every attempt is accepted with the fixed
                                step 1 / sqrt(||Ghat||_1 ||Ghat||_inf) (largest
                                column / row absolute sum of the rescaled matrix,
                                so that tau sigma ||Ghat||_2^2 <= 1) */
  int32_t use_duality_gap_restart; /* 1: at every check_freq-th iteration (the
                                paper's duality_gap_restart_freq) the restart
                                criterion is the normalized duality gap of Sec.
                                2.3 (KKT_omega when a gap is negative) */
  int32_t use_kkt_restart;   /* 0; 1: at every kkt_restart_freq-th iteration that
                                is not a gap check, the restart criterion is
                                KKT_omega (Sec. 2.3).  Checks with neither
                                criterion test termination and restart
                                condition 3 only */
  int32_t overlap_launches;  /* 0; 1: kernels of the captured loop bodies use
                                programmatic dependent launch (each may be
                                scheduled during its predecessor's last wave and
                                waits for it on the device).  Measured slower on
                                the portfolio (1955 against 2069 iterations/s) */
  int64_t kkt_restart_freq;  /* 2000 */
  int64_t print_freq;        /* 2000: with verbose, a line whenever the iteration
                                count passes a multiple (checked per period) */
  /* Infeasibility tests of Sec. 3.2.3 (exit codes 2-5), on the change of the
   * restart candidate between consecutive checks with the paper's ratios for
   * the homogeneous problem: primal infeasible when the dual error of
   * lambda = -G^T dy (plus the dual-cone violation of dy) over the dual
   * objective h^T dy + l^T lambda_1^+ - u^T lambda_1^- is below the threshold;
   * dual infeasible when the relative primal error of G dx (h = 0, plus the
   * violation of the recession cone of X by dx) over -c^T dx is below it.
   * The low-accuracy tests also need the candidates' dual objective (resp.
   * -c^T x) to have risen at each of the last 3 checks.  0 disables a test. */
  double eps_primal_infeasible_low_acc;   /* 1e-12 */
  double eps_dual_infeasible_low_acc;     /* 1e-12 */
  double eps_primal_infeasible_high_acc;  /* 1e-16 */
  double eps_dual_infeasible_high_acc;    /* 1e-16 */
} pdcs_options;

typedef struct {
  int32_t exit_code;  /* pdcs_exit_code */
  int32_t pad;
  double pobj, dobj;  /* c^T x and the dual objective of eq. dual_conic */
  double err_rel_p, err_rel_d, err_rel_gap;  /* eq. PDCS_terminate_tolerance_rel */
  double err_abs_p, err_abs_d, err_abs_gap;  /* eq. PDCS_terminate_tolerance_abs */
  double solve_time_s;   /* wall time of the call (setup excluded) */
  int64_t iters;         /* accepted PDHG iterations */
  int64_t attempts;      /* all PDHG attempts (kbar), rejected ones included */
  int64_t restarts;
} pdcs_result;

typedef struct pdcs_handle pdcs_handle;

/* Fill *opt with the defaults listed above. */
void pdcs_default_options(pdcs_options* opt);

/* Build a solver for one problem (Algorithm 2, line 1: rescaled instance data).
 *   out        receives the handle (NULL on failure).
 *   m, n       rows and columns of G (m >= 0, n >= 1).
 *   row_ptr    int64[m+1], col_idx int32[nnz], val float64[nnz]: CSR of G.
 *   h          float64[m];  c float64[n].
 *   nb         leading box-bounded columns (0 <= nb <= n).
 *   lb, ub     float64[nb] bounds (+-INFINITY allowed; lb <= ub); may be NULL
 *              when nb == 0.
 *   row_cones  n_row_cones blocks in order; their dims must sum to m.
 *   col_cones  n_col_cones blocks for x[nb:n]; dims must sum to n - nb.
 *   opt        options (NULL = defaults); copied.
 *   cuda_stream  caller's cudaStream_t (may be NULL).  The handle runs its
 *              kernels and graphs on a stream of its own; each call first makes
 *              that stream wait for work already queued on cuda_stream, and
 *              returns only after its own work has finished.
 * Errors: PDCS_ERR_INVALID for inconsistent sizes, unsorted or out-of-range
 * column indices, non-finite G/h/c entries, lb > ub, bad cone dims;
 * PDCS_ERR_NOMEM / PDCS_ERR_CUDA for device failures.  The handle owns all
 * device memory it allocates. */
int pdcs_setup(pdcs_handle** out, int64_t m, int64_t n, const int64_t* row_ptr,
               const int32_t* col_idx, const double* val, const double* h, const double* c,
               int64_t nb, const double* lb, const double* ub, const pdcs_cone* row_cones,
               int64_t n_row_cones, const pdcs_cone* col_cones, int64_t n_col_cones,
               const pdcs_options* opt, void* cuda_stream);

/* Run Algorithm 2 (Algorithm 1 on the rescaled problem, then unscale).
 *   x0 (n), y0 (m): optional warm start in the original variables (NULL = 0).
 *   x (n), y (m), s (m): caller-owned outputs (host or device; any may be NULL):
 *       primal x, dual y and slack s = G x - h of the returned point.
 *   res: summary (may be NULL).
 * Each call starts a fresh solve from (x0, y0). */
int pdcs_solve(pdcs_handle* handle, const double* x0, const double* y0, double* x, double* y,
               double* s, pdcs_result* res);

/* Complete solver state (checkpoint / resume; the loop variables of Algorithm 1).
 * Vectors that accompany it are in the solver's scaled, RSOC-reformulated
 * variables, float64: x, y = current Halpern iterate z^{t,k}; x0, y0 = anchor
 * z^{t,0}; xs, ys = running sums sum_i eta^{t,i} z^{t,i} of the weighted average. */
typedef struct {
  int64_t iter;      /* accepted iterations so far (all periods) */
  int64_t kbar;      /* attempts so far (accepted and rejected) */
  int64_t k;         /* accepted iterations in the current restart period */
  int64_t period;    /* restart period index t */
  int64_t restarts;
  double eta_hat;    /* step size of the next attempt */
  double eta_last;   /* accepted step of the last iteration */
  double omega;      /* primal weight */
  double wsum;       /* sum of accepted steps in the current period */
  int32_t has_ref;   /* a reference gap exists (t > 0) */
  int32_t has_prev;  /* a previous candidate of this period exists */
  double ref_rho, ref_abs_p, ref_abs_d, ref_abs_gap;     /* anchor's gap and 2-norm errors */
  double prev_rho, prev_abs_p, prev_abs_d, prev_abs_gap; /* previous candidate's */
} pdcs_state;

/* Copy the state left by the last pdcs_solve / pdcs_resume / pdcs_set_state.
 * Any vector pointer may be NULL; lengths n, m, n, m, n, m; host or device. */
int pdcs_get_state(pdcs_handle* handle, pdcs_state* state, double* x, double* y, double* x0,
                   double* y0, double* xs, double* ys);

/* Replace the solver state (all six vectors are required).  G x, G^T y and the
 * anchor's products are recomputed from the vectors.  Errors: PDCS_ERR_INVALID
 * for NULL arguments, a non-positive step size or primal weight, negative
 * counters. */
int pdcs_set_state(pdcs_handle* handle, const pdcs_state* state, const double* x,
                   const double* y, const double* x0, const double* y0, const double* xs,
                   const double* ys);

/* Continue Algorithm 1 from the current state until termination, the time
 * limit, or max_iter total accepted iterations (max_iter <= 0: the option's
 * value).  Outputs as in pdcs_solve. */
int pdcs_resume(pdcs_handle* handle, int64_t max_iter, double* x, double* y, double* s,
                pdcs_result* res);

/* Copy an internal iterate, in the solver's scaled and RSOC-reformulated
 * variables, to caller memory (host or device, float64).
 *   which: 0 = current Halpern iterate z^{t,k}, 1 = anchor z^{t,0},
 *          2 = last PDHG point zhat, 3 = scaling vectors (x <- D2, y <- D1). */
int pdcs_get_iterate(pdcs_handle* handle, int32_t which, double* x, double* y);

/* Copy up to cap trace rows (PDCS_TRACE_FIELDS doubles each, one per accepted
 * iteration, row i = iteration i + 1) to host memory; *count receives the
 * number of rows available.  Fields: iter, kbar, period, eta, eta_hat, beta,
 * omega, max_err, check, cand_avg, restart, rho_c (the candidate's restart
 * measure), fallback (1 at a check whose measure was KKT_omega, Sec. 2.3). */
#define PDCS_TRACE_FIELDS 13
int pdcs_get_trace(pdcs_handle* handle, double* out, int64_t cap, int64_t* count);

/* Device-measured cost of the sparse products of the last pdcs_solve /
 * pdcs_resume call (requires options.profile = 1; zero otherwise).  Each launch
 * is timed from the start of its first CTA to the end of its last CTA with the
 * GPU's global nanosecond timer.  bytes_* are the algorithmic bytes of one
 * launch: values once (8 bytes, 4 in FP32 mode), column indices once except
 * in the chunks of long rows (over 4096 nonzeros) that lie wholly inside the
 * row's column run (its longest stretch of at least 16 nonzeros with
 * consecutive columns, whose columns the kernel computes), row pointers once,
 * the gathered vector and the result vector once each; when the dual step
 * runs in the epilogue of G xhat (problems averaging 16 or more nonzeros per
 * row), g_bytes adds its per-row reads and writes. */
typedef struct {
  int64_t g_launches;    /* G xhat products (one per attempt) */
  double g_seconds;
  double g_bytes;        /* per launch */
  int64_t gt_launches;   /* G^T yhat products (one per accepted attempt) */
  double gt_seconds;
  double gt_bytes;       /* per launch */
  double nnz_flops;      /* 2 * nnz: multiply-adds of one launch, as flops */
  int64_t graph_launches;   /* check-period graphs launched by the call */
  int64_t kernel_launches;  /* kernels this library launched inside those graphs */
} pdcs_profile;

int pdcs_get_profile(pdcs_handle* handle, pdcs_profile* prof);

/* Device time of every kernel class during the last pdcs_solve / pdcs_resume
 * (requires options.profile = 1; *count = 0 otherwise), measured like
 * pdcs_profile.  Up to cap entries, in this order: spmv_g (G xhat), spmv_gt
 * (G^T yhat), spmv_check (products at checks and restarts), soc_grid (grid-wide
 * SOC projection), soc_cta (per-CTA SOC projection), exp (exponential-cone
 * projection), primal, dual, step (step-size test), res_prep, stats_attempt
 * (maxErr of zhat), stats_check (KKT statistics of the candidates), halpern,
 * probe_prep, probe_reduce (Algorithm 3 probes), check_misc. */
#define PDCS_KERNEL_CLASSES 16
int pdcs_get_kernel_times(pdcs_handle* handle, double* seconds, int64_t* launches, int32_t cap,
                          int32_t* count);

/* Sizes after set-up (m, n of the reformulated problem, nnz of G). */
int pdcs_get_sizes(pdcs_handle* handle, int64_t* m, int64_t* n, int64_t* nnz);

/* Release a handle (single problem or batch) and its device memory.  NULL-safe. */
void pdcs_free(pdcs_handle* handle);

/* Message for the calling thread's most recent failure. */
const char* pdcs_last_error(void);

/* ------------------------------------------------------------------------
 * Batched solves: many independent problems in one persistent kernel launch
 * (one thread block per problem at a time, largest first; every problem has
 * its own step sizes, primal weight, restarts and termination).  Each problem
 * is described as pdcs_setup's arguments; arrays may be host or device memory
 * and are copied.  SOC blocks of up to 4096 elements are projected with the
 * block held in registers, larger ones by streaming the block from memory on
 * every root-finding pass.  Limit: fewer than 2^31 columns in all.  Set-up also
 * picks the lanes per row of the sparse products for four size buckets by
 * timing a few problems of each (autotuning).  options.time_limit applies to
 * each problem from its start. */
typedef struct {
  int64_t m, n;
  const int64_t* row_ptr;
  const int32_t* col_idx;
  const double* val;
  const double* h;
  const double* c;
  int64_t nb;
  const double* lb;
  const double* ub;
  const pdcs_cone* row_cones;
  int64_t n_row_cones;
  const pdcs_cone* col_cones;
  int64_t n_col_cones;
} pdcs_instance;

int pdcs_setup_batch(pdcs_handle** out, const pdcs_instance* instances, int64_t count,
                     const pdcs_options* opt, void* cuda_stream);
/* Solve every problem from the cold start.  x (sum of n), y and s (sum of m):
 * the problems' outputs concatenated in input order (any may be NULL); res:
 * count results (solve_time_s = that problem's own time on its thread
 * block); finish_s (may be NULL): count times from the first problem's start
 * to each problem's end. */
int pdcs_solve_batch(pdcs_handle* handle, double* x, double* y, double* s, pdcs_result* res,
                     double* finish_s);

/* ------------------------------------------------------------------------
 * Warm-start network (the paper has no counterpart: a learned starting point
 * for parameterised problem families).  A fully connected ReLU network
 * in_dim -> hidden (n_hidden layers) -> out_dim trained with mean squared
 * error and Adam; GEMMs on the tensor cores in BF16 with FP32 accumulation,
 * master weights and Adam moments in FP32.  Weights start Glorot-uniform
 * (SplitMix64 stream from seed), biases at zero.
 * Data arguments are row-major FP32 (batch x in_dim inputs, batch x out_dim
 * targets / outputs), host or device memory; the calls return when their
 * outputs are in place.  Errors: PDCS_ERR_INVALID (arguments),
 * PDCS_ERR_NOMEM / PDCS_ERR_CUDA, PDCS_ERR_TIMEOUT (a GEMM wait gave up). */
typedef struct pdcs_mlp pdcs_mlp;

typedef struct {
  int64_t in_dim;     /* inputs per sample */
  int64_t hidden;     /* width of every hidden layer */
  int32_t n_hidden;   /* hidden layers (>= 1) */
  int32_t pad;
  int64_t out_dim;    /* outputs per sample */
  int64_t max_batch;  /* largest batch of any call */
  double lr, beta1, beta2, eps;  /* Adam */
  uint64_t seed;
} pdcs_mlp_config;

void pdcs_mlp_default_config(pdcs_mlp_config* cfg); /* hidden 512 x 3, batch 256, Adam 1e-3 */
int pdcs_mlp_create(pdcs_mlp** out, const pdcs_mlp_config* cfg, void* cuda_stream);
/* One Adam step on the batch's mean squared error; *loss (may be NULL)
 * receives the loss before the step. */
int pdcs_mlp_train_step(pdcs_mlp* net, const float* X, const float* T, int64_t batch, double* loss);
/* Gradients of the batch loss for one layer (dW: d_out x d_in, db: d_out;
 * either may be NULL), without updating anything. */
int pdcs_mlp_gradients(pdcs_mlp* net, const float* X, const float* T, int64_t batch, int32_t layer,
                       float* dW, float* db, double* loss);
int pdcs_mlp_predict(pdcs_mlp* net, const float* X, int64_t batch, float* Y);
/* Master (FP32) weights of layer 0 .. n_hidden: W is d_out x d_in row-major.
 * set_layer also resets the Adam moments and step count. */
int pdcs_mlp_get_layer(pdcs_mlp* net, int32_t layer, float* W, float* b);
int pdcs_mlp_set_layer(pdcs_mlp* net, int32_t layer, const float* W, const float* b);
void pdcs_mlp_free(pdcs_mlp* net); /* NULL-safe */

/* KKT errors of a given point (original variables; x: n, y: m, host or
 * device; NULL = zeros) under the termination definitions of Sec. 3.2.3:
 * res receives pobj, dobj and the err_* fields as pdcs_solve reports them,
 * exit_code 0 if the point meets the termination test and -1 otherwise,
 * iters = attempts = restarts = 0.  Replaces the handle's iterate, like a
 * solve would. */
int pdcs_kkt(pdcs_handle* handle, const double* x, const double* y, pdcs_result* res);

/* y = G x for a CSR matrix held in device memory, without allocating.  The
 * paper has no counterpart: this is a service for callers that must not
 * allocate device memory when they call, for example code running while a
 * caching allocator (such as PyTorch's) owns the device's whole memory
 * budget, where a cudaMalloc would fail or force the allocator to give its
 * cache back.
 *   m, n: rows and columns of G (m = 0: nothing to do).
 *   row_ptr int64 [m+1], col_idx int32 [nnz] (entries in [0, n)),
 *   val float64 [nnz], x float64 [n], y float64 [m] (written): all device
 *   memory of the current device; host pointers are rejected.
 *   cuda_stream: the stream the work is ordered on (NULL: legacy default).
 * Scratch: one fixed device array of about 0.8 MB inside the library, sized
 * for at most 4096 rows with more than 4096 nonzeros and at most 65536
 * chunks of 4096 nonzeros among them.  Rows of up to 4096 nonzeros have no
 * limit.  The call checks the matrix against those limits on the device: a
 * matrix beyond either is rejected there (nothing computed, y left as it
 * was) and counted, and pdcs_spmv_noalloc_status reports the count.
 * The call never synchronises: it enqueues two kernels on cuda_stream and
 * returns; y is ready when the stream reaches them.  It may be captured into
 * a graph, except the first call on a device (it looks up the scratch's
 * device address with that device current, then caches it), which returns
 * PDCS_ERR_INVALID inside a capture and leaves the capture intact.  It
 * allocates no device memory and, when it succeeds, no host memory either; a
 * rejected call stores its message for pdcs_last_error.
 * The scratch's tickets must be zero when a call starts: they are zero when
 * the library is loaded and every completed call leaves them zero (a call
 * cut short by a device error does not).  All calls on one device share the
 * scratch, so calls that overlap in time race: serialise them.  Results are
 * deterministic (fixed summation order) but round differently from the
 * solver's own product.
 * Returns PDCS_OK, PDCS_ERR_INVALID (sizes, NULL or host pointers, a first
 * call inside a capture) or PDCS_ERR_CUDA. */
int pdcs_spmv_noalloc(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                      const double* val, const double* x, double* y, void* cuda_stream);

/* How many pdcs_spmv_noalloc calls on the current device were rejected on
 * the device (matrix beyond the scratch's limits) since the previous query;
 * the count is then reset to zero.  Synchronises cuda_stream (the stream the
 * calls were ordered on, so that the count includes them); it therefore
 * returns PDCS_ERR_INVALID, without touching the count, while cuda_stream is
 * being captured.  rejected: host int64, written (0 on error).
 * Returns PDCS_OK, PDCS_ERR_INVALID or PDCS_ERR_CUDA. */
int pdcs_spmv_noalloc_status(void* cuda_stream, int64_t* rejected);

#ifdef __cplusplus
}
#endif

#endif /* PDCS_H */
