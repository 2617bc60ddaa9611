/*
 * mv.h -- C ABI of the GB300 (sm_103a) NPGA library for constrained
 * mean--variance portfolios.
 *
 * Problem (Sec. 1, Eq. mv; Sec. 3.1, Eq. npga-unified-grad):
 *     minimise  f(x) = ||L_eff^T x||_2^2 + gamma ||x||_2^2
 *     over      F = { x in R^n : mu^T x >= R_target, 1^T x = 1, x >= 0 }
 * where L_eff is the centered covariance factor L (Sec. 2.1), its sketch
 * L Phi (Sec. 2.3) or the STR factor (Sec. 2.5), so Sigma = L_eff L_eff^T.
 *
 * Conventions shared by every call
 *  - Pointers named d_* are DEVICE pointers owned by the caller; pointers
 *    named h_* are HOST pointers.  The library never frees caller memory and
 *    never allocates device memory inside a call: scratch comes from a
 *    caller-provided device workspace whose size the matching
 *    *_workspace_size query returns.  Workspaces must be 256-byte aligned.
 *  - Matrices are row-major: row i (one asset) holds T periods; element
 *    (i, t) sits at i * ld + t.  For 16-byte vector access, the base pointer
 *    must be 16-byte aligned and ld * sizeof(element) a multiple of 16
 *    (ld % 4 == 0 for F32, % 8 for BF16, % 16 for FP8).  Violations return
 *    MV_ERR_INVALID_ARG before anything is launched.
 *  - All work is enqueued on the given stream (NULL = legacy default
 *    stream).  Calls documented as "blocking" synchronise that stream before
 *    they return; the others are asynchronous.
 *  - Return codes are mv_status.  Argument errors are detected on the host
 *    before launch; failures found on the device are reported through the
 *    info structs named in each call.
 */
#ifndef MV_H
#define MV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t; declared here so this header needs no CUDA headers. */
typedef struct CUstream_st *mv_stream_t;

typedef enum {
    MV_OK = 0,
    MV_ERR_INVALID_ARG = 1,    /* bad pointer, size, alignment or option          */
    MV_ERR_INFEASIBLE = 2,     /* F is empty: R_target > max mu (or < min mu, EQ) */
    MV_ERR_NOT_CONVERGED = 3,  /* iteration budget hit; best iterate returned     */
    MV_ERR_TIMEOUT = 4,        /* a bounded device-side wait gave up               */
    MV_ERR_NUMERIC = 5,        /* NaN or Inf met in data or iterates               */
    MV_ERR_CUDA = 6,           /* a CUDA runtime call failed                       */
    MV_ERR_UNSUPPORTED = 7,    /* valid request this build does not implement      */
    MV_ERR_WORKSPACE = 8       /* workspace NULL, too small or misaligned          */
} mv_status;

typedef enum {
    MV_F32 = 0,        /* float                                                 */
    MV_BF16 = 1,       /* bfloat16 storage, FP32 accumulation                   */
    MV_FP8_E4M3 = 2    /* fp8 e4m3 storage with one FP32 scale per row (asset)  */
} mv_dtype;

typedef enum {
    MV_RETURN_GE = 0,  /* mu^T x >= R_target: the set F of Sec. 1 / Sec. 3.1    */
    MV_RETURN_EQ = 1   /* mu^T x == R_target: equality variant (nu of any sign) */
} mv_return_mode;

/* Storage layout of the factor L (n assets x T periods) in device memory. */
typedef enum {
    MV_LAYOUT_NT = 0,  /* n x T row-major (one asset per row), leading dim >= T  */
    MV_LAYOUT_TN = 1,  /* L^T stored: T x n row-major (one period per row),
                          leading dim >= n.  The solve's products read it in
                          long runs along assets, which streams faster.  Only
                          centering, the gradient and the single-problem solves
                          (plain and refined) accept it.                        */
    MV_LAYOUT_SIGMA = 2 /* not a factor: the problem's matrix is the explicit
                          covariance Sigma itself, n x n FP32 (symmetric; only
                          the entries on and above the diagonal are read),
                          leading dim ld >= n (a multiple of 4).  The gradient is
                          2 Sigma y + 2 gamma y (the classical model of Sec. 3's
                          remark); T is not read.  Formed by mv_sigma_form.
                          Accepted by mv_npga_workspace_size, mv_npga_solve,
                          mv_npga_solve_refined and mv_gradient (with d_z NULL). */
} mv_layout;

/* Human-readable name of a status code (static string, never NULL). */
const char *mv_status_string(int status);

/* Library version string, e.g. "mv 0.1 sm_103a". */
const char *mv_version(void);

/* Description of the last CUDA runtime failure seen by this thread (the call,
 * its error name and source location), or "" if none.  Valid until the next
 * failing call on the same thread. */
const char *mv_last_error(void);

/* ------------------------------------------------------------------------
 * 1. Centering (Sec. 2.1):  mu = R 1_T / T,   L = (R - mu 1_T^T) / sqrt(T - 1),
 *    trace(Sigma) = ||L||_F^2.
 *
 *  d_R        [in]  n x T returns, FP32, row-major with leading dim ldR >= T.
 *  out_dtype  [in]  storage type of L (MV_F32, MV_BF16 or MV_FP8_E4M3).
 *  layout     [in]  mv_layout of d_L.
 *  d_L        [out] the factor in that type: MV_LAYOUT_NT: n x T, leading dim
 *                   ldL >= T, columns T..ldL-1 of every row written as zeros;
 *                   MV_LAYOUT_TN: L^T, T x n, leading dim ldL >= n, columns
 *                   n..ldL-1 written as zeros (a tiled transpose on the way).
 *  d_row_scale[out] FP8 only (else may be NULL): n FP32 scales s_i such that
 *                   L(i,t) ~= s_i * q(i,t); s_i = max_t |L(i,t)| / 448.
 *  d_mu       [out] n FP64 sample means.
 *  d_trace    [out] one FP64: ||L||_F^2 = trace(Sigma), summed in FP64 from the
 *                   unrounded centered values.
 *  Sums are FP64.  Requires n >= 1, T >= 2.  Asynchronous.
 * ------------------------------------------------------------------------ */
size_t mv_center_workspace_size(int64_t n, int64_t T);
int mv_center_factor(const float *d_R, int64_t n, int64_t T, int64_t ldR,
                     int out_dtype, int layout, void *d_L, int64_t ldL, float *d_row_scale,
                     double *d_mu, double *d_trace,
                     void *d_ws, size_t ws_bytes, mv_stream_t stream);

/*  The same from returns in HOST memory: h_R is n x T FP32 row-major (ldR >= T),
 *  best page-locked.  The rows are uploaded in chunks of about 64 MB on an
 *  internal copy stream into two device staging buffers inside the
 *  workspace, and each chunk is centred on `stream` while the next one is in
 *  flight, so the upload and the centering overlap.  Outputs as
 *  mv_center_factor; workspace mv_center_host_workspace_size(n, T) bytes.
 *  Asynchronous with respect to the host for page-locked h_R; h_R must stay
 *  valid until `stream` reaches the end of the call's work. */
size_t mv_center_host_workspace_size(int64_t n, int64_t T);
int mv_center_factor_host(const float *h_R, int64_t n, int64_t T, int64_t ldR,
                          int out_dtype, int layout, void *d_L, int64_t ldL, float *d_row_scale,
                          double *d_mu, double *d_trace,
                          void *d_ws, size_t ws_bytes, mv_stream_t stream);

/* ------------------------------------------------------------------------
 * 2. Exact projection onto F (Sec. 3.1, Eqs. simplex-tau, simplex-proj,
 *    projF-dualpath), batched over problems that share mu.
 *
 *  x(nu) = Pi_Delta(v + nu mu) with the simplex threshold tau(nu) from
 *  sum_i max(v_i + nu mu_i - tau, 0) = 1; phi(nu) = mu^T x(nu) is
 *  nondecreasing.  If phi(0) >= R_target the simplex projection is returned
 *  (nu = 0); otherwise nu > 0 solves phi(nu) = R_target.  The search over
 *  tau and nu is a safeguarded Newton iteration on these piecewise-linear
 *  functions, finished exactly on the identified support S by solving the
 *  two linear equations of the budget and return rows.  FP64 throughout.
 *
 *  d_v        [in]  batch x n FP64 points to project (row b = problem b).
 *  d_mu       [in]  n FP64 expected returns, shared by the batch.
 *  d_R_target [in]  batch FP64 targets.
 *  mode       [in]  mv_return_mode.
 *  d_x        [out] batch x n FP64 projections.
 *  d_info     [out] batch mv_proj_info (device memory).  info.status is
 *                   MV_OK, MV_ERR_INFEASIBLE (x filled with NaN) or
 *                   MV_ERR_NOT_CONVERGED (step budget hit; best x kept).
 *  Needs no workspace.  1 <= n <= 32768, batch <= 65535.  One cluster of up to
 *  16 thread blocks per problem.  Asynchronous.
 * ------------------------------------------------------------------------ */
typedef struct {
    double nu;         /* multiplier of the return row (0 when inactive)      */
    double tau;        /* simplex threshold at nu                              */
    double residual;   /* mu^T x - R_target                                    */
    int32_t support;   /* |{i : x_i > 0}|                                      */
    int32_t status;    /* mv_status of this problem                            */
    int32_t steps;     /* block-wide reductions spent                          */
    int32_t active;    /* 1 if the return row is tight (nu != 0)               */
} mv_proj_info;

int mv_project(const double *d_v, const double *d_mu, const double *d_R_target,
               int64_t n, int64_t batch, int mode, double *d_x,
               mv_proj_info *d_info, mv_stream_t stream);

/* ------------------------------------------------------------------------
 * 3. NPGA solve (Algorithm 1 with the fixed step of Sec. 3.1).
 *
 *  Step size: alpha = 1 / (2 (lambda_hat (1 + power_safety) + gamma)) where
 *  lambda_hat = ||L_eff^T u||^2 after power_iters steps of the power method
 *  u <- L(L^T u)/||.|| (Sec. 3.1 remark), unless opts.alpha > 0 overrides it.
 *  With opts.lanczos = 1, lambda_hat is instead the other estimate the
 *  fixed step of Sec. 3.1 names, the largest singular value of L_eff
 *  (squared): the top eigenvalue of the tridiagonal matrix of power_iters
 *  Lanczos steps on L L^T from the same start vector (three-term recurrence
 *  on FP32 vectors with FP64 alpha_j, beta_j, no reorthogonalisation; the
 *  eigenvalue in FP64 by Sturm-count multisection).  It is never below the power
 *  method's estimate after power_iters - 1 steps and costs the same product
 *  per step, so far fewer steps reach the same accuracy on a clustered top
 *  spectrum.
 *  Iteration k: z = L^T y^k (FP32 accumulation), g = 2 L z + 2 gamma y^k,
 *  v = y^k - alpha g, x^{k+1} = Pi_F(v) (FP64), FISTA momentum
 *  t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2, beta_k = (t_k - 1)/t_{k+1},
 *  y^{k+1} = x^{k+1} + beta_k (x^{k+1} - x^k).  Every kkt_every iterations
 *  the residual ||Pi_F(x^k - alpha grad f(x^k)) - x^k||_2 is evaluated and
 *  the solve stops at x^k once it is <= eps.  grad f(x^k) is obtained from
 *  the products already computed at y^k by linearity
 *  (L L^T x^k = (L L^T y^k + beta_{k-1} L L^T x^{k-1}) / (1 + beta_{k-1})),
 *  so the check costs one projection and no extra pass over L.
 * ------------------------------------------------------------------------ */
typedef struct {
    const void *L;            /* d: the factor (dtype) in `layout`, leading dim ld       */
    int32_t dtype;            /* mv_dtype                                                */
    int32_t mode;             /* mv_return_mode                                          */
    const float *row_scale;   /* d: n FP32 row scales (FP8 only, else NULL)              */
    int64_t n, T, ld;         /* 1 <= n <= 32768 assets, T >= 1 periods; ld >= T (NT)
                                 or ld >= n (TN)                                         */
    double gamma;             /* ridge (0 for the full and sketched models)              */
    const double *mu;         /* d: n FP64 expected returns                              */
    double R_target;          /* target return                                           */
    const double *power_start;/* d: n FP64 start of the power method (or Lanczos); NULL =
                                 all ones                                                */
    int32_t layout;           /* mv_layout of L (MV_LAYOUT_TN: T x n, ld >= n)           */
    int32_t reserved;         /* 0                                                       */
} mv_problem;

typedef struct {
    int32_t max_iter;         /* iteration budget (default 10000)                        */
    int32_t kkt_every;        /* KKT check period (default 5, Sec. 5.2)                 */
    int32_t power_iters;      /* power-method (or Lanczos) steps (default 50)            */
    int32_t warm_start;       /* 1: x_inout holds x^0 in F; 0: x^0 = Pi_F(1/n)           */
    double eps;               /* KKT tolerance (default 1e-6)                            */
    double power_safety;      /* lambda_hat is multiplied by (1 + this); default 1e-3    */
    double alpha;             /* > 0: fixed step override; <= 0: from lambda_hat          */
    int32_t use_graph;        /* 1 (default): replay iterations as a CUDA graph          */
    int32_t timing;           /* 1: time every loop launch with CUDA events (kernels are
                                 then issued from the host instead of a graph)           */
    int32_t checkpoint_every; /* mv_npga_backward: iterations between checkpoints (50)   */
    int32_t two_pass;         /* 1: always stream L twice per product (z = L^T y, then
                                 L z); 0 (default): use the fused single pass for
                                 L L^T y where it applies (see below)                   */
    /* Step and momentum variants of Sec. 3.1 (mv_npga_solve only): */
    int32_t momentum;         /* 0 (default): the t_k-based FISTA update of Algorithm 1;
                                 1: the strongly convex specialisation, beta fixed at
                                 (1 - sqrt(alpha m_f)) / (1 + sqrt(alpha m_f))          */
    int32_t backtrack;        /* 1: accelerated backtracking from the trial step
                                 bt_alpha0 (<= 0: the power-method step times
                                 1 / bt_rho^4), shrunk by bt_rho until
                                 ||L^T d||^2 + gamma ||d||^2 <= ||d||^2 / (2 alpha),
                                 d = x+ - y; the step never grows again              */
    double m_f;               /* lower curvature bound for momentum = 1 (> 0; <= 0 takes
                                 2 gamma, which needs gamma > 0)                        */
    double bt_rho;            /* shrink factor in (0, 1) (default 0.5)                    */
    double bt_alpha0;         /* first trial step (see backtrack)                         */
    int32_t proj_budget;      /* outer steps of each projection's scalar search before
                                 the Dykstra safeguard takes over (default 100)         */
    int32_t dykstra_iters;    /* sweeps of the Dykstra safeguard (default 2000; 0: off)   */
    int32_t lanczos;          /* 1: lambda_hat from power_iters Lanczos steps (1..512); 0
                                 (default): the power method.  mv_npga_solve, the refined
                                 and the frontier solves; the batched and adjoint solves
                                 return MV_ERR_UNSUPPORTED for 1                        */
    int32_t reserved_opts;    /* 0                                                       */
} mv_solve_opts;

typedef struct {
    int32_t iterations;       /* k at return (x^k is returned)                           */
    int32_t status;           /* MV_OK, MV_ERR_NOT_CONVERGED, MV_ERR_INFEASIBLE, ...     */
    int32_t converged;        /* 1 if kkt <= eps                                         */
    int32_t proj_failures;    /* projections that hit their step budget                  */
    double kkt;               /* residual of the returned x                              */
    double objective;         /* f(x) = ||L^T x||^2 + gamma ||x||^2: x^T (L L^T x) from  */
                              /* the product the last KKT test kept, else one more pass  */
    double alpha;             /* step used                                               */
    double lambda_hat;        /* power or Lanczos estimate of ||L_eff||_2^2 (0 if overridden) */
    double nu;                /* return-row multiplier of the last projection            */
    int32_t launches;         /* kernels this call launched (including no-op tails)      */
    int32_t timed_pairs;      /* loop iterations whose kernels were timed (timing = 1)   */
    double t_gemv_t_ms;       /* summed device time of those gemv_t launches             */
    double t_gemv_n_ms;       /* summed device time of those gemv_n launches             */
    double t_step_ms;         /* summed device time of those step (projection) launches  */
    int32_t proj_steps;       /* block-wide reductions spent by all projections          */
    int32_t refine_iterations;/* mv_npga_solve_refined: iterations of the FP32 phase     */
    int32_t fused;            /* 1: the loop used the fused single pass over L;
                                 2: the symmetric pass over an explicit Sigma; 0: two
                                 passes over L                                            */
    double t_fused_ms;        /* summed device time of the timed single-pass products    */
    int32_t backtracks;       /* rejected trial steps (backtrack = 1)                     */
    int32_t dykstra;          /* projections finished through the Dykstra safeguard       */
} mv_solve_info;

void mv_solve_opts_default(mv_solve_opts *opts);
size_t mv_npga_workspace_size(const mv_problem *P);

/*  Fused single pass.  The loop and the power method need only the product
 *  L L^T y, never z = L^T y itself, so where n >= 1024 and T >= 4096 and a
 *  shape fits (n up to about 6800) the two half-products run in one pass
 *  over L: a cluster of 2 to 8 CTAs holds a 32- to 128-byte column block of
 *  all n rows in shared memory, forms that block's slice of L^T y from it,
 *  exchanges it through distributed shared memory and adds
 *  L_block (L_block^T y) to g from the same staged block.  L is then read
 *  from HBM once per iteration instead of twice.  opts.two_pass = 1 turns
 *  it off; elsewhere the two-pass kernels run.
 *
 *  d_x_inout [in/out] n FP64: x^0 when opts.warm_start = 1 (must lie in F),
 *                     the solution x^k on return.
 *  h_info    [out]    host struct, filled on return.
 *  Blocking: the call synchronises `stream` once per kkt_every iterations to
 *  read the device-side convergence flag, and returns when the solve is done. */
int mv_npga_solve(const mv_problem *P, const mv_solve_opts *opts, double *d_x_inout,
                  mv_solve_info *h_info, void *d_ws, size_t ws_bytes, mv_stream_t stream);

/* ------------------------------------------------------------------------
 * 3a'. Explicit covariance (Sec. 3, remark on the classical model).
 *
 *  mv_sigma_form writes Sigma = L L^T (n x n FP32, both triangles, exactly
 *  symmetric) from the centered factor P->L (MV_LAYOUT_NT; F32, BF16 or
 *  FP8 e4m3 with row scales).  Tensor cores (tcgen05, BF16 operands, FP32
 *  accumulation) multiply only the tiles on and above the diagonal:
 *    MV_BF16 / MV_FP8_E4M3  exact products of the stored values (FP8 values
 *                           are BF16 values; the row scales multiply the
 *                           result), FP32 sums;
 *    MV_F32                 L = H + D split into two BF16 parts and
 *                           Sigma = H H^T + H D^T + D H^T (three K-passes);
 *                           per product term the error is below about
 *                           2^-16 |L_it L_jt|, plus FP32 summation.
 *  The solve then takes a problem with layout MV_LAYOUT_SIGMA, L = Sigma,
 *  ld = ldS: each NPGA iteration reads the upper triangle of Sigma once
 *  (n^2/2 FP32, held in L2 for n up to about 5500) instead of L twice.
 *  d_ws: mv_sigma_workspace_size(P) bytes (256-byte aligned; the BF16
 *  split or expansion of L, 2 n T or 4 n T bytes).  Blocking: returns
 *  after the GEMM, MV_ERR_TIMEOUT if a pipeline wait gave up.
 * ------------------------------------------------------------------------ */
size_t mv_sigma_workspace_size(const mv_problem *P);
int mv_sigma_form(const mv_problem *P, float *d_Sigma, int64_t ldS, void *d_ws, size_t ws_bytes,
                  mv_stream_t stream);

/* ------------------------------------------------------------------------
 * 3b. Low-precision solve with FP32 refinement (an extension: the paper does
 *     not state its precision).  The bandwidth-bound products stream L in
 *     BF16 (half the bytes) or FP8 e4m3 with row scales (a quarter); the
 *     result is then refined on the FP32 copy of the same factor.
 *
 *  Phase 1: mv_npga_solve(P_lo) to a KKT residual <= eps_lo, with its own
 *  step estimate (power method, or Lanczos with opts->lanczos).  Phase 2: mv_npga_solve(P_hi) warm-started from that point,
 *  with the fixed step alpha_lo / (1 + 1e-2) (the spectral norms of the two
 *  copies differ by far less than 1%, so the step stays admissible) and no
 *  second estimate, until the KKT residual of P_hi is <= opts->eps.
 *  P_lo and P_hi must describe the same problem (n, T, gamma, mu, target,
 *  mode); P_hi->dtype must be MV_F32.  The two copies may use different
 *  layouts (each its fastest).  Workspace: the larger of the two
 *  mv_npga_workspace_size values.  h_info: iterations = both phases,
 *  refine_iterations = phase 2, kkt/objective/alpha of phase 2.  Blocking.
 * ------------------------------------------------------------------------ */
int mv_npga_solve_refined(const mv_problem *P_lo, const mv_problem *P_hi, const mv_solve_opts *opts,
                          double eps_lo, double *d_x_inout, mv_solve_info *h_info,
                          void *d_ws, size_t ws_bytes, mv_stream_t stream);

/* ------------------------------------------------------------------------
 * 3e. Efficient frontier: one factor, many targets (batched NPGA).
 *
 *  Solves the problem of P (L stored as MV_BF16) for n_targets <= 128
 *  targets R_b at once (up to 128 points on the efficient frontier).  The
 *  half-products of all targets are skinny tensor-core GEMMs
 *  Z = L^T [y_1..y_B], G = L Z (tcgen05, BF16 operands, FP32 accumulation)
 *  with the vector operands carried as a BF16 hi + lo pair, so accuracy is
 *  that of the BF16 model; L^T is formed once in the workspace.  One shared
 *  step estimate (power method, or Lanczos with opts->lanczos) sets alpha; each target has its own FISTA state, KKT test
 *  and stopping point; a chunk of kkt_every iterations is replayed as one
 *  CUDA graph.  P->R_target is ignored.
 *  d_R_targets [in]  n_targets FP64 targets (device).
 *  d_X         [out] n_targets x n FP64 solutions (row b = target b).
 *  h_infos     [out] n_targets host mv_solve_info (objective = BF16 model).
 *  Returns the first non-OK per-target status (or MV_OK).  Blocking.
 * ------------------------------------------------------------------------ */
size_t mv_frontier_workspace_size(const mv_problem *P, int64_t n_targets);
int mv_npga_solve_frontier(const mv_problem *P, const double *d_R_targets, int64_t n_targets,
                           const mv_solve_opts *opts, double *d_X, mv_solve_info *h_infos,
                           void *d_ws, size_t ws_bytes, mv_stream_t stream);

/*  The frontier with FP32 refinement (as mv_npga_solve_refined for one
 *  target): phase 1 is mv_npga_solve_frontier on P_lo (BF16 or FP8) until
 *  every target's KKT residual is <= eps_lo; phase 2 restarts every target
 *  from its phase-1 answer (FISTA state reset, warm start) on the FP32 factor
 *  P_hi (MV_LAYOUT_NT, same n, T, mu, gamma and mode), carried as the BF16
 *  pair H = bf16(L), D = bf16(L - H) (which carries each entry of L to
 *  2^-18 relative) and multiplied by both in every GEMM, with the phase-1
 *  step divided by 1.01, until
 *  each residual on the FP32 model is <= opts->eps.  h_infos: iterations =
 *  both phases, refine_iterations = phase 2, kkt and objective of the FP32
 *  model.  Workspace mv_frontier_refined_workspace_size (adds 4 n T bytes x 2
 *  for H, D and their transposes).  Blocking. */
size_t mv_frontier_refined_workspace_size(const mv_problem *P_lo, const mv_problem *P_hi, int64_t n_targets);
int mv_npga_solve_frontier_refined(const mv_problem *P_lo, const mv_problem *P_hi, const double *d_R_targets,
                                   int64_t n_targets, const mv_solve_opts *opts, double eps_lo, double *d_X,
                                   mv_solve_info *h_infos, void *d_ws, size_t ws_bytes, mv_stream_t stream);

/* ------------------------------------------------------------------------
 * 3g. Batch of independent problems of uneven size (n_i, T_i all different).
 *
 *  Solves count problems (same dtype; each with its own L, n, T, ld, layout,
 *  gamma, mu, R_target, mode and power start) with the semantics of
 *  mv_npga_solve, in lock-step.  Problems stored transposed (MV_LAYOUT_TN,
 *  L^T as T x n) take the fused single pass of mv_gradient, grouped: one
 *  launch per cluster size (1, 2, 4 or 8 CTAs, the smallest whose asset
 *  share fits shared memory) over a list of (problem, cluster) pairs, each
 *  problem with about 8 MB of L per cluster, its own tensor map and its own
 *  fixed-order reduction -- L is read once per product.  Problems stored
 *  n x T (MV_LAYOUT_NT) take two grouped GEMV launches per product over a
 *  tile list that spans their grids (row splits of 512 rows).  The two kinds
 *  may share a batch.  Each projection step is one launch with one
 *  thread-block cluster per problem.  Each problem has its own step size,
 *  FISTA state and KKT test; a converged problem's clusters and tiles
 *  return at once.  Chunks of kkt_every iterations replay as one CUDA graph.
 *  MV_ERR_UNSUPPORTED for MV_LAYOUT_SIGMA problems, and for a transposed
 *  problem whose n fits no cluster size (n above 24576).
 *  MV_ERR_TIMEOUT if a bounded wait of the fused pass gave up.
 *  h_x_dev [in]  host array of count device pointers; x_i (n_i FP64) is
 *                written to h_x_dev[i] on return.
 *  h_infos [out] count host mv_solve_info.
 *  Workspace: mv_batch_workspace_size(probs, count).  Returns the first
 *  non-OK per-problem status (or MV_OK).  Blocking.
 * ------------------------------------------------------------------------ */
/*  The grouped GEMVs' tiles (rows per split of the column-sum kernel, bytes of L
 *  per row per split of the row-dot kernel) are tuned on the batch itself: the
 *  first solve of a batch shape times nine candidates (256/512/1024 rows x
 *  8/16/32 KB) on one pass each and keeps the fastest for that shape
 *  (environment MV_BATCH_AUTOTUNE=0 keeps 512 rows x 16 KB).  The workspace
 *  has room for every candidate.  mv_batch_tiles reports the tiles a shape
 *  runs with: MV_OK once tuned, MV_ERR_NOT_CONVERGED (and the defaults)
 *  before.  A batch of transposed problems only has nothing to tune and
 *  keeps the defaults. */
int mv_batch_tiles(const mv_problem *probs, int64_t count, int32_t *h_t_rows, int32_t *h_n_split_bytes);
size_t mv_batch_workspace_size(const mv_problem *probs, int64_t count);
int mv_npga_solve_batch(const mv_problem *probs, int64_t count, const mv_solve_opts *opts,
                        double *const *h_x_dev, mv_solve_info *h_infos, void *d_ws, size_t ws_bytes,
                        mv_stream_t stream);

/* ------------------------------------------------------------------------
 * 3c. Sketch (Sec. 2.3; STR step 1 of Sec. 2.5):  tilde L = L Phi.
 *
 *  A BF16 x BF16 -> FP32 GEMM on the tcgen05 tensor cores (accumulator in
 *  tensor memory, operands staged by TMA with the 128-byte swizzle).
 *  d_L      [in]  n x T BF16, row-major, leading dim ldL (ldL*2 % 16 == 0).
 *  d_Phi_t  [in]  m x T BF16 = Phi transposed: row j holds sketch column j
 *                 (entries N(0, 1/m) for the Gaussian JL sketch), ldP*2 % 16 == 0.
 *  d_L_sketch [out] n x m FP32, row-major, leading dim ldS >= m.
 *  All pointers 16-byte aligned.  Blocking: returns MV_ERR_TIMEOUT if a
 *  pipeline wait exceeded its 2 s bound (no hang), MV_ERR_CUDA if the tensor
 *  map could not be encoded.
 * ------------------------------------------------------------------------ */
int mv_sketch(const void *d_L, int64_t n, int64_t T, int64_t ldL, const void *d_Phi_t, int64_t m,
              int64_t ldP, float *d_L_sketch, int64_t ldS, mv_stream_t stream);

/*  The same for a factor stored in any mv_dtype (MV_LAYOUT_NT, n x T, leading
 *  dim ldL >= T):
 *    MV_BF16      as mv_sketch (no workspace);
 *    MV_F32       L = H + D split into two BF16 parts in the workspace; both
 *                 are multiplied against each staged Phi tile into one
 *                 accumulator, so the only rounding of L is that of H + D
 *                 (below 2^-18 |L_it| per term);
 *    MV_FP8_E4M3  the stored values are expanded exactly to BF16 in the
 *                 workspace and row i of the result is scaled by
 *                 d_row_scale[i].
 *  Workspace: mv_sketch_workspace_size(dtype, n, T) bytes, 256-byte aligned
 *  (0 for BF16).  Blocking. */
size_t mv_sketch_workspace_size(int32_t dtype, int64_t n, int64_t T);
int mv_sketch_dtype(const void *d_L, int32_t dtype, const float *d_row_scale, int64_t n, int64_t T, int64_t ldL,
                    const void *d_Phi_t, int64_t m, int64_t ldP, float *d_L_sketch, int64_t ldS,
                    void *d_ws, size_t ws_bytes, mv_stream_t stream);

/*  Seeded draws of the sketch maps of Sec. 2.3, made on the device.  The
 *  generator is Philox4x32-10 (Salmon et al., SC'11), counter-based, with the
 *  key (seed mod 2^32, seed div 2^32):
 *  mv_gaussian_sketch writes Phi^T (m x T BF16, leading dim ldP >= T, ldP a
 *    multiple of 8, columns T..ldP-1 zero): entry (j, t) is the Box--Muller
 *    normal of the Philox block at counter (t div 4, j, 0, 0) -- words w_0..w_3
 *    give u = ((w_a >> 8) + 1) 2^-24 (a = 0, 2) and v = (w_b >> 8) 2^-24
 *    (b = 1, 3); r = sqrt(-2 ln u); (r cos 2 pi v, r sin 2 pi v) for (u_0, v_1)
 *    and (u_2, v_3) are the normals for t mod 4 = 0, 1, 2, 3 -- times
 *    1/sqrt(m), computed in FP32 and rounded to BF16.
 *  mv_countsketch_draw writes the CountSketch hash and signs (T entries
 *    each) from the block at counter (t, 0, 1, 0): h(t) = (w_0 m) >> 32 and
 *    s_t = 1 - 2 (w_1 & 1); they feed mv_countsketch unchanged.
 *  Asynchronous; deterministic for a given seed. */
int mv_gaussian_sketch(uint64_t seed, int64_t m, int64_t T, void *d_Phi_t, int64_t ldP, mv_stream_t stream);
int mv_countsketch_draw(uint64_t seed, int64_t T, int64_t m, int32_t *d_hash, int8_t *d_sign, mv_stream_t stream);

/* ------------------------------------------------------------------------
 * 4b. CountSketch (Sec. 2.3, construction (2)): the sparse alternative to
 *     the Gaussian sketch.  Phi (T x m) has one nonzero per row,
 *     Phi(t, h(t)) = s_t in {-1, +1}, so column j of tilde L = L Phi is the
 *     signed sum of the columns t of L with h(t) = j.  O(nT) work, no GEMM:
 *     L is read once (HBM-bound).
 *
 *  d_L        [in]  the factor, dtype F32 / BF16 / FP8 e4m3 (with d_row_scale),
 *                   MV_LAYOUT_TN (L^T, T x n, ldL >= n) or MV_LAYOUT_NT
 *                   (n x T, ldL >= T; T x element size at most 200 KB).
 *  d_hash     [in]  T int32 buckets h(t) in [0, m) (device).
 *  d_sign     [in]  T int8 signs s_t, -1 or +1 (device; any negative value is -1).
 *  d_L_sketch [out] n x m FP32, row-major, leading dim ldS >= m.
 *  d_ws       [in]  mv_countsketch_workspace_size(T, m) bytes, 256-byte aligned.
 *  Each output is summed over its bucket's periods in ascending order
 *  (deterministic).  Blocking.  MV_ERR_INVALID_ARG for a bucket outside
 *  [0, m); MV_ERR_UNSUPPORTED for a bucket of more than 4096 periods or an
 *  NT row that does not fit shared memory.  The result feeds
 *  mv_str_truncate unchanged.
 * ------------------------------------------------------------------------ */
size_t mv_countsketch_workspace_size(int64_t T, int64_t m);
int mv_countsketch(const void *d_L, int32_t dtype, int32_t layout, const float *d_row_scale, int64_t n,
                   int64_t T, int64_t ldL, const int32_t *d_hash, const int8_t *d_sign, int64_t m,
                   float *d_L_sketch, int64_t ldS, void *d_ws, size_t ws_bytes, mv_stream_t stream);

/* ------------------------------------------------------------------------
 * 3d. Truncate + ridge (Sec. 2.5 steps 2-3; App. D.3).
 *
 *  From tilde L (n x m FP32) computes the k largest eigenpairs of the Gram
 *  matrix K = tilde L tilde L^T (eigenvalues sigma_i^2, eigenvectors U) and
 *  writes L_eff = U_k diag(sigma_k) (n x k FP32, row-major, columns in
 *  descending sigma) and sigma (k FP64, descending).  The ridge returned in
 *  *h_gamma_out is `gamma` if gamma >= 0, else 1e-4 * trace_sigma / n.
 *  Method (the partial decomposition the paper's complexity discussion of
 *  STR points to): K formed FP32-accurate on the tensor cores (three-piece
 *  BF16 splits, chunked accumulation), then Chebyshev-filtered subspace
 *  iteration on a block of b = max(2k, k + 512) columns (rounded up to 64)
 *  with Lowdin orthonormalisation, and a final Rayleigh--Ritz step whose
 *  b x b eigenproblem is solved in FP64.  For n <= 1024, or b >= n, all n
 *  eigenpairs of K come from a dense FP64 eigensolver instead.  The small
 *  eigenproblems use cuSOLVER (DSYEVD / SSYEVD) loaded at run time:
 *  MV_ERR_UNSUPPORTED if it cannot be loaded.  Accuracy: eigenvalues within
 *  about 1e-6 sigma_1^2 of those of the exact K of the given tilde L, and
 *  L_eff^T L_eff = diag(sigma^2) to FP32 rounding.  Workspace:
 *  mv_str_workspace_size(n, m, k) bytes (K, the n x b panels and the
 *  eigensolver's buffer).  Blocking; the first call on a device also
 *  captures the orthonormalisation into a CUDA graph that later calls of the
 *  same shape and workspace replay.  MV_ERR_NUMERIC if the eigensolver
 *  reports a failure or the iteration produces a non-finite value.
 * ------------------------------------------------------------------------ */
size_t mv_str_workspace_size(int64_t n, int64_t m, int64_t k);
int mv_str_truncate(const float *d_L_sketch, int64_t n, int64_t m, int64_t ldS, int64_t k, double gamma,
                    double trace_sigma, float *d_L_eff, int64_t ldE, double *d_sigma, double *h_gamma_out,
                    void *d_ws, size_t ws_bytes, mv_stream_t stream);

/*  mv_str_truncate with the data-driven choices of App. D: the rank is the
 *  knee of the sketched spectrum lam_i = sigma_i^2(tilde L) (nonincreasing),
 *      l = max{ i : lam_i / lam_1 >= tau  and  lam_{i+1} / lam_i <= rho }
 *  (App. D.1; tau in (0, 1] the minimum relative signal level, rho in (0, 1)
 *  the knee ratio), capped at k_max; and, if kappa_target > 1, the ridge
 *      gamma = lam_1 / (kappa_target - 1)
 *  so that the STR covariance has condition number kappa_target (App. D.2);
 *  otherwise gamma as in mv_str_truncate.  L_eff has k_max columns of which
 *  the first l are U_l diag(sigma_l) and the rest zero (sigma likewise).
 *  *h_k_out = l.  MV_ERR_NUMERIC if no i satisfies the rule.  Workspace:
 *  mv_str_workspace_size(n, m, k_max).  Blocking. */
int mv_str_truncate_knee(const float *d_L_sketch, int64_t n, int64_t m, int64_t ldS, double tau, double rho,
                         int64_t k_max, double kappa_target, double gamma, double trace_sigma, float *d_L_eff,
                         int64_t ldE, double *d_sigma, int64_t *h_k_out, double *h_gamma_out, void *d_ws,
                         size_t ws_bytes, mv_stream_t stream);

/* ------------------------------------------------------------------------
 * 3h. The whole STR build of Sec. 2.5 from a seed: (1) Phi drawn on the
 *     device by mv_gaussian_sketch(seed, m, T) (Gaussian JL, N(0, 1/m)),
 *     (2) tilde L = L Phi by mv_sketch_dtype, (3) truncation to rank k and
 *     the ridge by mv_str_truncate.
 *
 *  d_L          [in]  the factor, dtype F32 / BF16 / FP8 e4m3 (d_row_scale
 *                     then holds the n row scales), n x T, leading dim ldL.
 *  d_L_sketch   [out] n x m FP32 (leading dim ldS >= m), or NULL: tilde L is
 *                     then kept in the workspace only.
 *  d_L_eff, ldE, d_sigma, h_gamma_out: as mv_str_truncate.
 *  Workspace: mv_sketch_str_workspace_size(dtype, n, T, m, k, own_sketch)
 *  bytes, own_sketch = 1 when d_L_sketch is NULL.  The sketch stage (Phi^T,
 *  m T BF16, and the BF16 copy of L) and the truncation reuse the same bytes.
 *  Blocking.
 * ------------------------------------------------------------------------ */
size_t mv_sketch_str_workspace_size(int32_t dtype, int64_t n, int64_t T, int64_t m, int64_t k, int32_t own_sketch);
int mv_sketch_str(const void *d_L, int32_t dtype, const float *d_row_scale, int64_t n, int64_t T, int64_t ldL,
                  int64_t m, uint64_t seed, int64_t k, double gamma, double trace_sigma, float *d_L_sketch,
                  int64_t ldS, float *d_L_eff, int64_t ldE, double *d_sigma, double *h_gamma_out, void *d_ws,
                  size_t ws_bytes, mv_stream_t stream);

/* ------------------------------------------------------------------------
 * 3f. Adjoint of the unrolled solve (an extension; the paper does not
 *     differentiate its solver).
 *
 *  The forward is Algorithm 1 unrolled for exactly K = opts->max_iter
 *  iterations (no early stop; mv_npga_solve with the same opts and eps = 0,
 *  kkt_every = 0 gives the same x_K) from x^0 = d_x0 (NULL: Pi_F(1/n 1)),
 *  with alpha from opts (power method or override).  alpha, x^0 and
 *  R_target are treated as constants.  Given d loss / d x_K, the call returns
 *      d_dmu [out] n FP64  d loss / d mu  (through the projection's return row)
 *      d_dL  [out] n x ldD FP32  d loss / d L  (overwritten)
 *  Reverse sweep: the forward is recomputed segment by segment from
 *  checkpoints taken every opts->checkpoint_every iterations; each backward
 *  step applies the projection's Jacobian on the active set
 *  (P = I - C (C^T C)^{-1} C^T on the support, C = [1, mu] or [1]) and the
 *  transposed products (one pass over L each); dL accumulates
 *  -2 alpha (v_bar z_k^T + y_k (L^T v_bar)^T) per segment as one tcgen05
 *  GEMM whose FP32 operands are split into three BF16 pieces (six piece
 *  products, FP32-accurate), added into d_dL in place.  d_dL 16-byte
 *  aligned with ldD a multiple of 4 for the vector path (any other pitch is
 *  handled element by element).  FP32 factor only.  Blocking.
 * ------------------------------------------------------------------------ */
size_t mv_backward_workspace_size(const mv_problem *P, const mv_solve_opts *opts);
int mv_npga_backward(const mv_problem *P, const mv_solve_opts *opts, const double *d_x0,
                     const double *d_dloss_dx, double *d_dmu, float *d_dL, int64_t ldD,
                     mv_solve_info *h_info, void *d_ws, size_t ws_bytes, mv_stream_t stream);

/* ------------------------------------------------------------------------
 * 4. Gradient building block (Eq. npga-unified-grad), exposed for tests and
 *    for callers with their own outer loop:
 *        d_g = 2 L_eff (L_eff^T y) + 2 gamma y,   d_z = L_eff^T y.
 *  d_y FP64 n, d_z FP32 T (may be NULL), d_g FP64 n.  Uses the workspace of
 *  mv_npga_workspace_size.  With d_z NULL the product runs as the fused
 *  single pass described under mv_npga_solve where that applies.
 *  Asynchronous.
 * ------------------------------------------------------------------------ */
int mv_gradient(const mv_problem *P, const double *d_y, float *d_z, double *d_g,
                void *d_ws, size_t ws_bytes, mv_stream_t stream);

/* ------------------------------------------------------------------------
 * 5. Allocation-free gradient.  The paper has no counterpart: this is a
 *    service for callers that cannot allocate device memory -- code that is
 *    handed only pre-allocated input and output buffers by a host framework
 *    that owns the device memory pool (plug-ins, user-defined functions), or
 *    a latency-bound loop that cannot absorb the device-wide synchronisation
 *    cudaMalloc implies.
 *
 *  Same inputs, outputs and result as mv_gradient, but no workspace
 *  argument: the scratch lives in one file-scope device array of
 *  MV_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads
 *  the library keeps until the process exits.  The call allocates nothing
 *  (no cudaMalloc, cudaFree or allocating library routine).
 *  - Limit: the call always runs the two-pass GEMV product (never the fused
 *    single pass), and its scratch is that path's: the vectors plus the
 *    partial sums of the row splits, whose count follows the device's SM
 *    count.  mv_gradient_noalloc_scratch_size(P) returns that figure for
 *    the current device (0 for an invalid problem); problems for which it
 *    exceeds MV_NOALLOC_SCRATCH_BYTES are rejected on the host with
 *    MV_ERR_UNSUPPORTED before anything is launched, and mv_last_error()
 *    then states the bytes needed.  On a 152-SM GB300 the 5440 x 48374 FP32
 *    problem needs about 8 MiB in either layout.
 *  - Device address: the array's host-side name is not a device address, so
 *    the call looks the address up with the device current.  The first call
 *    on a device does this set-up; make it before any stream capture.
 *    Later calls made outside stream capture repeat the look-up, so they
 *    stay right across a device reset (which reloads the library's module
 *    at a new address).
 *  - Every call on a device shares the one array and leaves its contents
 *    behind; the call clears what must start at zero.  Calls whose work
 *    overlaps on the GPU (different streams, or different host threads)
 *    race on the array and must be serialised by the caller.
 *  Asynchronous.
 * ------------------------------------------------------------------------ */
#define MV_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)

size_t mv_gradient_noalloc_scratch_size(const mv_problem *P);
int mv_gradient_noalloc(const mv_problem *P, const double *d_y, float *d_z, double *d_g,
                        mv_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* MV_H */
