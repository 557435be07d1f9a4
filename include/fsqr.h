/*
 * fsqr.h - C ABI of the GB300 FS-QRPPA library: weighted-l1 penalised
 * quantile regression for p >> n by the feature-splitting proximal point
 * algorithm (FS-QRPPA) of "Scalable Ultra-High-Dimensional Quantile
 * Regression with Genomic Applications" (arXiv 2601.02826).
 *
 * Problem (Section 1, eq. vanilla_QR with eq. weight_l1_penalty):
 *
 *   min_beta (1/n) sum_i rho_tau(y_i - x~_i^T beta) + sum_{j>=1} lambda_j |beta_j|,
 *   rho_tau(u) = (tau - 1{u<0}) u,  lambda_j = lambda * omega_j,  omega_0 = 0.
 *
 * x~_i is row i of the standardised design X~ = [1 | C~ | G~]: column 0 is
 * the intercept, columns 1..c are dense covariates, columns c+1..c+p the
 * stored feature (genotype) columns. Every column but the intercept is
 * standardised on the fly when design.standardize = 1 (Section 7: mean and
 * population sd over non-missing entries; a missing genotype is imputed by
 * the column mean, i.e. standardised value 0; a constant column is all 0).
 * All coefficient vectors below (beta, omega) index these P = 1 + c + p
 * columns and are on the standardised scale unless stated otherwise.
 *
 * Iteration (Section 4, eq. fsppa_update, Algorithm 1) over a partition of
 * the P columns into G contiguous blocks (eq. decompose_x):
 *   beta_g <- soft-threshold (eq. beta_update) with step 1/eta_g,
 *   z      <- pinball prox (eq. z_update) with parameter mu,
 *   theta  <- theta - mu/(G+1) (2 r^{k+1} - r^k),  r = X~ beta + z - y.
 *
 * Stopping test (the paper defers it to an appendix that is not part of the
 * text; this library's reading): every check_every iterations, on the
 * current iterate, KKT = max(R_p, R_z, R_b, R_1) <= tol with
 *   R_p = ||y - X~ beta - z||_inf / (1 + ||y||_inf)
 *   R_z = max_i dist(n theta_i, d rho_tau(z_i))
 *   R_b = max_{j>=1} dist((X~^T theta)_j, lambda_j d|beta_j|) / lambda_norm
 *   R_1 = |sum_i theta_i|
 * where lambda_norm = lambda_max(tau) (1 if that is 0).
 *
 * Conventions for every entry point:
 *   - Device pointers are caller-owned CUDA global memory on the context's
 *     device; the library never frees them. Host pointers are named so.
 *   - Every call is ordered on the context's stream and returns after that
 *     stream has finished the call's work (synchronous), unless stated.
 *   - Return value: FSQR_OK (0) or an FSQR_E* code; fsqr_last_error() then
 *     holds a one-line message. On FSQR_EINVAL nothing was launched.
 *   - Not thread-safe per context; distinct contexts are independent.
 */
#ifndef FSQR_H
#define FSQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FSQR_OK 0
#define FSQR_EINVAL 1   /* invalid argument (nothing launched) */
#define FSQR_ENOCONV 2  /* max_iter reached before KKT <= tol; outputs valid */
#define FSQR_ETIMEOUT 3 /* wall-clock budget (opts.timeout_ms) exhausted; outputs valid */
#define FSQR_ENUMERIC 4 /* NaN/Inf in inputs or iterates */
#define FSQR_ECUDA 5    /* a CUDA call failed; message has the CUDA error */
#define FSQR_ENOMEM 6   /* device workspace allocation failed */

/* ---- storage formats of the p feature columns (SNP-major) -------------- */
#define FSQR_DENSE_F64 0 /* n doubles per column */
#define FSQR_INT8 1      /* 1 byte per sample: 0/1/2, any other value = missing */
#define FSQR_2BIT 2      /* 4 samples per byte, sample i in bits 2*(i%4) of byte i/4;
                            codes 0/1/2, code 3 = missing */

/* ---- arithmetic of the inner products ----------------------------------- */
#define FSQR_FP64 0       /* plain FP64 for every product and reduction */
#define FSQR_MIXED 1      /* exact integer products, FP64 state and reductions:
                             X~^T theta on the tensor cores with theta split
                             into base-16 digits (E4M3) against the genotype
                             codes read as E4M3, FP32 accumulation that stays
                             exact; X~ beta likewise from base-16 digits of
                             a_j beta_j over the active columns, int64 sums.
                             int8 or 2-bit storage; tensor cores with <= 63
                             covariates and n, p <= 2^20 (where the digit sums
                             stay exact; the X~ beta pass also needs fewer than
                             2^19 active columns and fails with FSQR_ECUDA
                             beyond), else for int8 the kernels of
                             FSQR_MIXED_SIMT and for 2-bit FSQR_EINVAL. */
#define FSQR_MIXED_SIMT 2 /* as FSQR_MIXED, with X~^T theta from int8 digits of
                             theta by DP4A on the SIMT cores instead */

/* ---- starting point ------------------------------------------------------ */
#define FSQR_WARM_NONE 0  /* beta = 0, z = y, theta = 0 */
#define FSQR_WARM_GIVEN 1 /* beta, z, theta arrays are read as the start */
#define FSQR_WARM_PATH 2  /* fsqr_fit_batch only: along each tau's lambda path,
                             fit l starts from fit l-1's solution (Section 7) */
#define FSQR_WARM_LEARNED 3 /* every fit starts from the learned warm start of the
                               network opts.warm_params (fsqr_warm_start at
                               lambda / lambda_max(tau)); beta, z, theta are
                               overwritten by that start, then by the fit */

typedef struct fsqr_ctx fsqr_ctx;

/* Design matrix X = [1 | C | G]; see the column conventions above. */
typedef struct {
  int64_t n;              /* samples, >= 1 */
  int64_t p;              /* stored feature columns, >= 0 */
  int64_t c;              /* dense covariate columns, >= 0 */
  int32_t geno_format;    /* FSQR_DENSE_F64 | FSQR_INT8 | FSQR_2BIT */
  int32_t standardize;    /* 1: standardise covariates and features on the fly; 0: raw */
  const void *geno;       /* device; column j (0-based) at geno + j*geno_ld bytes;
                             16-byte aligned; NULL allowed when p == 0 */
  int64_t geno_ld;        /* bytes per column: multiple of 16, >= bytes for n samples */
  const double *cov;      /* device; covariate k at cov + k*n; NULL allowed when c == 0 */
  const double *col_mean; /* device, length c+p, or NULL: computed (one pass over X) */
  const double *col_sd;   /* device, length c+p, or NULL: computed with col_mean */
} fsqr_design;

typedef struct {
  double tol;             /* KKT tolerance; default 1e-6 */
  int32_t max_iter;       /* default 100000; the run stops at the first stop test
                             (multiple of check_every) at or after max_iter */
  int32_t check_every;    /* K: stop test every K iterations; default 10 */
  double mu;              /* > 0, or <= 0 for the default 1/(n sd(y)) */
  const double *eta;      /* host, length G, each > 0; or NULL: power method */
  double eta_margin;      /* eta_g = (1+margin) mu Lambda_hat_g; default 0.05 */
  int32_t power_iters;    /* power-method steps cap; default 100 */
  double power_tol;       /* power-method relative change stop; default 1e-6 */
  int32_t precision;      /* FSQR_FP64 | FSQR_MIXED; default FSQR_FP64 */
  int32_t warm;           /* FSQR_WARM_*; default FSQR_WARM_NONE */
  int32_t digits;         /* FSQR_MIXED_SIMT: int8 (7-bit) digits per theta entry, 3..5;
                             FSQR_MIXED uses 7 base-16 digits (6 when digits == 3);
                             default 4 */
  int32_t max_group;      /* fits advanced together per X pass, 1..32, or 0: chosen by
                             timing the candidates 1, 2, 3, 4, min(B, 8) and, on the
                             tensor-core path with B > 8 fits, 16 and 32 on the first
                             fits (a short cold run of each, cached per context, problem
                             shape and block partition; fsqr_profile.tuned_group reports
                             it); default 4. Above 8, on the tensor-core path only
                             (FSQR_MIXED, int8 storage), the fits of fsqr_fit_batch stream
                             through 16 (max_group <= 16) or 32 slots of one solve: a
                             slot whose fit has stopped takes the next fit (with
                             FSQR_WARM_PATH, the next fit of a tau's path starts from
                             its predecessor's solution as soon as that one stops).
                             Elsewhere values above 8 act as 8. */
  int64_t timeout_ms;     /* > 0: stop with FSQR_ETIMEOUT after this wall time */
  const float *warm_params; /* device, fsqr_mlp_param_count() floats: the network of
                               FSQR_WARM_LEARNED; default NULL */
  double ridge;           /* gamma >= 0: weighted elastic net (Section 5, closing remark),
                             Omega(beta) = sum_j lambda_j |beta_j| + (gamma/2) sum_j omega_j beta_j^2;
                             the beta step divides the soft threshold by eta_g + gamma omega_j,
                             R_b measures dist(s_j - gamma omega_j beta_j, lambda_j d|beta_j|),
                             info.primal includes the quadratic term and info.gap is NaN
                             when gamma > 0; default 0 (the weighted-l1 penalty) */
  int32_t screen;         /* 1 (fsqr_fit_batch with FSQR_WARM_PATH, at most 32 taus): the
                             sequential strong rule along each tau's path. At stage l a stored
                             column j is left out of the stage's fits when, for every tau,
                             beta_j = 0 at lambda_{l-1} and |x~_j^T theta| < omega_j (2 lambda_l -
                             lambda_{l-1}) there (at l = 0 the lambda_max direction, with
                             lambda_{-1} = lambda_max); the fits run on the kept columns only, and
                             every left-out column is then checked on the full design: one with
                             (|x~_j^T theta| - lambda_j)_+ / lambda_max > tol is put back and the
                             stage re-solved, so returned fits meet the stop test on all columns.
                             fsqr_profile.screen_kept/screen_total count the columns streamed.
                             default 0 */
} fsqr_opts;

/* Per-fit report. */
typedef struct {
  int32_t status;         /* FSQR_OK, FSQR_ENOCONV, FSQR_ETIMEOUT or FSQR_ENUMERIC */
  int32_t iters;          /* iteration k of the returned iterate w^k */
  double kkt, r_p, r_z, r_beta, r_1; /* stop-test residuals of the returned iterate */
  double primal;          /* (1/n) sum rho_tau(y - X~ beta) + sum lambda_j |beta_j| */
  double dual, gap;       /* dual value and relative gap (P-D)/(1+|P|+|D|);
                             NaN when some omega_j = 0 for j >= 1 */
  double lambda, lambda_max, mu;
  int64_t active;         /* number of j >= 1 with beta_j != 0 */
  double t_setup_ms, t_solve_ms;
} fsqr_info;

/* Version of this ABI (major*10000 + minor*100 + patch). */
int fsqr_version(void);

/* Fills opts with the defaults listed above. */
void fsqr_opts_default(fsqr_opts *opts);

/* Creates a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). The context owns its
 * device workspace, grown on demand and released by fsqr_destroy. */
int fsqr_create(fsqr_ctx **ctx, int device, void *cuda_stream);
int fsqr_destroy(fsqr_ctx *ctx);
/* Last error message of this context ("" if none); valid until the next call. */
const char *fsqr_last_error(const fsqr_ctx *ctx);

/* Column statistics (Section 7, standardisation of the features): mean and
 * population sd over non-missing entries of the c covariates and p feature
 * columns. mean_out/sd_out: device, length c+p. */
int fsqr_col_stats(fsqr_ctx *ctx, const fsqr_design *X, double *mean_out, double *sd_out);

/* lambda_max(tau) = max_{j>=1, omega_j>0} |x~_j^T v| / (n omega_j) with
 * v_i = tau - 1{y_i < y_(ceil(n tau))}: the smallest lambda at which
 * beta_{1..} = 0 is optimal up to ties (penalty path, Section 7).
 * y, omega: device (omega length P). out: host scalar.
 * For int8 and 2-bit storage x~_j^T v is an exact integer sum of the codes
 * with v rounded once to 52-bit fixed point (the accuracy of FP64
 * arithmetic); dense storage computes it in FP64. The same holds for the
 * power method of fsqr_eta. */
int fsqr_lambda_max(fsqr_ctx *ctx, const fsqr_design *X, const double *y, double tau,
                    const double *omega, double *out);

/* Step metric (Section 4): eta_g = (1+margin) mu Lambda_hat(X~_g^T X~_g), with
 * Lambda_hat from the power method started at v = 1/sqrt(p_g) and stopped
 * after max_iter steps or a relative change <= tol; a zero block gets
 * (1+margin) mu. block_ptr: host, G+1 offsets, 0 = block_ptr[0] < ... <
 * block_ptr[G] = P. eta_out: host, length G. */
int fsqr_eta(fsqr_ctx *ctx, const fsqr_design *X, const int64_t *block_ptr, int G, double mu,
             double margin, int max_iter, double tol, double *eta_out);

/* One FS-QRPPA fit (Algorithm 1) at quantile tau in (0,1) and penalty
 * lambda >= 0, lambda_j = lambda omega_j.
 *   y: device, length n. omega: device, length P, omega[0] == 0, omega >= 0.
 *   block_ptr: host, G+1 offsets as for fsqr_eta.
 *   beta (P), z (n), theta (n): device, in/out. Read as the start when
 *   opts.warm == FSQR_WARM_GIVEN; on return they hold the iterate that
 *   passed the stop test (or the last one), beta on the standardised scale.
 *   info: host, may be NULL.
 * Returns FSQR_OK, or FSQR_ENOCONV / FSQR_ETIMEOUT with valid outputs. */
int fsqr_fit(fsqr_ctx *ctx, const fsqr_design *X, const double *y, double tau, double lambda,
             const double *omega, const int64_t *block_ptr, int G, const fsqr_opts *opts,
             double *beta, double *z, double *theta, fsqr_info *info);

/* A tau x lambda grid of fits sharing X, y, omega, the blocks and eta.
 *   taus: host, n_tau values in (0,1). lambdas: host, n_tau*n_lambda values,
 *   lambdas[t*n_lambda + l] for tau t (each tau has its own path).
 *   Fit b = t*n_lambda + l. beta: device, B*P (fit b at beta + b*P);
 *   z, theta: device, B*n. infos: host, B entries, may be NULL.
 * With opts.warm == FSQR_WARM_PATH the lambdas of each tau should decrease;
 * fit (t, l) starts from fit (t, l-1). Returns FSQR_OK if every fit met the
 * tolerance, else the first non-OK per-fit status. */
int fsqr_fit_batch(fsqr_ctx *ctx, const fsqr_design *X, const double *y, int n_tau,
                   const double *taus, int n_lambda, const double *lambdas, const double *omega,
                   const int64_t *block_ptr, int G, const fsqr_opts *opts, double *beta,
                   double *z, double *theta, fsqr_info *infos);

/* ---- folded-concave penalties (Section 6, Algorithm 2) ------------------ */
#define FSQR_PEN_SCAD 1 /* p' of eq. scad: lambda (t <= lambda), (a lambda - t)/(a - 1)
                           (lambda < t < a lambda), 0 (t >= a lambda); a > 2 */
#define FSQR_PEN_MCP 2  /* p' of eq. mcp: lambda - t/a (t <= a lambda), 0 beyond; a > 1 */

/* L-step local linear approximation (LLA) for SCAD or MCP (Algorithm 2):
 * the weighted-l1 fit at lambda_j = lambda omega_j (as fsqr_fit), then L
 * fits with lambda_j = omega_j p'_lambda(|beta~_j|) from the previous fit's
 * beta~ (standardised scale), each started from the previous (beta, z,
 * theta) with the same eta_g. The paper uses L = 1, a = 3.7 (SCAD), a = 3
 * (MCP). R_b of every step is divided by lambda_max(tau) of omega.
 *   lambda > 0; omega as for fsqr_fit (its zeros stay unpenalised).
 *   beta, z, theta: device, in/out as for fsqr_fit (opts.warm applies to
 *   the first fit); on return the last step's iterate.
 *   lam_out: device, length P, or NULL: the last step's lambda_j.
 *   info: the last step's report, with iters = the steps of all L + 1 fits.
 * Returns the last fit's status (FSQR_OK, FSQR_ENOCONV, FSQR_ETIMEOUT). */
int fsqr_fit_lla(fsqr_ctx *ctx, const fsqr_design *X, const double *y, double tau, double lambda,
                 const double *omega, const int64_t *block_ptr, int G, int penalty, double a, int L,
                 const fsqr_opts *opts, double *beta, double *z, double *theta, double *lam_out,
                 fsqr_info *info);

/* fsqr_fit_batch from HOST buffers: X->geno, X->cov, X->col_mean/col_sd, y,
 * omega, beta, z, theta are host pointers. The library copies the inputs to
 * device workspace, solves, and copies beta/z/theta back; the copies are
 * part of the call. */
int fsqr_fit_batch_host(fsqr_ctx *ctx, const fsqr_design *X, const double *y, int n_tau,
                        const double *taus, int n_lambda, const double *lambdas,
                        const double *omega, const int64_t *block_ptr, int G,
                        const fsqr_opts *opts, double *beta, double *z, double *theta,
                        fsqr_info *infos);

/* Stop-test residuals, primal value and duality gap of a given iterate
 * (the saddle-point conditions of Proposition 1 and the dual of the
 * penalised problem). y, omega, beta (P), z, theta (n): device.
 * lambda_norm > 0 divides R_b. out: host. */
int fsqr_kkt(fsqr_ctx *ctx, const fsqr_design *X, const double *y, double tau, double lambda,
             const double *omega, double lambda_norm, const double *beta, const double *z,
             const double *theta, fsqr_info *out);

/* Quantile predictions q_tau(x) = x~^T beta (Section 7.1) for B coefficient
 * vectors: out[b*n + i] = x~_i^T beta_b with beta_b at beta + b*P (device,
 * standardised scale). For new samples pass the training col_mean/col_sd
 * in X so that they are standardised the same way. out: device, B*n. */
int fsqr_predict(fsqr_ctx *ctx, const fsqr_design *X, const double *beta, int B, double *out);

/* Model selection along a lambda path (Section 7). For B fits (beta: device,
 * B*P, standardised scale; taus: host, B quantile levels) evaluated on the
 * design X with response y (device, n): the training data for HBIC, or a
 * validation set (its col_mean/col_sd set to the training ones) for the
 * validation loss. Host outputs of B entries, each may be NULL:
 *   loss[b]   = (1/n) sum_i rho_tau_b(y_i - x~_i^T beta_b)
 *   active[b] = #{j >= 1 : beta_b,j != 0}
 *   hbic[b]   = log(sum_i rho_tau_b(y_i - x~_i^T beta_b))
 *               + active[b] (log log n / n) log(P - 1)   (C_n = log p)
 * The paper picks the lambda of least HBIC in sparse settings and of least
 * validation loss in dense ones. */
int fsqr_path_stats(fsqr_ctx *ctx, const fsqr_design *X, const double *y, int B, const double *taus,
                    const double *beta, double *loss, int64_t *active, double *hbic);

/* Prediction intervals [q_lo(x), q_hi(x)] = [x~^T beta_lo, x~^T beta_hi]
 * (Section 7.1, e.g. the fits at tau = 0.1 and 0.9) on the samples of X,
 * y (device). Host outputs, each may be NULL: coverage = fraction of samples
 * with q_lo <= y <= q_hi whose interval does not cross (q_lo <= q_hi; a
 * crossing counts as a miss); width = mean of q_hi - q_lo; crossings =
 * number of samples with q_lo > q_hi. */
int fsqr_interval_coverage(fsqr_ctx *ctx, const fsqr_design *X, const double *y, const double *beta_lo,
                           const double *beta_hi, double *coverage, double *width, int64_t *crossings);

/* Maps B standardised coefficient vectors to the original feature scale
 * (Section 7): b_j / sd_j for j >= 1 (0 for a constant column) and
 * b_0 - sum_j mean_j b_j / sd_j. beta_std, beta_out: device, B*P. */
int fsqr_back_transform(fsqr_ctx *ctx, const fsqr_design *X, const double *beta_std, int B,
                        double *beta_out);

/* Kernel timing sampled inside the solver (no counterpart in the paper;
 * used to report the column pass against the memory roofline). When
 * enabled, every replay of the captured iteration graph records CUDA events
 * around one launch of each iteration kernel on the context's stream; the
 * sums and counts accumulate until fsqr_profile_reset. kernel_launches
 * counts every kernel the library launched (graph replays included). */
typedef struct {
  int64_t col_samples;  double col_ms;   /* column pass: X~^T theta + beta prox */
  int64_t xb_samples;   double xb_ms;    /* X~ beta over the active columns; on the
                                            tensor-core path it includes the z, r,
                                            theta update, fused into that pass */
  int64_t vec_samples;  double vec_ms;   /* z, r, theta update (separate kernel only
                                            off the tensor-core path) */
  int64_t iterations;                    /* FS-QRPPA steps executed */
  int64_t kernel_launches;
  int64_t col_bytes;                     /* algorithmic bytes of the last column pass */
  int64_t tuned_group;                   /* group size the autotuner chose last (0: none) */
  int64_t tc_groups;                     /* groups of <= 8 fits solved on the tensor-core passes */
  int64_t simt_groups;                   /* groups solved on the SIMT passes (FP64, FSQR_MIXED_SIMT,
                                            2-bit storage, or sizes beyond the tensor-core bounds) */
  int64_t wide_groups;                   /* wide solves (16 or 32 slots, tensor cores) */
  int64_t screen_kept, screen_total;     /* screened path solves: stored columns kept / all, summed
                                            over stages, rounds and quantiles */
} fsqr_profile;

int fsqr_profile_enable(fsqr_ctx *ctx, int on);

/* Self-test of the device-side failure detection (no counterpart in the
 * paper). Every wait inside the pipelined kernels gives up after a cycle
 * budget (about one second), records a code in a device error word and
 * returns, so that a stalled pipeline ends the call with an error instead of
 * hanging the GPU. This entry point runs that wait in isolation: one CTA
 * waits on a barrier with a budget of budget_cycles (0..4e9); with arrive = 0
 * nothing ever arrives on it, with arrive = 1 its one arrival comes first.
 * wait_ok (host, may be NULL) receives 1 if the wait succeeded. Returns
 * FSQR_ETIMEOUT when the wait ran out (the context stays usable), FSQR_OK
 * when it succeeded. */
int fsqr_wait_selftest(fsqr_ctx *ctx, int64_t budget_cycles, int arrive, int *wait_ok);
int fsqr_profile_get(fsqr_ctx *ctx, fsqr_profile *out);
int fsqr_profile_reset(fsqr_ctx *ctx);

/* ---- learned warm start ------------------------------------------------
 * The paper warm-starts each fit of a lambda path from the previous
 * solution (Section 7). The learned warm start extends that idea; the paper
 * defines no network, so the definitions are this library's:
 *   inputs of feature column j >= 1 of a fit (tau, lambda):
 *     u_j = (tau, lambda / lambda_max(tau), x~_j^T v / (n lambda_max(tau))),
 *     v_i = tau - 1{y_i < y_(ceil(n tau))}  (the direction of fsqr_lambda_max);
 *   network: FSQR_MLP_IN -> 256 -> 256 -> 256 -> 1, ReLU on the hidden
 *     layers, FP32 parameters, flat: W_0 (row-major d_0 x d_1), b_0, W_1,
 *     b_1, W_2, b_2, W_3, b_3 (fsqr_mlp_param_count() floats);
 *   start: beta_0 = y_(ceil(n tau)), beta_j = sd(y) f(u_j),
 *     z = y - X~ beta, theta_i = (tau - 1{z_i < 0}) / n;
 *   training: Adam (b1 0.9, b2 0.999, eps 1e-8, bias-corrected) on
 *     sum_r w_r (f(u_r) - t_r)^2 / sum_r w_r over uniformly drawn batches.
 * Solving from the start (fsqr_fit with FSQR_WARM_GIVEN) reaches the same
 * stop test as a cold start; only the iteration count changes. All arrays
 * are caller-owned device memory; rows x FSQR_MLP_IN inputs are row-major. */
#define FSQR_MLP_IN 3
int64_t fsqr_mlp_param_count(void);
/* He-uniform weights U(-sqrt(6/fan_in), +) from splitmix64(seed + index), zero biases. */
int fsqr_mlp_init(fsqr_ctx *ctx, float *params, uint64_t seed);
/* out[r] = f(x_r), r < rows. */
int fsqr_mlp_forward(fsqr_ctx *ctx, const float *params, const float *x, int64_t rows, float *out);
/* grad (param-count floats) = gradient of the weighted loss over the rows;
 * loss: host, may be NULL. 1 <= rows <= 2^24. */
int fsqr_mlp_grad(fsqr_ctx *ctx, const float *params, const float *x, const float *t, const float *w,
                  int64_t rows, float *grad, double *loss);
/* `steps` Adam steps numbered step0+1 .. step0+steps (m, v: moment arrays
 * of param-count floats, zero before the first step). Step k draws `batch`
 * rows r_i = splitmix64(splitmix64(seed ^ k * 0xD1B54A32D192ED03) + i) mod rows.
 * losses: host, `steps` batch losses, may be NULL. */
int fsqr_mlp_train(fsqr_ctx *ctx, float *params, float *m, float *v, int64_t step0, const float *x,
                   const float *t, const float *w, int64_t rows, int steps, int batch, float lr,
                   uint64_t seed, double *losses);
/* u: device, (P-1) x FSQR_MLP_IN inputs of one fit; lambda_max: host, may be NULL. */
int fsqr_warm_features(fsqr_ctx *ctx, const fsqr_design *X, const double *y, double tau,
                       double lam_frac, const double *omega, float *u, double *lambda_max);
/* The start proposed by the network for (tau, lambda_frac * lambda_max(tau)):
 * beta (P), z (n), theta (n), device. */
int fsqr_warm_start(fsqr_ctx *ctx, const fsqr_design *X, const double *y, double tau,
                    double lam_frac, const double *omega, const float *params, double *beta,
                    double *z, double *theta);

/* ---- lambda_max without device allocation -------------------------------
 * The paper has no counterpart: this entry point is a property of the
 * library, not of the method. It computes exactly what fsqr_lambda_max
 * computes, with the same kernels in the same order, but allocates no device
 * memory. It is for callers that cannot allocate at call time: a serving
 * process whose device memory is reserved up front by its own pool
 * allocator, or one that cannot accept the device-wide synchronisation that
 * cudaMalloc and cudaFree imply.
 *
 * Scratch: one static device array of FSQR_NOALLOC_SCRATCH_BYTES (8 MiB) per
 * device, part of the library image. A call needs about 40*P + 8*pad16(n)
 * bytes of it (P = 1 + c + p; each buffer rounded up to 256 bytes). Larger
 * designs return FSQR_EINVAL, with the byte counts in fsqr_last_error; use
 * fsqr_lambda_max for them. For example, n = 5,000 with P = 100,006 fits.
 * Arguments, result, and the other errors are those of fsqr_lambda_max. The
 * call is synchronous on the context's stream.
 *
 * The first call on a device looks up the array's address
 * (cudaGetSymbolAddress, once per device, with that device current) and may
 * load kernel code. Make that first call before any stream capture begins.
 * Every context on a device shares the array, and it keeps the previous
 * call's contents. Calls that overlap in time on one device race: from
 * several host threads, or from several contexts or streams. They then
 * return wrong results. Serialise such calls. */
#define FSQR_NOALLOC_SCRATCH_BYTES 8388608
int fsqr_lambda_max_noalloc(fsqr_ctx *ctx, const fsqr_design *X, const double *y, double tau,
                            const double *omega, double *out);

#ifdef __cplusplus
}
#endif

#endif /* FSQR_H */
