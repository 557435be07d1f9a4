// Internal declarations shared by the FS-QRPPA kernels and the C-ABI layer.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fsqr.h"

namespace fsqr {

constexpr int kMaxNB = 8;          // fits advanced together per X pass (narrow kernels)
constexpr int kWideMax = 32;       // slots of a wide group (k_wide.cu)
constexpr int kAThreads = 256;     // column kernel: 8 warps
constexpr int kAWarps = kAThreads / 32;
constexpr int kACols = 4;          // columns register-blocked per warp
constexpr int kBThreads = 256;     // X~ beta kernel
constexpr int kBRowsPerThread = 8;
constexpr int kBRows = kBThreads * kBRowsPerThread;
constexpr int kBMaxSplits = 64;
constexpr int kBMinColsPerSplit = 16;
constexpr int kCThreads = 32;      // vector-update kernel: one sample row per thread
constexpr int kCPartials = 4;      // r_p max, r_z max, sum theta, max |theta|
constexpr int kReport = 8;         // kkt, r_p, r_z, r_b, r_1, status, bound, iters

// Column kernel modes.
enum AMode { A_PROX = 0, A_XT = 1, A_XT_BLOCK = 2, A_LIST = 3 };

// The standardised design as the kernels see it. Column j in [0, P):
// x~_ij = a[j] * x_ij + b[j] for an observed entry; a[0] = 0, b[0] = 1
// makes column 0 the intercept. 1 <= j <= c: x_ij = cov[(j-1)*n + i];
// j > c: stored column j-1-c.
struct Dsg {
  int64_t n, p, c, P;
  int fmt;
  const uint8_t *geno;
  int64_t ld;
  const double *cov;
  const double *a;
  const double *b;
  // missing genotype entries (mean imputation, standardised value 0): per
  // stored column s the sample indices midx[mptr[s] .. mptr[s+1]), ascending;
  // both NULL when there are none. The stored codes read as 0 there, so every
  // product of X~ subtracts b_j at those entries (the correction below).
  const int64_t *mptr;
  const int32_t *midx;
};

// State and parameters of a group of NB fits advanced together.
// Per-column arrays are interleaved by fit: v[j*NB + b]; per-sample arrays
// likewise v[i*NB + b] with npad >= n rows whose padding stays 0.
struct Fits {
  int nb;                 // live fits in the group (<= NB); slots >= nb are idle
  int64_t n;              // samples
  int64_t npad;           // rows of the per-sample arrays (multiple of 16)
  const double *y;        // n
  double ymax;            // ||y||_inf
  const double *omega;    // P
  double *beta[2];        // P*NB each; iterate k lives in beta[k & 1]
  double *z, *theta, *r;  // npad*NB
  const int64_t *block_ptr;
  int G;
  const double *eta;      // G
  const double *inv_eta;  // G
  double tau[kMaxNB], lam[kMaxNB], lamnorm[kMaxNB];
  double mu, sigma, tol;
  double ridge;           // elastic-net gamma: the quadratic weight of column j is ridge * omega_j
  int K, max_iter;
  // column-kernel outputs, one slot per CTA of the column kernel
  int gridA, T;
  double *a_rb;   // gridA*NB: max_j dist(s_j, lam_j d|beta_j|)
  double *a_ct;   // gridA*NB: sum_j b_j beta_j (constant part of X~ beta)
  int *a_cnt;     // gridA: active columns found by the CTA
  int *a_list;    // gridA*T: those columns, ascending
  // X~ beta partial sums and their bookkeeping
  double *xb_part;  // kBMaxSplits * npad * NB (FP64 path)
  long long *xb_ipart;  // kBMaxSplits * npad * NB exact integer partials (mixed path)
  double *a_wmax;   // gridA*NB: max |a_j beta_j| over stored columns (mixed path)
  int *meta_i;      // [0] = splits used by the last X~ beta pass, [1] = active columns
  double *meta_d;   // 2*kMaxNB: [0..NB) constant term, [kMaxNB..kMaxNB+NB) integer scale of the last pass
  // vector-kernel partials of the iterate of each parity
  int gridC;
  double *c_part[2];  // gridC * NB * kCPartials
  // totals reduced by the last CTA of each pass (fsqr_device.cuh)
  double *tot_c[2];   // NB * kCPartials per parity
  double *tot_a;      // NB * 3: max dist, constant term, max |a_j beta_j|
  int *a_pre;         // gridA + 1: exclusive prefix of a_cnt
  unsigned *tickets;  // [0] column pass, [1] vector kernel
  unsigned *xb_tick;  // per 128-row tile: splits of the fused X~ beta pass done (tensor-core path)
  // per-fit status
  int *done;        // NB: iteration whose iterate is final, -1 while running
  int *n_done;      // counter of finished fits
  double *report;   // NB * kReport
  const int *it_base;
  // mixed precision
  int mixed, D;
  int dbits;        // bits per digit of theta: 7 (int8 DP4A) or 4 (E4M3 tensor cores)
  int DW;           // digits of the X~ beta weights in the mixed path
  double th_unit;   // 2^(-dbits*D): the last digit's weight relative to the theta scale
  double xb_unit;   // 2^(-7*DW): the same for the X~ beta weights
  int64_t n4p;      // digit words per (fit, digit) row = npad / 4
  int32_t *digits;  // NB * D * n4p words, 4 samples per word
  double *scale;    // NB: quantisation scale 2^e
  double *qcorr;    // npad*NB: - sum_j b_j beta_jb over the missing entries (i, j) of the
                    // active stored columns, added and cleared by the vector update (NULL: none)
  double colbound;  // max_j a_j * sum_i |x_ij| over stored columns
  // wide groups (k_wide.cu): per-slot parameters on the device, so that the
  // host can refill a slot between replays of the captured iteration
  const double *w_tau, *w_lam, *w_lamnorm;  // NB each
  const int *w_k0;  // NB: iteration at which the slot's fit entered (its w^0)
};

// ---- launchers (kernels.cu) -------------------------------------------------
cudaError_t launch_col_stats(const Dsg &X, double *mean, double *sd, int *missing,
                             cudaStream_t s);
cudaError_t launch_affine(const Dsg &X, const double *mean, const double *sd, int standardize,
                          double *a, double *b, cudaStream_t s);
cudaError_t launch_colbound(const Dsg &X, const double *mean, double *out, cudaStream_t s);

// One pass over all columns; see kernels.cu for the four modes.
cudaError_t launch_col_pass(int mode, int NB, const Dsg &X, const Fits &F, int off,
                            const double *vec, const double *vsum, double *s_out,
                            const double *beta_in, cudaStream_t s);
size_t col_pass_smem(int mode, const Fits &F, int NB);
int col_pass_occupancy(int NB, int mixed, int D, size_t smem);
cudaError_t launch_xbeta(int NB, const Dsg &X, const Fits &F, int off, const double *beta_in,
                         cudaStream_t s);
cudaError_t launch_quantize(int NB, const Fits &F, int off, cudaStream_t s);
cudaError_t launch_check(int NB, const Fits &F, int off, cudaStream_t s);
cudaError_t launch_vec(int NB, const Dsg &X, const Fits &F, int off, int init, cudaStream_t s);
cudaError_t launch_advance(int *it_base, int M, cudaStream_t s);
cudaError_t launch_gather_xb(int NB, const Fits &F, double *out, int64_t ldo, int nb,
                             cudaStream_t s);  // out[b*ldo + i], i < F.n (FP64 path)

// Tensor-core column pass (k_tc.cu). Schedule: CTA c takes `rounds` whole
// 128-column tiles (c, c + grid, ...); the rem tiles left over go whole to
// CTAs 0 .. rem-1 (slices = 0) or are cut into `slices` sample slices each,
// computed by CTAs 0 .. rem*slices-1.
struct TcSchedule {
  int grid, rounds, rem, slices;
  int list_stride;  // F.T: 128 * (rounds + 1) + 64
  int slots;        // F.gridA: grid, plus rem list slots when sliced
};
void col_tc_schedule(int64_t p, int64_t n, int num_sms, TcSchedule *out);
int tc_tail_rows(int NB, int D);  // int32 digit sums per tail column and slice
cudaError_t launch_col_tc(int NB, int D, const Dsg &X, const Fits &F, int off, const uint8_t *xt,
                          const uint8_t *dgt, const TcSchedule &sc, int32_t *tail_part,
                          unsigned *tail_tick, int *err, cudaStream_t s);
cudaError_t launch_tile_x(const Dsg &X, uint8_t *xt, int64_t nk, cudaStream_t s);
cudaError_t launch_tile_x2(const Dsg &X, uint8_t *xt, int64_t nk, cudaStream_t s);  // 2-bit, 4 KB tiles

// Wide groups (k_wide.cu), NB in {16, 32} slots. Digit matrix: 8 NB rows x
// npad E4M3 bytes (tiled as for k_quantize_tc); X~ beta weight tiles:
// 11 NB rows x 128 bytes per block of 128 active positions.
bool wide_ok(int NB);
size_t wcol_smem(int NB, int T);
size_t wxbeta_smem(int NB);
int wide_rows(int NB);     // 8 NB
int wide_xrows(int NB);    // 11 NB
cudaError_t launch_wquant(int NB, const Fits &F, int off, uint8_t *dg, cudaStream_t s);
cudaError_t launch_wcol(int NB, const Dsg &X, const Fits &F, int off, const uint8_t *xt, const uint8_t *dgt,
                        int rounds, int *err, cudaStream_t s);
cudaError_t launch_wcheck(int NB, const Fits &F, int off, cudaStream_t s);
// fuse = 1: X~ beta^{k+1} and the vector update of iterate k; fuse = 0 with
// beta_in: the integer partials of X~ beta_in only (start of a solve).
cudaError_t launch_wxbeta(int NB, const Dsg &X, const Fits &F, int off, int fuse, const double *beta_in,
                          int *scol, uint8_t *wtile, int *err, int num_sms, cudaStream_t s);
// Stop-test and quantisation partials of the current iterate of the slots
// with mask[b] != 0, into tot_c[par] (a fit entering its slot).
cudaError_t launch_slot_init(int NB, const Fits &F, int par, const int *mask, cudaStream_t s);
cudaError_t launch_resid_slot(const double *xb, const double *z, const double *y, int64_t n, double *r, int slot,
                              int NB, cudaStream_t s);
// fuse = 1: the same launch also runs the vector update (k_vec) of the
// iterate; fuse = 0: it leaves the integer partials for k_vec.
cudaError_t launch_xbeta_tc(int NB, const Dsg &X, const Fits &F, int off, int fuse, const double *beta_in,
                            int *scol, uint8_t *wtile, int *err, int num_sms, cudaStream_t s);
int xbeta_tc_rows(int NB);
cudaError_t launch_quantize_tc(int NB, int D, const Fits &F, int off, uint8_t *dg, cudaStream_t s);
size_t col_tc_smem(int NB, int D, int T, int f2);
int tc_rows(int NB, int D);

// Learned warm start (k_mlp.cu): a 3 -> 256 -> 256 -> 256 -> 1 ReLU network
// in FP32, flat parameters W_0, b_0, W_1, ... (W_l row-major d_l x d_{l+1}).
constexpr int kMlpIn = 3, kMlpHidden = 256, kMlpLayers = 4;
int64_t mlp_param_count();
cudaError_t mlp_forward(const float *params, const float *x, int64_t rows, float *const *H, float *out,
                        cudaStream_t s);
cudaError_t mlp_grad(const float *params, const float *x, const float *t, const float *w, int64_t rows,
                     float *const *H, float *G0, float *G1, float *f, float *g, float *grad, double *loss,
                     cudaStream_t s);
cudaError_t mlp_adam(float *p, const float *g, float *m, float *v, int64_t count, int64_t step, float lr,
                     cudaStream_t s);
cudaError_t mlp_sample(const float *x, const float *t, const float *w, int64_t rows, int batch, uint64_t seed,
                       int64_t step, float *xb, float *tb, float *wb, cudaStream_t s);
cudaError_t mlp_init(float *p, int *d_dims, uint64_t seed, cudaStream_t s);
cudaError_t launch_warm_features(const double *s_col, int64_t P, int64_t n, double tau, double frac,
                                 const double *lmax, float *u, cudaStream_t s);
cudaError_t launch_warm_beta(const float *f, int64_t P, const double *q, double sdy, double *beta, cudaStream_t s);
cudaError_t launch_warm_dual(const double *y, const double *xb, int64_t n, double tau, double *z, double *theta,
                             cudaStream_t s);

// Setup and reporting helpers (k_setup.cu).
cudaError_t launch_vec_stats(const double *v, int64_t n, double *out3, cudaStream_t s);
cudaError_t launch_sum_cols(const double *v, int64_t n, int64_t ldv, int nvec, double *sums,
                            double *sqsums, cudaStream_t s);
cudaError_t launch_select(const double *y, int64_t n, int64_t k, double *out, cudaStream_t s);
cudaError_t launch_lmax_vec(const double *y, int64_t n, int64_t npad, double tau,
                            const double *q, double *v, cudaStream_t s);
cudaError_t launch_colmax_ratio(const double *s_col, const double *omega, int64_t P,
                                double scale, double *out, cudaStream_t s);
cudaError_t launch_power_init(double *v, const int64_t *block_ptr, int G, int64_t P,
                              cudaStream_t s);
cudaError_t launch_power_step(const double *w, const int64_t *block_ptr, int G, int64_t P,
                              double *v, double *wnorm, cudaStream_t s);
cudaError_t launch_xv_blocks(const Dsg &X, const double *v, const int64_t *splits,
                             const int *split_of_block, int G, int nsplit, double *u,
                             int64_t npad, double *part, cudaStream_t s);
cudaError_t launch_pack(const double *src, int64_t lds, double *dst, int64_t len, int nb,
                        int NB, int64_t dst_rows, cudaStream_t s);
cudaError_t launch_unpack(const double *src, double *dst, int64_t lds, int64_t len, int nb,
                          int NB, cudaStream_t s);
cudaError_t launch_fill(double *p, double v, int64_t n, cudaStream_t s);
cudaError_t launch_init_state(int NB, const Fits &F, int nb, int warm, cudaStream_t s);
cudaError_t launch_dual_point(int NB, const double *theta, int64_t n, int64_t npad,
                              const double *taus, int nb, double *out, double *sums,
                              cudaStream_t s);
cudaError_t launch_min_omega(const double *omega, int64_t P, double *out, cudaStream_t s);
cudaError_t launch_summary(int NB, int nb, int64_t n, int64_t P, const double *y,
                           const double *z, const double *r, const double *beta,
                           const double *omega, const double *taus, const double *lams,
                           const double *s_chk, const double *tc, double ridge, double *out, cudaStream_t s);
cudaError_t launch_kkt_given(int64_t n, int64_t P, const double *y, const double *xb,
                             const double *z, const double *theta, const double *s,
                             const double *beta, const double *omega, double tau, double lam,
                             double *out, cudaStream_t st);
cudaError_t launch_back_transform(const Dsg &X, const double *beta, int B, double *out,
                                  cudaStream_t s);
cudaError_t launch_path_stats(const double *q, const double *y, const double *taus, int64_t n, const double *beta,
                              int64_t P, int B, double *out, cudaStream_t s);
cudaError_t launch_coverage(const double *qlo, const double *qhi, const double *y, int64_t n, double *out,
                            cudaStream_t s);
// Missing genotype entries (k_setup.cu): counts per stored column, the
// column-major index lists, and an int8 copy with the missing codes set to 0.
cudaError_t launch_miss_count(const Dsg &X, int *cnt, cudaStream_t s);
cudaError_t launch_miss_fill(const Dsg &X, const int64_t *mptr, int32_t *midx, cudaStream_t s);
cudaError_t launch_sanitize_int8(const Dsg &X, uint8_t *dst, cudaStream_t s);
// u[g*npad + i] -= b_j v_j for the missing entries (i, j) of block g's stored
// columns (the power method's X~_g v).
cudaError_t launch_miss_xv(const Dsg &X, const double *v, const int64_t *block_ptr, int G, double *u,
                           int64_t npad, cudaStream_t s);
// qcorr[i*NB + b] -= b_j beta_jb over the missing entries of the active stored
// columns (listed by the column pass), beta = beta_in or beta^{k+1}.
cudaError_t launch_miss_xb(int NB, const Dsg &X, const Fits &F, int off, const double *beta_in, cudaStream_t s);
cudaError_t launch_gather_cols(const uint8_t *src, int64_t ld, const int32_t *sel, int64_t nsel, uint8_t *dst,
                               cudaStream_t s);
cudaError_t launch_index_copy(const double *src, int64_t lds, const int32_t *idx, int64_t m, int nb, double *dst,
                              int64_t ldd, int scatter, cudaStream_t s);
cudaError_t launch_wait_selftest(long long budget, int arrive, int *err, int *ok, cudaStream_t s);
cudaError_t launch_lla_weights(const double *src, const double *omega, int64_t P, double lam, double a, int type,
                               double scale, double *out, cudaStream_t s);

}  // namespace fsqr
