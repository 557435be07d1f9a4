// C-ABI layer of the FS-QRPPA library: argument checks, device workspace,
// setup (column statistics, lambda_max, eta by the power method) and the
// driver of the inner iteration, which advances groups of up to 8 fits per X
// pass and replays the iteration as captured CUDA graphs of M steps.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fsqr_internal.h"

using namespace fsqr;

struct fsqr_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  std::string err;
  std::map<std::string, std::pair<void *, size_t>> ws;
  std::map<std::string, int> tuned;  // autotuned fits per X pass, by problem shape
  double *hpin = nullptr;  // pinned host scratch
  size_t hpin_n = 0;
  bool prof = false;
  fsqr_profile pf{};
  cudaEvent_t ev[6] = {};
  cudaEvent_t legacy_ev = nullptr;
};

namespace {

constexpr int kVersion = 10000;

int fail(fsqr_ctx *ctx, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, FSQR_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),        \
                  __FILE__, __LINE__);                                                    \
  } while (0)

// A kernel launch through a launcher: counted, then checked.
#define LK(call)                       \
  do {                                 \
    ctx->pf.kernel_launches += 1;      \
    CK(call);                          \
  } while (0)

#define TRY(expr)              \
  do {                         \
    int rc_ = (expr);          \
    if (rc_ != FSQR_OK) return rc_; \
  } while (0)

// Start of every entry point: select the device and, when the library owns
// its stream, order it after work already queued on the legacy default
// stream (where callers without an explicit stream put their inputs).
int enter(fsqr_ctx *ctx) {
  ctx->err.clear();
  CK(cudaSetDevice(ctx->device));
  if (ctx->own_stream) {
    CK(cudaEventRecord(ctx->legacy_ev, cudaStreamLegacy));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->legacy_ev, 0));
  }
  return FSQR_OK;
}

// Named device workspace, grown on demand (contents are not preserved).
template <class T>
int wsget(fsqr_ctx *ctx, const char *name, size_t count, T **out) {
  size_t bytes = std::max<size_t>(count * sizeof(T), 16);
  auto &slot = ctx->ws[name];
  if (slot.second < bytes) {
    if (slot.first) cudaFree(slot.first);
    slot.first = nullptr;
    slot.second = 0;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, FSQR_ENOMEM, "cudaMalloc(%zu bytes) for %s: %s", bytes, name,
                  cudaGetErrorString(e));
    }
    slot.first = p;
    slot.second = bytes;
  }
  *out = static_cast<T *>(slot.first);
  return FSQR_OK;
}

int pinned(fsqr_ctx *ctx, size_t count, double **out) {
  if (ctx->hpin_n < count) {
    if (ctx->hpin) cudaFreeHost(ctx->hpin);
    ctx->hpin = nullptr;
    ctx->hpin_n = 0;
    CK(cudaMallocHost(&ctx->hpin, count * sizeof(double)));
    ctx->hpin_n = count;
  }
  *out = ctx->hpin;
  return FSQR_OK;
}

int64_t pad16(int64_t n) { return (n + 15) / 16 * 16; }

int64_t col_bytes(int64_t n, int fmt) {
  if (fmt == FSQR_DENSE_F64) return 8 * n;
  if (fmt == FSQR_INT8) return n;
  return (n + 3) / 4;
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int check_design(fsqr_ctx *ctx, const fsqr_design *d) {
  if (!d) return fail(ctx, FSQR_EINVAL, "design is NULL");
  if (d->n < 1) return fail(ctx, FSQR_EINVAL, "n must be >= 1 (got %lld)", (long long)d->n);
  if (d->p < 0 || d->c < 0) return fail(ctx, FSQR_EINVAL, "p and c must be >= 0");
  if (1 + d->c + d->p > (int64_t)INT32_MAX - 1024)
    return fail(ctx, FSQR_EINVAL, "too many columns (P = %lld)", (long long)(1 + d->c + d->p));
  if (d->n > (int64_t)1 << 24) return fail(ctx, FSQR_EINVAL, "n > 2^24 is not supported");
  if (d->geno_format < FSQR_DENSE_F64 || d->geno_format > FSQR_2BIT)
    return fail(ctx, FSQR_EINVAL, "unknown geno_format %d", d->geno_format);
  if (d->standardize != 0 && d->standardize != 1)
    return fail(ctx, FSQR_EINVAL, "standardize must be 0 or 1");
  if (d->p > 0) {
    if (!d->geno) return fail(ctx, FSQR_EINVAL, "geno is NULL with p > 0");
    if (((uintptr_t)d->geno) % 16) return fail(ctx, FSQR_EINVAL, "geno must be 16-byte aligned");
    if (d->geno_ld % 16) return fail(ctx, FSQR_EINVAL, "geno_ld must be a multiple of 16");
    if (d->geno_ld < col_bytes(d->n, d->geno_format))
      return fail(ctx, FSQR_EINVAL, "geno_ld %lld < %lld bytes needed per column",
                  (long long)d->geno_ld, (long long)col_bytes(d->n, d->geno_format));
  }
  if (d->c > 0 && !d->cov) return fail(ctx, FSQR_EINVAL, "cov is NULL with c > 0");
  if ((d->col_mean == nullptr) != (d->col_sd == nullptr))
    return fail(ctx, FSQR_EINVAL, "col_mean and col_sd must be given together");
  return FSQR_OK;
}

int check_blocks(fsqr_ctx *ctx, const int64_t *bp, int G, int64_t P) {
  if (G < 1) return fail(ctx, FSQR_EINVAL, "G must be >= 1");
  if (!bp) return fail(ctx, FSQR_EINVAL, "block_ptr is NULL");
  if (bp[0] != 0) return fail(ctx, FSQR_EINVAL, "block_ptr[0] must be 0");
  for (int g = 0; g < G; ++g)
    if (bp[g + 1] <= bp[g]) return fail(ctx, FSQR_EINVAL, "block_ptr must be strictly increasing");
  if (bp[G] != P)
    return fail(ctx, FSQR_EINVAL, "block_ptr[G] = %lld must equal P = %lld", (long long)bp[G],
                (long long)P);
  return FSQR_OK;
}

// Design prepared for the kernels: affine maps a_j, b_j from the column
// statistics (given or computed), and the count of missing entries.
struct Prep {
  Dsg X;
  const double *mean = nullptr;  // length c+p
  const double *sd = nullptr;
  int missing = 0;
  double colbound = 0.0;
};

int prepare(fsqr_ctx *ctx, const fsqr_design *d, Prep *pp, bool need_colbound) {
  TRY(check_design(ctx, d));
  Prep &p = *pp;
  Dsg &X = p.X;
  X.n = d->n;
  X.p = d->p;
  X.c = d->c;
  X.P = 1 + d->c + d->p;
  X.fmt = d->geno_format;
  X.geno = static_cast<const uint8_t *>(d->geno);
  X.ld = d->geno_ld;
  X.cov = d->cov;
  const int64_t F = d->c + d->p;
  double *mean, *sd, *a, *b;
  int *miss;
  TRY(wsget(ctx, "stat_mean", F, &mean));
  TRY(wsget(ctx, "stat_sd", F, &sd));
  TRY(wsget(ctx, "aff_a", X.P, &a));
  TRY(wsget(ctx, "aff_b", X.P, &b));
  TRY(wsget(ctx, "stat_missing", 1, &miss));
  CK(cudaMemsetAsync(miss, 0, sizeof(int), ctx->stream));
  LK(launch_col_stats(X, mean, sd, miss, ctx->stream));
  p.mean = d->col_mean ? d->col_mean : mean;
  p.sd = d->col_sd ? d->col_sd : sd;
  LK(launch_affine(X, p.mean, p.sd, d->standardize, a, b, ctx->stream));
  X.a = a;
  X.b = b;
  int hmiss = 0;
  CK(cudaMemcpyAsync(&hmiss, miss, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  if (need_colbound) {
    double *cb;
    TRY(wsget(ctx, "colbound", 1, &cb));
    LK(launch_colbound(X, p.mean, cb, ctx->stream));
    CK(cudaMemcpyAsync(&p.colbound, cb, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  p.missing = hmiss;
  if (hmiss > 0)
    return fail(ctx, FSQR_EINVAL,
                "%d missing genotype entries: mean imputation of missing entries is not "
                "supported by this library",
                hmiss);
  return FSQR_OK;
}

// Column-pass tiling: CTA c owns T consecutive columns; T is a multiple of
// 32 and the grid fits in one wave of resident CTAs when P allows it.
void col_tiling(fsqr_ctx *ctx, int64_t P, int per_sm, int *gridA, int *T) {
  const int64_t target = std::max<int64_t>(1, (int64_t)ctx->num_sms * std::max(1, per_sm));
  int64_t t = (P + target - 1) / target;
  t = std::max<int64_t>(32, (t + 31) / 32 * 32);
  *T = (int)t;
  *gridA = (int)((P + t - 1) / t);
}

// Totals, list prefix and last-CTA tickets of a pass (zeroed tickets).
int alloc_totals(fsqr_ctx *ctx, Fits &F, const char *tag) {
  std::string t(tag);
  TRY(wsget(ctx, (t + "_totc0").c_str(), (size_t)kMaxNB * kCPartials, &F.tot_c[0]));
  TRY(wsget(ctx, (t + "_totc1").c_str(), (size_t)kMaxNB * kCPartials, &F.tot_c[1]));
  TRY(wsget(ctx, (t + "_tota").c_str(), (size_t)kMaxNB * 3, &F.tot_a));
  TRY(wsget(ctx, (t + "_apre").c_str(), (size_t)F.gridA + 1, &F.a_pre));
  TRY(wsget(ctx, (t + "_tick").c_str(), 2, &F.tickets));
  CK(cudaMemsetAsync(F.tickets, 0, 2 * sizeof(unsigned), ctx->stream));
  CK(cudaMemsetAsync(F.tot_c[0], 0, sizeof(double) * kMaxNB * kCPartials, ctx->stream));
  CK(cudaMemsetAsync(F.tot_c[1], 0, sizeof(double) * kMaxNB * kCPartials, ctx->stream));
  return FSQR_OK;
}

int nb_template(int nb) {
  if (nb <= 1) return 1;
  if (nb == 2) return 2;
  if (nb == 3) return 3;
  if (nb == 4) return 4;
  return 8;
}

// Host-side y statistics: ||y||_inf and population sd.
int y_stats(fsqr_ctx *ctx, const double *y, int64_t n, double *ymax, double *ysd) {
  double *st;
  TRY(wsget(ctx, "ystats", 3, &st));
  LK(launch_vec_stats(y, n, st, ctx->stream));
  double h[3];
  CK(cudaMemcpyAsync(h, st, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const double m = h[0] / (double)n;
  double v = h[1] / (double)n - m * m;
  *ymax = h[2];
  *ysd = sqrt(v > 0 ? v : 0.0);
  if (!(h[0] == h[0]) || !(h[1] == h[1]) || isinf(h[1]))
    return fail(ctx, FSQR_ENUMERIC, "y contains NaN or Inf");
  return FSQR_OK;
}

// A Fits with only the column tiling set, for the non-iteration passes.
Fits pass_fits(fsqr_ctx *ctx, const Dsg &X) {
  Fits F{};
  F.n = X.n;
  F.npad = pad16(X.n);
  col_tiling(ctx, X.P, 4, &F.gridA, &F.T);
  return F;
}

// Device side of lambda_max(tau): q = y_(ceil(n tau)), s = X~^T v with
// v_i = tau - 1{y_i < q}, and o = lambda_max, all left in the workspace.
struct LmaxDev {
  double *q, *s, *o;
};

int lambda_max_dev(fsqr_ctx *ctx, const Prep &pr, const double *y, double tau, const double *omega,
                   LmaxDev *out) {
  const Dsg &X = pr.X;
  const int64_t n = X.n, npad = pad16(n);
  double *q, *v, *vs, *s, *o;
  TRY(wsget(ctx, "lmax_q", 1, &q));
  TRY(wsget(ctx, "lmax_v", npad, &v));
  TRY(wsget(ctx, "lmax_vs", 1, &vs));
  TRY(wsget(ctx, "lmax_s", X.P, &s));
  TRY(wsget(ctx, "lmax_o", 1, &o));
  int64_t k = (int64_t)ceil((double)n * tau);
  if (k < 1) k = 1;
  if (k > n) k = n;
  LK(launch_select(y, n, k, q, ctx->stream));
  LK(launch_lmax_vec(y, n, npad, tau, q, v, ctx->stream));
  LK(launch_sum_cols(v, n, npad, 1, vs, nullptr, ctx->stream));
  Fits F = pass_fits(ctx, X);
  LK(launch_col_pass(A_XT, 1, X, F, 0, v, vs, s, nullptr, ctx->stream));
  LK(launch_colmax_ratio(s, omega, X.P, (double)n, o, ctx->stream));
  *out = LmaxDev{q, s, o};
  return FSQR_OK;
}

// lambda_max(tau) for one tau (host result).
int lambda_max_impl(fsqr_ctx *ctx, const Prep &pr, const double *y, double tau, const double *omega,
                    double *out) {
  LmaxDev L;
  TRY(lambda_max_dev(ctx, pr, y, tau, omega, &L));
  CK(cudaMemcpyAsync(out, L.o, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FSQR_OK;
}

// eta_g = (1 + margin) mu Lambda_hat_g by the batched power method.
int eta_impl(fsqr_ctx *ctx, const Prep &pr, const int64_t *bp, int G, double mu, double margin,
             int max_iter, double tol, double *eta_out) {
  const Dsg &X = pr.X;
  const int64_t n = X.n, npad = pad16(n), P = X.P;
  // split table: ranges of at most C columns inside one block
  const int64_t C = std::max<int64_t>(256, (P + 1023) / 1024);
  std::vector<int64_t> splits;
  std::vector<int> sob(G + 1, 0);
  for (int g = 0; g < G; ++g) {
    sob[g] = (int)(splits.size() / 2);
    for (int64_t j = bp[g]; j < bp[g + 1]; j += C) {
      splits.push_back(j);
      splits.push_back(std::min(bp[g + 1], j + C));
    }
  }
  sob[G] = (int)(splits.size() / 2);
  const int nsplit = sob[G];
  int64_t *d_splits, *d_bp;
  int *d_sob;
  double *v, *U, *part, *usum, *usq, *w, *wn;
  TRY(wsget(ctx, "pw_splits", splits.size(), &d_splits));
  TRY(wsget(ctx, "pw_sob", (size_t)G + 1, &d_sob));
  TRY(wsget(ctx, "pw_bp", (size_t)G + 1, &d_bp));
  TRY(wsget(ctx, "pw_v", P, &v));
  TRY(wsget(ctx, "pw_U", (size_t)G * npad, &U));
  TRY(wsget(ctx, "pw_part", (size_t)nsplit * npad, &part));
  TRY(wsget(ctx, "pw_usum", G, &usum));
  TRY(wsget(ctx, "pw_usq", G, &usq));
  TRY(wsget(ctx, "pw_w", P, &w));
  TRY(wsget(ctx, "pw_wn", G, &wn));
  CK(cudaMemcpyAsync(d_splits, splits.data(), splits.size() * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(d_sob, sob.data(), sob.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(d_bp, bp, (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
  LK(launch_power_init(v, d_bp, G, P, ctx->stream));
  Fits F = pass_fits(ctx, X);
  F.block_ptr = d_bp;
  F.G = G;
  std::vector<double> lam(G, 0.0), res(G, 0.0), hq(G), hw(G);
  std::vector<char> frozen(G, 0);
  int left = G;
  for (int t = 1; t <= max_iter && left > 0; ++t) {
    LK(launch_xv_blocks(X, v, d_splits, d_sob, G, nsplit, U, npad, part, ctx->stream));
    LK(launch_sum_cols(U, n, npad, G, usum, usq, ctx->stream));
    LK(launch_col_pass(A_XT_BLOCK, 1, X, F, 0, U, usum, w, nullptr, ctx->stream));
    LK(launch_power_step(w, d_bp, G, P, v, wn, ctx->stream));
    CK(cudaMemcpyAsync(hq.data(), usq, G * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(hw.data(), wn, G * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int g = 0; g < G; ++g) {
      if (frozen[g]) continue;
      if (hw[g] == 0.0) {
        res[g] = 0.0;
        frozen[g] = 1;
        --left;
      } else if (fabs(hq[g] - lam[g]) <= tol * hq[g]) {
        res[g] = hq[g];
        frozen[g] = 1;
        --left;
      } else {
        lam[g] = hq[g];
      }
    }
  }
  for (int g = 0; g < G; ++g) {
    const double L = frozen[g] ? res[g] : lam[g];
    eta_out[g] = (1.0 + margin) * mu * (L > 0.0 ? L : 1.0);
  }
  return FSQR_OK;
}

int check_opts(fsqr_ctx *ctx, const fsqr_opts *o, int G) {
  if (!o) return fail(ctx, FSQR_EINVAL, "opts is NULL");
  if (!(o->tol >= 0.0)) return fail(ctx, FSQR_EINVAL, "tol must be >= 0");
  if (o->max_iter < 0) return fail(ctx, FSQR_EINVAL, "max_iter must be >= 0");
  if (o->check_every < 1) return fail(ctx, FSQR_EINVAL, "check_every must be >= 1");
  if (o->precision != FSQR_FP64 && o->precision != FSQR_MIXED && o->precision != FSQR_MIXED_SIMT)
    return fail(ctx, FSQR_EINVAL, "unknown precision %d", o->precision);
  if (o->warm < FSQR_WARM_NONE || o->warm > FSQR_WARM_LEARNED)
    return fail(ctx, FSQR_EINVAL, "unknown warm mode %d", o->warm);
  if (o->warm == FSQR_WARM_LEARNED && !o->warm_params)
    return fail(ctx, FSQR_EINVAL, "FSQR_WARM_LEARNED needs opts.warm_params");
  if (o->precision != FSQR_FP64 && (o->digits < 3 || o->digits > 5))
    return fail(ctx, FSQR_EINVAL, "digits must be in 3..5");
  if (o->max_group < 0 || o->max_group > kMaxNB)
    return fail(ctx, FSQR_EINVAL, "max_group must be in 0..8");
  if (o->eta)
    for (int g = 0; g < G; ++g)
      if (!(o->eta[g] > 0.0) || isinf(o->eta[g]))
        return fail(ctx, FSQR_EINVAL, "eta[%d] must be finite and > 0", g);
  if (!(o->eta_margin >= 0.0)) return fail(ctx, FSQR_EINVAL, "eta_margin must be >= 0");
  return FSQR_OK;
}

// One group of nb fits advanced together to convergence.
struct GroupSpec {
  int nb;
  double tau[kMaxNB], lam[kMaxNB], lamnorm[kMaxNB];
  int fit[kMaxNB];          // output fit index of each slot
  int src_fit[kMaxNB];      // start: fit index to read beta/z/theta from (-1 = cold)
};

struct SolveEnv {
  const Prep *pr;
  const double *y;
  const double *omega;
  int64_t *d_bp;
  int G;
  double *d_eta, *d_ieta;
  double mu, ymax;
  bool gap_defined;
  const fsqr_opts *o;
  double *beta, *z, *theta;  // user arrays (fit-major)
  fsqr_info *infos;
  double deadline_ms;        // <= 0: none
};

int solve_group(fsqr_ctx *ctx, const SolveEnv &E, const GroupSpec &gs) {
  const Dsg &X = E.pr->X;
  const int nb = gs.nb;
  const int NB = nb_template(nb);
  const int64_t n = X.n, npad = pad16(n), P = X.P;
  const bool mixed = E.o->precision == FSQR_MIXED || E.o->precision == FSQR_MIXED_SIMT;
  // tensor-core passes: int8 storage, at most 63 covariates, <= 8 fits, and
  // sizes for which the integer arithmetic stays exact: a digit-product sum
  // over n samples (or over the active columns of an X~ beta split, at most
  // p) of |g t| <= 16 is a multiple of 2^-9 below 2^24 * 2^-9 in FP32 when
  // n, p <= 2^20; the recombined X~ beta, sum_j g_ij W_j with |W_j| < 2^43,
  // stays below 2^63 in int64 when p <= 2^19
  const bool tc = E.o->precision == FSQR_MIXED && X.fmt == FSQR_INT8 && X.p > 0 && X.c <= 63 && NB <= 8 &&
                  X.n <= ((int64_t)1 << 20) && X.p <= ((int64_t)1 << 19);
  const double t0 = now_ms();
  cudaStream_t st = ctx->stream;

  Fits F{};
  F.nb = nb;
  F.n = n;
  F.npad = npad;
  F.y = E.y;
  F.ymax = E.ymax;
  F.omega = E.omega;
  F.block_ptr = E.d_bp;
  F.G = E.G;
  F.eta = E.d_eta;
  F.inv_eta = E.d_ieta;
  for (int b = 0; b < kMaxNB; ++b) {
    F.tau[b] = b < nb ? gs.tau[b] : 0.5;
    F.lam[b] = b < nb ? gs.lam[b] : 0.0;
    F.lamnorm[b] = b < nb ? gs.lamnorm[b] : 1.0;
  }
  F.mu = E.mu;
  F.sigma = E.mu / (double)(E.G + 1);
  F.tol = E.o->tol;
  F.K = E.o->check_every;
  F.max_iter = E.o->max_iter;
  F.mixed = mixed ? 1 : 0;
  F.D = mixed ? (tc ? (E.o->digits >= 4 ? 7 : 6) : E.o->digits) : 0;
  F.dbits = tc ? 4 : 7;
  F.DW = mixed ? 6 : 0;
  F.th_unit = ldexp(1.0, -F.dbits * F.D);
  F.xb_unit = tc ? ldexp(1.0, -4 * 11) : ldexp(1.0, -7 * F.DW);
  F.n4p = npad / 4;
  F.colbound = E.pr->colbound;
  // tiling from the occupancy of the kernel this group runs
  TcSchedule tsc{};
  if (tc) {
    col_tc_schedule(X.p, n, ctx->num_sms, &tsc);
    F.T = tsc.list_stride;  // whole-tile columns, then up to 64 dense columns
    F.gridA = tsc.slots;
  } else {
    Fits tmp = F;
    tmp.T = 32;
    size_t smem_est = col_pass_smem(A_PROX, tmp, NB) + 4096;
    int per_sm = col_pass_occupancy(NB, F.mixed, F.D, smem_est);
    if (per_sm < 1)
      return fail(ctx, FSQR_EINVAL, "group of %d fits does not fit on an SM (shared memory %zu B)",
                  nb, smem_est);
    col_tiling(ctx, P, per_sm, &F.gridA, &F.T);
  }
  F.gridC = (int)((n + kCThreads - 1) / kCThreads);  // row CTAs; the grid's y is the fit
  TRY(wsget(ctx, "g_beta0", (size_t)P * NB, &F.beta[0]));
  TRY(wsget(ctx, "g_beta1", (size_t)P * NB, &F.beta[1]));
  TRY(wsget(ctx, "g_z", (size_t)npad * NB, &F.z));
  TRY(wsget(ctx, "g_theta", (size_t)npad * NB, &F.theta));
  TRY(wsget(ctx, "g_r", (size_t)npad * NB, &F.r));
  TRY(wsget(ctx, "g_arb", (size_t)F.gridA * NB, &F.a_rb));
  TRY(wsget(ctx, "g_act", (size_t)F.gridA * NB, &F.a_ct));
  TRY(wsget(ctx, "g_acnt", (size_t)F.gridA, &F.a_cnt));
  TRY(wsget(ctx, "g_alist", (size_t)F.gridA * F.T, &F.a_list));
  TRY(wsget(ctx, "g_xbpart", (size_t)kBMaxSplits * npad * NB, &F.xb_part));
  TRY(wsget(ctx, "g_metai", 4, &F.meta_i));
  TRY(wsget(ctx, "g_metad", 2 * kMaxNB, &F.meta_d));
  TRY(wsget(ctx, "g_cpart0", (size_t)F.gridC * NB * kCPartials, &F.c_part[0]));
  TRY(wsget(ctx, "g_cpart1", (size_t)F.gridC * NB * kCPartials, &F.c_part[1]));
  TRY(alloc_totals(ctx, F, "g"));
  TRY(wsget(ctx, "g_done", kMaxNB, &F.done));
  TRY(wsget(ctx, "g_ndone", 1, &F.n_done));
  TRY(wsget(ctx, "g_report", (size_t)kMaxNB * kReport, &F.report));
  int *it_base;
  TRY(wsget(ctx, "g_itbase", 1, &it_base));
  F.it_base = it_base;
  uint8_t *dg = nullptr, *xt = nullptr, *wtile = nullptr;
  int *d_err = nullptr, *scol = nullptr;
  int32_t *tail_part = nullptr;
  unsigned *tail_tick = nullptr;
  if (tc) {
    // tiled copy of X (byte image of the swizzled operand tiles) and the
    // tiled digit matrix, one 128 x N block per 128-sample chunk
    const int N = tc_rows(NB, F.D);
    const int64_t nk = (n + 127) / 128;
    const int64_t ntile = (X.p + 127) / 128;
    TRY(wsget(ctx, "g_dgt", (size_t)(nk * N * 128), &dg));
    TRY(wsget(ctx, "g_xt", (size_t)(ntile * nk * 16384), &xt));
    TRY(wsget(ctx, "g_err", 1, &d_err));
    CK(cudaMemsetAsync(dg, 0, (size_t)(nk * N * 128), st));
    CK(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    LK(launch_tile_x(X, xt, nk, st));
    const int64_t maxkb = (P + 127) / 128;
    TRY(wsget(ctx, "g_scol", (size_t)(maxkb * 128), &scol));
    TRY(wsget(ctx, "g_wtile", (size_t)(maxkb * xbeta_tc_rows(NB) * 128), &wtile));
    TRY(wsget(ctx, "g_xbtick", (size_t)((n + 127) / 128), &F.xb_tick));
    CK(cudaMemsetAsync(F.xb_tick, 0, sizeof(unsigned) * (size_t)((n + 127) / 128), st));
    TRY(wsget(ctx, "g_tailpart", (size_t)std::max(1, tsc.rem * tsc.slices) * tc_tail_rows(NB, F.D) * 128,
              &tail_part));
    TRY(wsget(ctx, "g_tailtick", (size_t)std::max(1, tsc.rem), &tail_tick));
    CK(cudaMemsetAsync(tail_tick, 0, sizeof(unsigned) * (size_t)std::max(1, tsc.rem), st));
    const size_t smem = col_tc_smem(NB, F.D, F.T);
    if (smem > 200 * 1024)
      return fail(ctx, FSQR_EINVAL, "tensor-core column pass needs %zu B of shared memory", smem);
  }
  if (mixed) {
    TRY(wsget(ctx, "g_digits", (size_t)NB * std::max(F.D, 1) * F.n4p, &F.digits));
    TRY(wsget(ctx, "g_scale", kMaxNB, &F.scale));
    TRY(wsget(ctx, "g_xbipart", (size_t)kBMaxSplits * npad * NB, &F.xb_ipart));
    TRY(wsget(ctx, "g_awmax", (size_t)F.gridA * NB, &F.a_wmax));
  }
  if (!tc) {
    const size_t smem = col_pass_smem(A_PROX, F, NB);
    if (smem > 227 * 1024)
      return fail(ctx, FSQR_EINVAL, "mixed group needs %zu B of shared memory (> 227 KB)", smem);
  }

  // ---- start point
  CK(cudaMemsetAsync(F.report, 0, sizeof(double) * kMaxNB * kReport, st));
  CK(cudaMemsetAsync(F.z, 0, sizeof(double) * npad * NB, st));
  CK(cudaMemsetAsync(F.theta, 0, sizeof(double) * npad * NB, st));
  CK(cudaMemsetAsync(F.r, 0, sizeof(double) * npad * NB, st));
  CK(cudaMemsetAsync(F.beta[0], 0, sizeof(double) * P * NB, st));
  CK(cudaMemsetAsync(F.beta[1], 0, sizeof(double) * P * NB, st));
  bool cold = true;
  for (int b = 0; b < nb; ++b) cold = cold && gs.src_fit[b] < 0;
  LK(launch_init_state(NB, F, nb, cold ? FSQR_WARM_NONE : FSQR_WARM_GIVEN, st));
  if (!cold) {
    // per slot: warm slots copy from the user's arrays, cold ones take y
    for (int b = 0; b < nb; ++b) {
      const int sf = gs.src_fit[b];
      if (sf >= 0) {
        LK(launch_pack(E.beta + (int64_t)sf * P, P, F.beta[0] + b, P, 1, NB, P, st));
        LK(launch_pack(E.z + (int64_t)sf * n, n, F.z + b, n, 1, NB, npad, st));
        LK(launch_pack(E.theta + (int64_t)sf * n, n, F.theta + b, n, 1, NB, npad, st));
      } else {
        LK(launch_pack(E.y, n, F.z + b, n, 1, NB, npad, st));
      }
    }
  }
  LK(launch_col_pass(A_LIST, NB, X, F, 0, nullptr, nullptr, nullptr, F.beta[0], st));
  if (tc) LK(launch_xbeta_tc(NB, X, F, 0, 0, F.beta[0], scol, wtile, d_err, ctx->num_sms, st));
  else LK(launch_xbeta(NB, X, F, 0, F.beta[0], st));
  LK(launch_vec(NB, X, F, 0, 1, st));

  // ---- the iteration as a captured graph of M steps
  const int K = F.K;
  const int M = K * std::max(1, (20 + K - 1) / K);
  const bool prof = ctx->prof;
  if (prof && !ctx->ev[0])
    for (int e = 0; e < 6; ++e) CK(cudaEventCreate(&ctx->ev[e]));
  // kernels per step: [quantize] col [check] (xprep + fused xbeta/vector | xbeta + vec)
  int per_graph = 1;  // the advance kernel
  for (int off = 0; off < M; ++off) per_graph += (mixed ? 1 : 0) + 3 + (off % K == 0 ? 1 : 0);
  // Enqueues steps base..base+M-1 (kernels read the base from it_base); with
  // sample set, events bracket the kernels of the last step. The stop test of
  // w^k reads only the column pass of step k and the vector pass of step k-1,
  // so it runs before the X~ beta pass, which on the tensor-core path also
  // applies the vector update.
  auto enqueue = [&](bool sample) -> cudaError_t {
    cudaError_t ce = cudaSuccess;
    for (int off = 0; off < M && ce == cudaSuccess; ++off) {
      const bool sm = sample && off == M - 1;
      if (tc) ce = launch_quantize_tc(NB, F.D, F, off, dg, st);
      else if (mixed) ce = launch_quantize(NB, F, off, st);
      if (sm && ce == cudaSuccess) ce = cudaEventRecord(ctx->ev[0], st);
      if (tc) {
        if (ce == cudaSuccess) ce = launch_col_tc(NB, F.D, X, F, off, xt, dg, tsc, tail_part, tail_tick, d_err, st);
      } else if (ce == cudaSuccess) {
        ce = launch_col_pass(A_PROX, NB, X, F, off, nullptr, nullptr, nullptr, nullptr, st);
      }
      if (sm && ce == cudaSuccess) ce = cudaEventRecord(ctx->ev[1], st);
      if (off % K == 0 && ce == cudaSuccess) ce = launch_check(NB, F, off, st);
      if (sm && ce == cudaSuccess) ce = cudaEventRecord(ctx->ev[2], st);
      if (ce == cudaSuccess)
        ce = tc ? launch_xbeta_tc(NB, X, F, off, 1, nullptr, scol, wtile, d_err, ctx->num_sms, st)
                : launch_xbeta(NB, X, F, off, nullptr, st);
      if (sm && ce == cudaSuccess) ce = cudaEventRecord(ctx->ev[3], st);
      if (!tc && ce == cudaSuccess) ce = launch_vec(NB, X, F, off, 0, st);
      if (sm && ce == cudaSuccess) ce = cudaEventRecord(ctx->ev[4], st);
    }
    if (ce == cudaSuccess) ce = launch_advance(it_base, M, st);
    return ce;
  };
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  cudaError_t ce = enqueue(false);
  cudaError_t ee = cudaStreamEndCapture(st, &graph);
  if (ce != cudaSuccess || ee != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return fail(ctx, FSQR_ECUDA, "graph capture failed: %s",
                cudaGetErrorString(ce != cudaSuccess ? ce : ee));
  }
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return fail(ctx, FSQR_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));

  double *hp;
  TRY(pinned(ctx, 64, &hp));
  int *hdone = reinterpret_cast<int *>(hp);
  const int64_t max_launch = (int64_t)E.o->max_iter / M + 3;
  bool timed_out = false;
  int host_base = 0;
  int rc = FSQR_OK;
  for (int64_t l = 0;; ++l) {
    // every 4th replay runs eagerly with events around its last step's kernels
    const bool sample = prof && (l % 4 == 0);
    ce = sample ? enqueue(true) : cudaGraphLaunch(exec, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(hdone, F.n_done, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
      rc = fail(ctx, FSQR_ECUDA, "iteration graph: %s", cudaGetErrorString(ce));
      break;
    }
    host_base += M;
    ctx->pf.kernel_launches += per_graph;
    if (sample) {
      float a = 0.f, b = 0.f, c = 0.f;
      if (cudaEventElapsedTime(&a, ctx->ev[0], ctx->ev[1]) == cudaSuccess &&
          cudaEventElapsedTime(&b, ctx->ev[2], ctx->ev[3]) == cudaSuccess &&
          cudaEventElapsedTime(&c, ctx->ev[3], ctx->ev[4]) == cudaSuccess) {
        ctx->pf.col_ms += a;
        ctx->pf.col_samples += 1;
        ctx->pf.xb_ms += b;
        ctx->pf.xb_samples += 1;
        if (!tc) {  // the tensor-core path has no separate vector kernel
          ctx->pf.vec_ms += c;
          ctx->pf.vec_samples += 1;
        }
      } else {
        cudaGetLastError();
      }
    }
    if (*hdone >= nb) break;
    if (E.deadline_ms > 0 && now_ms() > E.deadline_ms) {
      timed_out = true;
      break;
    }
    if (l > max_launch) {
      rc = fail(ctx, FSQR_ECUDA, "iteration did not stop after %d steps", host_base);
      break;
    }
  }
  cudaGraphExecDestroy(exec);
  if (rc != FSQR_OK) return rc;
  if (tc) {
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (herr != 0)
      return fail(ctx, FSQR_ECUDA, "tensor-core column pass: a pipeline wait ran out of time (code %d)", herr);
  }
  {
    // iterations actually taken by the live fits (done fits idle afterwards)
    int hd0[kMaxNB];
    CK(cudaMemcpyAsync(hd0, F.done, sizeof(int) * NB, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int kmax = 0;
    for (int b = 0; b < nb; ++b) kmax = std::max(kmax, hd0[b] >= 0 ? hd0[b] : host_base);
    ctx->pf.iterations += kmax;
    // algorithmic bytes of one column pass: the stored X, the covariates,
    // beta^k read and beta^{k+1} written for the NB interleaved fits
    const int64_t xbytes = (X.fmt == FSQR_DENSE_F64 ? 8 * n : X.fmt == FSQR_INT8 ? n : (n + 3) / 4) * X.p;
    ctx->pf.col_bytes = xbytes + 8 * n * X.c + 2 * 8 * P * NB;
  }

  // ---- results
  int hd[kMaxNB];
  double rep[kMaxNB * kReport];
  CK(cudaMemcpyAsync(hd, F.done, sizeof(int) * NB, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(rep, F.report, sizeof(double) * NB * kReport, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int b = 0; b < nb; ++b) {
    const int k_fin = (hd[b] >= 0) ? hd[b] : host_base;
    const int f = gs.fit[b];
    LK(launch_unpack(F.beta[k_fin & 1] + b, E.beta + (int64_t)f * P, P, P, 1, NB, st));
    LK(launch_unpack(F.z + b, E.z + (int64_t)f * n, n, n, 1, NB, st));
    LK(launch_unpack(F.theta + b, E.theta + (int64_t)f * n, n, n, 1, NB, st));
  }
  const double t_solve = now_ms() - t0;

  if (E.infos) {
    // primal value, active count and duality gap of each returned iterate
    double *bfin, *tc, *tcs, *schk, *summ, *dtaus, *dlams;
    TRY(wsget(ctx, "r_bfin", (size_t)P * NB, &bfin));
    TRY(wsget(ctx, "r_tc", (size_t)npad * NB, &tc));
    TRY(wsget(ctx, "r_tcs", kMaxNB, &tcs));
    TRY(wsget(ctx, "r_schk", (size_t)P * NB, &schk));
    TRY(wsget(ctx, "r_summ", (size_t)kMaxNB * 8, &summ));
    TRY(wsget(ctx, "r_taus", kMaxNB, &dtaus));
    TRY(wsget(ctx, "r_lams", kMaxNB, &dlams));
    CK(cudaMemsetAsync(bfin, 0, sizeof(double) * P * NB, st));
    for (int b = 0; b < nb; ++b)
      LK(launch_pack(E.beta + (int64_t)gs.fit[b] * P, P, bfin + b, P, 1, NB, P, st));
    CK(cudaMemcpyAsync(dtaus, F.tau, sizeof(double) * kMaxNB, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dlams, F.lam, sizeof(double) * kMaxNB, cudaMemcpyHostToDevice, st));
    const double *schk_use = nullptr, *tc_use = nullptr;
    if (E.gap_defined) {
      LK(launch_dual_point(NB, F.theta, n, npad, dtaus, nb, tc, tcs, st));
      Fits Fx = F;
      LK(launch_col_pass(A_XT, NB, X, Fx, 0, tc, tcs, schk, nullptr, st));
      schk_use = schk;
      tc_use = tc;
    }
    LK(launch_summary(NB, nb, n, P, E.y, F.z, F.r, bfin, E.omega, dtaus, dlams, schk_use, tc_use,
                      summ, st));
    double hs[kMaxNB * 8];
    CK(cudaMemcpyAsync(hs, summ, sizeof(double) * kMaxNB * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int b = 0; b < nb; ++b) {
      fsqr_info &I = E.infos[gs.fit[b]];
      const double *rp = rep + b * kReport;
      I.status = timed_out && hd[b] < 0 ? FSQR_ETIMEOUT : (int)rp[5];
      I.iters = hd[b] >= 0 ? hd[b] : host_base;
      I.kkt = rp[0];
      I.r_p = rp[1];
      I.r_z = rp[2];
      I.r_beta = rp[3];
      I.r_1 = rp[4];
      I.primal = hs[b * 8 + 0] + hs[b * 8 + 1];
      I.active = (int64_t)hs[b * 8 + 2];
      if (E.gap_defined) {
        I.dual = hs[b * 8 + 3] * hs[b * 8 + 4];
        I.gap = (I.primal - I.dual) / (1.0 + fabs(I.primal) + fabs(I.dual));
      } else {
        I.dual = NAN;
        I.gap = NAN;
      }
      I.lambda = gs.lam[b];
      I.lambda_max = gs.lamnorm[b];
      I.mu = E.mu;
      I.t_solve_ms = t_solve;
    }
  } else {
    CK(cudaStreamSynchronize(st));
  }
  return timed_out ? FSQR_ETIMEOUT : FSQR_OK;
}

int warm_start_impl(fsqr_ctx *ctx, const Prep &pr, const double *y, double tau, double frac,
                    const double *omega, const float *params, double ysd, double *beta, double *z,
                    double *theta);

// Autotuner of the fits advanced together per X pass (opts.max_group = 0).
// For each candidate g (1, 2, 3, 4 and min(B, 8), up to B), the first g
// fits run cold for I1 and then I2 iterations; the difference of the two
// wall times over I2 - I1 is the time per iteration t(g) without the set-up,
// and the g with the least ceil(B / g) t(g) is chosen. The integer and FP64
// results do not depend on g. The users' arrays of those fits are saved and
// restored around the runs; the choice is cached per context and shape.
int tune_group(fsqr_ctx *ctx, const SolveEnv &E, int B, int n_lambda, const double *taus,
               const double *lambdas, const std::vector<double> &lmax, int *out) {
  const Dsg &X = E.pr->X;
  const fsqr_opts *o = E.o;
  char key[160];
  snprintf(key, sizeof key, "%lld/%lld/%lld/%d/%d/%d/%d/%d", (long long)X.n, (long long)X.p, (long long)X.c,
           X.fmt, o->precision, o->digits, B, o->warm);
  auto it = ctx->tuned.find(key);
  if (it != ctx->tuned.end()) {
    *out = it->second;
    ctx->pf.tuned_group = it->second;
    return FSQR_OK;
  }
  std::vector<int> cand;
  for (int g : {1, 2, 3, 4, std::min(B, kMaxNB)})
    if (g <= B && (cand.empty() || g > cand.back())) cand.push_back(g);
  const int gmax = cand.back();
  if (cand.size() == 1) {
    *out = gmax;
    ctx->pf.tuned_group = gmax;
    return FSQR_OK;
  }
  const int64_t P = X.P, n = X.n;
  // save the first gmax fits' arrays (starts of FSQR_WARM_GIVEN / LEARNED)
  double *sv_b, *sv_z, *sv_t;
  TRY(wsget(ctx, "tune_b", (size_t)(gmax * P), &sv_b));
  TRY(wsget(ctx, "tune_z", (size_t)(gmax * n), &sv_z));
  TRY(wsget(ctx, "tune_t", (size_t)(gmax * n), &sv_t));
  cudaStream_t st = ctx->stream;
  CK(cudaMemcpyAsync(sv_b, E.beta, sizeof(double) * gmax * P, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(sv_z, E.z, sizeof(double) * gmax * n, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(sv_t, E.theta, sizeof(double) * gmax * n, cudaMemcpyDeviceToDevice, st));
  std::vector<fsqr_info> scratch((size_t)B);
  fsqr_opts tmp = *o;
  tmp.tol = 0.0;
  tmp.timeout_ms = 0;
  SolveEnv E2 = E;
  E2.o = &tmp;
  E2.infos = scratch.data();
  E2.deadline_ms = 0.0;
  const int K = std::max(1, o->check_every);
  const int I1 = K * std::max(1, 20 / K), I2 = I1 + K * std::max(1, 80 / K);
  double best = 0.0;
  int bestg = cand[0];
  const fsqr_profile keep = ctx->pf;
  for (int g : cand) {
    GroupSpec gs{};
    gs.nb = g;
    for (int q = 0; q < g; ++q) {
      const int t = q / n_lambda;
      gs.tau[q] = taus[t];
      gs.lam[q] = lambdas[q];
      gs.lamnorm[q] = lmax[t] > 0.0 ? lmax[t] : 1.0;
      gs.fit[q] = q;
      gs.src_fit[q] = -1;
    }
    double w[2];
    for (int r = 0; r < 2; ++r) {
      tmp.max_iter = r == 0 ? I1 : I2;
      CK(cudaStreamSynchronize(st));
      const double t0 = now_ms();
      TRY(solve_group(ctx, E2, gs));
      CK(cudaStreamSynchronize(st));
      w[r] = now_ms() - t0;
    }
    const double per_iter = std::max(w[1] - w[0], 1e-6) / (double)(I2 - I1);
    const double cost = (double)((B + g - 1) / g) * per_iter;
    if (g == cand[0] || cost < best) { best = cost; bestg = g; }
  }
  // the timing runs' kernels count as launches; their samples do not enter the profile
  const int64_t launches = ctx->pf.kernel_launches;
  ctx->pf = keep;
  ctx->pf.kernel_launches = launches;
  CK(cudaMemcpyAsync(E.beta, sv_b, sizeof(double) * gmax * P, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(E.z, sv_z, sizeof(double) * gmax * n, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(E.theta, sv_t, sizeof(double) * gmax * n, cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  ctx->tuned[key] = bestg;
  ctx->pf.tuned_group = bestg;
  *out = bestg;
  return FSQR_OK;
}

int fit_batch_impl(fsqr_ctx *ctx, const fsqr_design *Xd, const double *y, int n_tau,
                   const double *taus, int n_lambda, const double *lambdas, const double *omega,
                   const int64_t *block_ptr, int G, const fsqr_opts *opts, double *beta, double *z,
                   double *theta, fsqr_info *infos) {
  const double t0 = now_ms();
  TRY(check_opts(ctx, opts, G));
  if (n_tau < 1 || n_lambda < 1) return fail(ctx, FSQR_EINVAL, "n_tau and n_lambda must be >= 1");
  if (!taus || !lambdas) return fail(ctx, FSQR_EINVAL, "taus/lambdas are NULL");
  if (!y || !omega || !beta || !z || !theta) return fail(ctx, FSQR_EINVAL, "NULL array argument");
  for (int t = 0; t < n_tau; ++t)
    if (!(taus[t] > 0.0 && taus[t] < 1.0)) return fail(ctx, FSQR_EINVAL, "tau must be in (0,1)");
  for (int t = 0; t < n_tau * n_lambda; ++t)
    if (!(lambdas[t] >= 0.0) || isinf(lambdas[t]))
      return fail(ctx, FSQR_EINVAL, "lambda must be finite and >= 0");
  if (opts->precision != FSQR_FP64 && Xd && Xd->geno_format != FSQR_INT8)
    return fail(ctx, FSQR_EINVAL, "mixed precision needs FSQR_INT8 genotype storage");
  Prep pr;
  TRY(prepare(ctx, Xd, &pr, opts->precision != FSQR_FP64));
  const Dsg &X = pr.X;
  const int64_t P = X.P, n = X.n;
  TRY(check_blocks(ctx, block_ptr, G, P));
  // omega: omega[0] == 0, omega >= 0; gap defined iff omega_j > 0 for j >= 1
  double om[2];
  {
    double *d;
    TRY(wsget(ctx, "omega_chk", 2, &d));
    CK(cudaMemcpyAsync(d, omega, sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    LK(launch_min_omega(omega, P, d + 1, ctx->stream));
    CK(cudaMemcpyAsync(om, d, sizeof om, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  if (om[0] != 0.0) return fail(ctx, FSQR_EINVAL, "omega[0] must be 0 (intercept unpenalised)");
  if (P > 1 && !(om[1] >= 0.0)) return fail(ctx, FSQR_EINVAL, "omega must be >= 0");
  double ymax, ysd;
  TRY(y_stats(ctx, y, n, &ymax, &ysd));
  const double mu = opts->mu > 0.0 ? opts->mu : 1.0 / ((double)n * (ysd > 0.0 ? ysd : 1.0));
  std::vector<double> eta(G);
  if (opts->eta) {
    for (int g = 0; g < G; ++g) eta[g] = opts->eta[g];
  } else {
    TRY(eta_impl(ctx, pr, block_ptr, G, mu, opts->eta_margin, opts->power_iters, opts->power_tol,
                 eta.data()));
  }
  std::vector<double> lmax(n_tau);
  for (int t = 0; t < n_tau; ++t) TRY(lambda_max_impl(ctx, pr, y, taus[t], omega, &lmax[t]));
  if (opts->warm == FSQR_WARM_LEARNED)
    for (int t = 0; t < n_tau; ++t)
      for (int l = 0; l < n_lambda; ++l) {
        const int f = t * n_lambda + l;
        const double frac = lmax[t] > 0.0 ? lambdas[f] / lmax[t] : 1.0;
        TRY(warm_start_impl(ctx, pr, y, taus[t], frac, omega, opts->warm_params, ysd, beta + (int64_t)f * P,
                            z + (int64_t)f * n, theta + (int64_t)f * n));
      }

  SolveEnv E{};
  E.pr = &pr;
  E.y = y;
  E.omega = omega;
  E.G = G;
  E.mu = mu;
  E.ymax = ymax;
  E.gap_defined = (P == 1) || (om[1] > 0.0);
  E.o = opts;
  E.beta = beta;
  E.z = z;
  E.theta = theta;
  E.infos = infos;
  E.deadline_ms = opts->timeout_ms > 0 ? t0 + (double)opts->timeout_ms : 0.0;
  TRY(wsget(ctx, "eta", G, &E.d_eta));
  TRY(wsget(ctx, "ieta", G, &E.d_ieta));
  TRY(wsget(ctx, "bp", (size_t)G + 1, &E.d_bp));
  std::vector<double> ieta(G);
  for (int g = 0; g < G; ++g) ieta[g] = 1.0 / eta[g];
  CK(cudaMemcpyAsync(E.d_eta, eta.data(), G * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(E.d_ieta, ieta.data(), G * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(E.d_bp, block_ptr, (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
  const double t_setup = now_ms() - t0;

  // groups of fits
  const int B = n_tau * n_lambda;
  int mg = opts->max_group;
  if (mg == 0) TRY(tune_group(ctx, E, B, n_lambda, taus, lambdas, lmax, &mg));
  std::vector<GroupSpec> groups;
  if (opts->warm == FSQR_WARM_PATH) {
    for (int l = 0; l < n_lambda; ++l)
      for (int t0g = 0; t0g < n_tau; t0g += mg) {
        GroupSpec gs{};
        gs.nb = std::min(mg, n_tau - t0g);
        for (int q = 0; q < gs.nb; ++q) {
          const int t = t0g + q, f = t * n_lambda + l;
          gs.tau[q] = taus[t];
          gs.lam[q] = lambdas[f];
          gs.lamnorm[q] = lmax[t] > 0.0 ? lmax[t] : 1.0;
          gs.fit[q] = f;
          gs.src_fit[q] = (l == 0) ? -1 : f - 1;
        }
        groups.push_back(gs);
      }
  } else {
    for (int f0 = 0; f0 < B; f0 += mg) {
      GroupSpec gs{};
      gs.nb = std::min(mg, B - f0);
      for (int q = 0; q < gs.nb; ++q) {
        const int f = f0 + q, t = f / n_lambda;
        gs.tau[q] = taus[t];
        gs.lam[q] = lambdas[f];
        gs.lamnorm[q] = lmax[t] > 0.0 ? lmax[t] : 1.0;
        gs.fit[q] = f;
        gs.src_fit[q] = (opts->warm == FSQR_WARM_GIVEN || opts->warm == FSQR_WARM_LEARNED) ? f : -1;
      }
      groups.push_back(gs);
    }
  }
  int worst = FSQR_OK;
  for (const GroupSpec &gs : groups) {
    int rc = solve_group(ctx, E, gs);
    if (rc != FSQR_OK && rc != FSQR_ETIMEOUT) return rc;
    if (rc == FSQR_ETIMEOUT) E.deadline_ms = 1.0;  // later groups stop right away
  }
  if (infos)
    for (int f = 0; f < B; ++f) {
      infos[f].t_setup_ms = t_setup;
      if (worst == FSQR_OK && infos[f].status != FSQR_OK) worst = infos[f].status;
    }
  return worst;
}

// out[b*n + i] = x~_i^T beta_b for B coefficient vectors (FP64 path).
int predict_impl(fsqr_ctx *ctx, const Prep &pr, const double *beta, int B, double *out) {
  const Dsg &X = pr.X;
  const int64_t n = X.n, npad = pad16(n), P = X.P;
  cudaStream_t st = ctx->stream;
  Fits F = pass_fits(ctx, X);
  TRY(wsget(ctx, "p_xbpart", (size_t)kBMaxSplits * npad * kMaxNB, &F.xb_part));
  TRY(wsget(ctx, "p_arb", (size_t)F.gridA * kMaxNB, &F.a_rb));
  TRY(wsget(ctx, "p_act", (size_t)F.gridA * kMaxNB, &F.a_ct));
  TRY(wsget(ctx, "p_acnt", (size_t)F.gridA, &F.a_cnt));
  TRY(wsget(ctx, "p_alist", (size_t)F.gridA * F.T, &F.a_list));
  TRY(wsget(ctx, "p_metai", 4, &F.meta_i));
  TRY(wsget(ctx, "p_metad", 2 * kMaxNB, &F.meta_d));
  TRY(alloc_totals(ctx, F, "p"));
  int *done;
  TRY(wsget(ctx, "p_done", kMaxNB, &done));
  F.done = done;
  CK(cudaMemsetAsync(done, 0xff, sizeof(int) * kMaxNB, st));
  double *bg;
  TRY(wsget(ctx, "p_bg", (size_t)P * kMaxNB, &bg));
  CK(cudaMemsetAsync(bg, 0, sizeof(double) * P * kMaxNB, st));
  for (int b0 = 0; b0 < B; b0 += kMaxNB) {
    const int nb = std::min(kMaxNB, B - b0);
    const int NB = nb_template(nb);
    F.nb = nb;
    LK(launch_pack(beta + (int64_t)b0 * P, P, bg, P, nb, NB, P, st));
    LK(launch_col_pass(A_LIST, NB, X, F, 0, nullptr, nullptr, nullptr, bg, st));
    LK(launch_xbeta(NB, X, F, 0, bg, st));
    LK(launch_gather_xb(NB, F, out + (int64_t)b0 * n, n, nb, st));
  }
  CK(cudaStreamSynchronize(st));
  return FSQR_OK;
}

}  // namespace

// ================================================================ C ABI

extern "C" {

int fsqr_version(void) { return kVersion; }

void fsqr_opts_default(fsqr_opts *o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->tol = 1e-6;
  o->max_iter = 100000;
  o->check_every = 10;
  o->mu = 0.0;
  o->eta = nullptr;
  o->eta_margin = 0.05;
  o->power_iters = 100;
  o->power_tol = 1e-6;
  o->precision = FSQR_FP64;
  o->warm = FSQR_WARM_NONE;
  o->digits = 4;
  o->max_group = 4;
  o->timeout_ms = 0;
}

int fsqr_create(fsqr_ctx **out, int device, void *cuda_stream) {
  if (!out) return FSQR_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return FSQR_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return FSQR_ECUDA;
  fsqr_ctx *ctx = new fsqr_ctx();
  ctx->device = device;
  if (cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return FSQR_ECUDA;
    }
    ctx->own_stream = true;
  }
  if (cudaEventCreateWithFlags(&ctx->legacy_ev, cudaEventDisableTiming) != cudaSuccess) {
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return FSQR_ECUDA;
  }
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (ctx->num_sms <= 0) ctx->num_sms = 1;
  *out = ctx;
  return FSQR_OK;
}

int fsqr_destroy(fsqr_ctx *ctx) {
  if (!ctx) return FSQR_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto &kv : ctx->ws)
    if (kv.second.first) cudaFree(kv.second.first);
  if (ctx->hpin) cudaFreeHost(ctx->hpin);
  for (int e = 0; e < 6; ++e)
    if (ctx->ev[e]) cudaEventDestroy(ctx->ev[e]);
  if (ctx->legacy_ev) cudaEventDestroy(ctx->legacy_ev);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return FSQR_OK;
}

const char *fsqr_last_error(const fsqr_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int fsqr_col_stats(fsqr_ctx *ctx, const fsqr_design *X, double *mean_out, double *sd_out) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  if (!mean_out || !sd_out) return fail(ctx, FSQR_EINVAL, "NULL output");
  Prep pr;
  TRY(prepare(ctx, X, &pr, false));
  const int64_t F = X->c + X->p;
  if (F > 0) {
    CK(cudaMemcpyAsync(mean_out, pr.mean, F * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(sd_out, pr.sd, F * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return FSQR_OK;
}

int fsqr_lambda_max(fsqr_ctx *ctx, const fsqr_design *X, const double *y, double tau,
                    const double *omega, double *out) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  if (!y || !omega || !out) return fail(ctx, FSQR_EINVAL, "NULL argument");
  if (!(tau > 0.0 && tau < 1.0)) return fail(ctx, FSQR_EINVAL, "tau must be in (0,1)");
  Prep pr;
  TRY(prepare(ctx, X, &pr, false));
  return lambda_max_impl(ctx, pr, y, tau, omega, out);
}

int fsqr_eta(fsqr_ctx *ctx, const fsqr_design *X, const int64_t *block_ptr, int G, double mu,
             double margin, int max_iter, double tol, double *eta_out) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  if (!eta_out) return fail(ctx, FSQR_EINVAL, "NULL output");
  if (!(mu > 0.0)) return fail(ctx, FSQR_EINVAL, "mu must be > 0");
  if (!(margin >= 0.0) || max_iter < 1 || !(tol >= 0.0))
    return fail(ctx, FSQR_EINVAL, "bad margin/max_iter/tol");
  Prep pr;
  TRY(prepare(ctx, X, &pr, false));
  TRY(check_blocks(ctx, block_ptr, G, pr.X.P));
  return eta_impl(ctx, pr, block_ptr, G, mu, margin, max_iter, tol, eta_out);
}

int fsqr_fit_batch(fsqr_ctx *ctx, const fsqr_design *X, const double *y, int n_tau,
                   const double *taus, int n_lambda, const double *lambdas, const double *omega,
                   const int64_t *block_ptr, int G, const fsqr_opts *opts, double *beta, double *z,
                   double *theta, fsqr_info *infos) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  std::vector<fsqr_info> local;
  if (!infos) {
    local.resize((size_t)std::max(1, n_tau * n_lambda));
    infos = local.data();
  }
  memset(infos, 0, sizeof(fsqr_info) * (size_t)std::max(0, n_tau * n_lambda));
  return fit_batch_impl(ctx, X, y, n_tau, taus, n_lambda, lambdas, omega, block_ptr, G, opts,
                        beta, z, theta, infos);
}

int fsqr_fit(fsqr_ctx *ctx, const fsqr_design *X, const double *y, double tau, double lambda,
             const double *omega, const int64_t *block_ptr, int G, const fsqr_opts *opts,
             double *beta, double *z, double *theta, fsqr_info *info) {
  if (!ctx) return FSQR_EINVAL;
  if (opts && opts->warm == FSQR_WARM_PATH)
    return fail(ctx, FSQR_EINVAL, "FSQR_WARM_PATH applies to fsqr_fit_batch only");
  fsqr_info tmp;
  return fsqr_fit_batch(ctx, X, y, 1, &tau, 1, &lambda, omega, block_ptr, G, opts, beta, z, theta,
                        info ? info : &tmp);
}

int fsqr_fit_batch_host(fsqr_ctx *ctx, const fsqr_design *X, const double *y, int n_tau,
                        const double *taus, int n_lambda, const double *lambdas,
                        const double *omega, const int64_t *block_ptr, int G,
                        const fsqr_opts *opts, double *beta, double *z, double *theta,
                        fsqr_info *infos) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  TRY(check_design(ctx, X));
  if (!y || !omega || !beta || !z || !theta || n_tau < 1 || n_lambda < 1)
    return fail(ctx, FSQR_EINVAL, "NULL array argument or empty grid");
  const int64_t n = X->n, P = 1 + X->c + X->p, F = X->c + X->p;
  const int64_t B = (int64_t)n_tau * n_lambda;
  cudaStream_t st = ctx->stream;
  fsqr_design D = *X;
  uint8_t *dg = nullptr;
  double *dc = nullptr, *dm = nullptr, *ds = nullptr, *dy, *dom, *db, *dz, *dt;
  if (X->p > 0) {
    TRY(wsget(ctx, "h_geno", (size_t)(X->p * X->geno_ld), &dg));
    CK(cudaMemcpyAsync(dg, X->geno, (size_t)(X->p * X->geno_ld), cudaMemcpyHostToDevice, st));
  }
  if (X->c > 0) {
    TRY(wsget(ctx, "h_cov", (size_t)(X->c * n), &dc));
    CK(cudaMemcpyAsync(dc, X->cov, (size_t)(X->c * n) * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  if (X->col_mean) {
    TRY(wsget(ctx, "h_mean", (size_t)F, &dm));
    TRY(wsget(ctx, "h_sd", (size_t)F, &ds));
    CK(cudaMemcpyAsync(dm, X->col_mean, F * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ds, X->col_sd, F * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  TRY(wsget(ctx, "h_y", (size_t)n, &dy));
  TRY(wsget(ctx, "h_omega", (size_t)P, &dom));
  TRY(wsget(ctx, "h_beta", (size_t)(B * P), &db));
  TRY(wsget(ctx, "h_z", (size_t)(B * n), &dz));
  TRY(wsget(ctx, "h_theta", (size_t)(B * n), &dt));
  CK(cudaMemcpyAsync(dy, y, n * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dom, omega, P * sizeof(double), cudaMemcpyHostToDevice, st));
  if (opts && opts->warm == FSQR_WARM_GIVEN) {
    CK(cudaMemcpyAsync(db, beta, B * P * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dz, z, B * n * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dt, theta, B * n * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  D.geno = dg;
  D.cov = dc;
  D.col_mean = dm;
  D.col_sd = ds;
  int rc = fsqr_fit_batch(ctx, &D, dy, n_tau, taus, n_lambda, lambdas, dom, block_ptr, G, opts, db,
                          dz, dt, infos);
  if (rc != FSQR_OK && rc != FSQR_ENOCONV && rc != FSQR_ETIMEOUT) return rc;
  CK(cudaMemcpyAsync(beta, db, B * P * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(z, dz, B * n * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(theta, dt, B * n * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return rc;
}

int fsqr_kkt(fsqr_ctx *ctx, const fsqr_design *Xd, const double *y, double tau, double lambda,
             const double *omega, double lambda_norm, const double *beta, const double *z,
             const double *theta, fsqr_info *out) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  if (!y || !omega || !beta || !z || !theta || !out) return fail(ctx, FSQR_EINVAL, "NULL argument");
  if (!(tau > 0.0 && tau < 1.0) || !(lambda >= 0.0) || !(lambda_norm > 0.0))
    return fail(ctx, FSQR_EINVAL, "bad tau/lambda/lambda_norm");
  Prep pr;
  TRY(prepare(ctx, Xd, &pr, false));
  const Dsg &X = pr.X;
  const int64_t n = X.n, npad = pad16(n), P = X.P;
  cudaStream_t st = ctx->stream;
  Fits F = pass_fits(ctx, X);
  F.nb = 1;
  double *xb, *th, *ths, *s, *o4, *tc, *tcs, *schk, *summ, *dt, *dl, *om;
  TRY(wsget(ctx, "k_xbpart", (size_t)kBMaxSplits * npad, &F.xb_part));
  TRY(wsget(ctx, "k_arb", (size_t)F.gridA, &F.a_rb));
  TRY(wsget(ctx, "k_act", (size_t)F.gridA, &F.a_ct));
  TRY(wsget(ctx, "k_acnt", (size_t)F.gridA, &F.a_cnt));
  TRY(wsget(ctx, "k_alist", (size_t)F.gridA * F.T, &F.a_list));
  TRY(wsget(ctx, "k_metai", 4, &F.meta_i));
  TRY(wsget(ctx, "k_metad", 2 * kMaxNB, &F.meta_d));
  TRY(alloc_totals(ctx, F, "k"));
  int *done;
  TRY(wsget(ctx, "k_done", kMaxNB, &done));
  F.done = done;
  CK(cudaMemsetAsync(done, 0xff, sizeof(int) * kMaxNB, st));
  TRY(wsget(ctx, "k_xb", (size_t)npad, &xb));
  TRY(wsget(ctx, "k_th", (size_t)npad, &th));
  TRY(wsget(ctx, "k_ths", 1, &ths));
  TRY(wsget(ctx, "k_s", (size_t)P, &s));
  TRY(wsget(ctx, "k_o4", 4, &o4));
  TRY(wsget(ctx, "k_tc", (size_t)npad, &tc));
  TRY(wsget(ctx, "k_tcs", 1, &tcs));
  TRY(wsget(ctx, "k_schk", (size_t)P, &schk));
  TRY(wsget(ctx, "k_summ", 8, &summ));
  TRY(wsget(ctx, "k_tau", 1, &dt));
  TRY(wsget(ctx, "k_lam", 1, &dl));
  TRY(wsget(ctx, "k_om", 2, &om));
  // X~ beta
  LK(launch_col_pass(A_LIST, 1, X, F, 0, nullptr, nullptr, nullptr, beta, st));
  LK(launch_xbeta(1, X, F, 0, beta, st));
  LK(launch_gather_xb(1, F, xb, npad, 1, st));
  // s = X~^T theta (padded copy of theta)
  LK(launch_pack(theta, n, th, n, 1, 1, npad, st));
  LK(launch_sum_cols(th, n, npad, 1, ths, nullptr, st));
  LK(launch_col_pass(A_XT, 1, X, F, 0, th, ths, s, nullptr, st));
  LK(launch_kkt_given(n, P, y, xb, z, theta, s, beta, omega, tau, lambda, o4, st));
  CK(cudaMemcpyAsync(dt, &tau, sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dl, &lambda, sizeof(double), cudaMemcpyHostToDevice, st));
  LK(launch_min_omega(omega, P, om, st));
  double hom = 0.0, h4[4];
  CK(cudaMemcpyAsync(&hom, om, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h4, o4, sizeof h4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  // the summary kernel's loss uses z - r = y - X~ beta; passing y for z and
  // X~ beta for r gives the primal loss of beta
  double *ypad;
  TRY(wsget(ctx, "k_ypad", (size_t)npad, &ypad));
  LK(launch_pack(y, n, ypad, n, 1, 1, npad, st));
  const bool gap_def = (P == 1) || (hom > 0.0);
  const double *schk_use = nullptr, *tc_use = nullptr;
  if (gap_def) {
    LK(launch_dual_point(1, th, n, npad, dt, 1, tc, tcs, st));
    LK(launch_col_pass(A_XT, 1, X, F, 0, tc, tcs, schk, nullptr, st));
    schk_use = schk;
    tc_use = tc;
  }
  LK(launch_summary(1, 1, n, P, y, ypad, xb, beta, omega, dt, dl, schk_use, tc_use, summ, st));
  double hs[8];
  CK(cudaMemcpyAsync(hs, summ, sizeof hs, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  memset(out, 0, sizeof *out);
  out->r_p = h4[0];
  out->r_z = h4[1];
  out->r_beta = h4[2] / lambda_norm;
  out->r_1 = h4[3];
  out->kkt = std::max(std::max(out->r_p, out->r_z), std::max(out->r_beta, out->r_1));
  out->primal = hs[0] + hs[1];
  out->active = (int64_t)hs[2];
  if (gap_def) {
    out->dual = hs[3] * hs[4];
    out->gap = (out->primal - out->dual) / (1.0 + fabs(out->primal) + fabs(out->dual));
  } else {
    out->dual = NAN;
    out->gap = NAN;
  }
  out->lambda = lambda;
  out->lambda_max = lambda_norm;
  out->status = FSQR_OK;
  return FSQR_OK;
}

int fsqr_predict(fsqr_ctx *ctx, const fsqr_design *Xd, const double *beta, int B, double *out) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  if (!beta || !out || B < 0) return fail(ctx, FSQR_EINVAL, "bad arguments");
  if (B == 0) return FSQR_OK;
  Prep pr;
  TRY(prepare(ctx, Xd, &pr, false));
  return predict_impl(ctx, pr, beta, B, out);
}

int fsqr_profile_enable(fsqr_ctx *ctx, int on) {
  if (!ctx) return FSQR_EINVAL;
  ctx->prof = on != 0;
  return FSQR_OK;
}

int fsqr_profile_get(fsqr_ctx *ctx, fsqr_profile *out) {
  if (!ctx || !out) return FSQR_EINVAL;
  *out = ctx->pf;
  return FSQR_OK;
}

int fsqr_profile_reset(fsqr_ctx *ctx) {
  if (!ctx) return FSQR_EINVAL;
  ctx->pf = fsqr_profile{};
  return FSQR_OK;
}

int fsqr_back_transform(fsqr_ctx *ctx, const fsqr_design *Xd, const double *beta_std, int B,
                        double *beta_out) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  if (!beta_std || !beta_out || B < 0) return fail(ctx, FSQR_EINVAL, "bad arguments");
  Prep pr;
  TRY(prepare(ctx, Xd, &pr, false));
  LK(launch_back_transform(pr.X, beta_std, B, beta_out, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FSQR_OK;
}

}  // extern "C"

// ---- learned warm start ------------------------------------------------------

namespace {

// Work buffers of the network for `rows` inputs at a time.
struct MlpWs {
  float *H[kMlpLayers - 1];
  float *G0, *G1, *f, *g;
};

int mlp_ws(fsqr_ctx *ctx, int64_t rows, MlpWs *w) {
  const size_t hid = (size_t)rows * kMlpHidden;
  TRY(wsget(ctx, "mlp_h0", hid, &w->H[0]));
  TRY(wsget(ctx, "mlp_h1", hid, &w->H[1]));
  TRY(wsget(ctx, "mlp_h2", hid, &w->H[2]));
  TRY(wsget(ctx, "mlp_g0", hid, &w->G0));
  TRY(wsget(ctx, "mlp_g1", hid, &w->G1));
  TRY(wsget(ctx, "mlp_f", (size_t)rows, &w->f));
  TRY(wsget(ctx, "mlp_g", (size_t)rows, &w->g));
  return FSQR_OK;
}

constexpr int64_t kMlpChunk = 32768;  // inference rows per forward pass

int mlp_forward_chunked(fsqr_ctx *ctx, const float *params, const float *x, int64_t rows, float *out) {
  MlpWs w;
  TRY(mlp_ws(ctx, std::min(rows, kMlpChunk), &w));
  for (int64_t r0 = 0; r0 < rows; r0 += kMlpChunk) {
    const int64_t nr = std::min(kMlpChunk, rows - r0);
    LK(mlp_forward(params, x + r0 * kMlpIn, nr, w.H, out + r0, ctx->stream));
  }
  return FSQR_OK;
}

// The inputs u of every feature column of one fit (device, (P-1) x 3), with
// the lambda_max pieces left on the device.
int warm_features_impl(fsqr_ctx *ctx, const Prep &pr, const double *y, double tau, double frac,
                       const double *omega, float *u, LmaxDev *L) {
  TRY(lambda_max_dev(ctx, pr, y, tau, omega, L));
  LK(launch_warm_features(L->s, pr.X.P, pr.X.n, tau, frac, L->o, u, ctx->stream));
  return FSQR_OK;
}

// The start the network proposes for (tau, frac * lambda_max(tau)): beta (P),
// z (n), theta (n) on the device; ysd = sd(y).
int warm_start_impl(fsqr_ctx *ctx, const Prep &pr, const double *y, double tau, double frac,
                    const double *omega, const float *params, double ysd, double *beta, double *z,
                    double *theta) {
  const Dsg &X = pr.X;
  float *u, *f;
  double *xb;
  TRY(wsget(ctx, "warm_u", (size_t)std::max<int64_t>(1, X.P - 1) * kMlpIn, &u));
  TRY(wsget(ctx, "warm_f", (size_t)std::max<int64_t>(1, X.P - 1), &f));
  TRY(wsget(ctx, "warm_xb", (size_t)X.n, &xb));
  LmaxDev L;
  TRY(warm_features_impl(ctx, pr, y, tau, frac, omega, u, &L));
  if (X.P > 1) TRY(mlp_forward_chunked(ctx, params, u, X.P - 1, f));
  LK(launch_warm_beta(f, X.P, L.q, ysd, beta, ctx->stream));
  TRY(predict_impl(ctx, pr, beta, 1, xb));
  LK(launch_warm_dual(y, xb, X.n, tau, z, theta, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FSQR_OK;
}

int check_warm_args(fsqr_ctx *ctx, const double *y, double tau, double frac, const double *omega) {
  if (!y || !omega) return fail(ctx, FSQR_EINVAL, "NULL argument");
  if (!(tau > 0.0 && tau < 1.0)) return fail(ctx, FSQR_EINVAL, "tau must be in (0,1)");
  if (!(frac > 0.0)) return fail(ctx, FSQR_EINVAL, "lambda_frac must be > 0");
  return FSQR_OK;
}

}  // namespace

extern "C" {

int64_t fsqr_mlp_param_count(void) { return mlp_param_count(); }

int fsqr_mlp_init(fsqr_ctx *ctx, float *params, uint64_t seed) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  if (!params) return fail(ctx, FSQR_EINVAL, "NULL params");
  int *dd;
  TRY(wsget(ctx, "mlp_dims", kMlpLayers + 1, &dd));
  LK(mlp_init(params, dd, seed, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FSQR_OK;
}

int fsqr_mlp_forward(fsqr_ctx *ctx, const float *params, const float *x, int64_t rows, float *out) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  if (!params || !x || !out || rows < 0) return fail(ctx, FSQR_EINVAL, "bad arguments");
  if (rows == 0) return FSQR_OK;
  TRY(mlp_forward_chunked(ctx, params, x, rows, out));
  CK(cudaStreamSynchronize(ctx->stream));
  return FSQR_OK;
}

int fsqr_mlp_grad(fsqr_ctx *ctx, const float *params, const float *x, const float *t, const float *w,
                  int64_t rows, float *grad, double *loss) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  if (!params || !x || !t || !w || !grad || rows < 1) return fail(ctx, FSQR_EINVAL, "bad arguments");
  if (rows > (int64_t)1 << 24) return fail(ctx, FSQR_EINVAL, "rows > 2^24");
  MlpWs ws;
  TRY(mlp_ws(ctx, rows, &ws));
  double *dl;
  TRY(wsget(ctx, "mlp_loss", 1, &dl));
  LK(mlp_grad(params, x, t, w, rows, ws.H, ws.G0, ws.G1, ws.f, ws.g, grad, dl, ctx->stream));
  double hl = 0.0;
  CK(cudaMemcpyAsync(&hl, dl, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (loss) *loss = hl;
  return FSQR_OK;
}

int fsqr_mlp_train(fsqr_ctx *ctx, float *params, float *m, float *v, int64_t step0, const float *x,
                   const float *t, const float *w, int64_t rows, int steps, int batch, float lr,
                   uint64_t seed, double *losses) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  if (!params || !m || !v || !x || !t || !w || rows < 1 || steps < 0 || batch < 1 || step0 < 0 ||
      !(lr > 0.f))
    return fail(ctx, FSQR_EINVAL, "bad arguments");
  if (batch > (1 << 20)) return fail(ctx, FSQR_EINVAL, "batch > 2^20");
  if (steps == 0) return FSQR_OK;
  MlpWs ws;
  TRY(mlp_ws(ctx, batch, &ws));
  float *xb, *tb, *wb, *grad;
  double *dl;
  const int64_t count = mlp_param_count();
  TRY(wsget(ctx, "mlp_xb", (size_t)batch * kMlpIn, &xb));
  TRY(wsget(ctx, "mlp_tb", (size_t)batch, &tb));
  TRY(wsget(ctx, "mlp_wb", (size_t)batch, &wb));
  TRY(wsget(ctx, "mlp_grad", (size_t)count, &grad));
  TRY(wsget(ctx, "mlp_losses", (size_t)steps, &dl));
  cudaStream_t st = ctx->stream;
  for (int k = 0; k < steps; ++k) {
    const int64_t step = step0 + k + 1;
    LK(mlp_sample(x, t, w, rows, batch, seed, step, xb, tb, wb, st));
    LK(mlp_grad(params, xb, tb, wb, batch, ws.H, ws.G0, ws.G1, ws.f, ws.g, grad, dl + k, st));
    LK(mlp_adam(params, grad, m, v, count, step, lr, st));
  }
  if (losses) CK(cudaMemcpyAsync(losses, dl, sizeof(double) * steps, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return FSQR_OK;
}

int fsqr_warm_features(fsqr_ctx *ctx, const fsqr_design *Xd, const double *y, double tau, double lam_frac,
                       const double *omega, float *u, double *lambda_max) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  TRY(check_warm_args(ctx, y, tau, lam_frac, omega));
  if (!u) return fail(ctx, FSQR_EINVAL, "NULL output");
  Prep pr;
  TRY(prepare(ctx, Xd, &pr, false));
  LmaxDev L;
  TRY(warm_features_impl(ctx, pr, y, tau, lam_frac, omega, u, &L));
  double h = 0.0;
  CK(cudaMemcpyAsync(&h, L.o, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (lambda_max) *lambda_max = h;
  return FSQR_OK;
}

int fsqr_warm_start(fsqr_ctx *ctx, const fsqr_design *Xd, const double *y, double tau, double lam_frac,
                    const double *omega, const float *params, double *beta, double *z, double *theta) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  TRY(check_warm_args(ctx, y, tau, lam_frac, omega));
  if (!params || !beta || !z || !theta) return fail(ctx, FSQR_EINVAL, "NULL argument");
  Prep pr;
  TRY(prepare(ctx, Xd, &pr, false));
  double ymax = 0.0, ysd = 0.0;
  TRY(y_stats(ctx, y, pr.X.n, &ymax, &ysd));
  return warm_start_impl(ctx, pr, y, tau, lam_frac, omega, params, ysd, beta, z, theta);
}

}  // extern "C"

// ---- lambda_max without device allocation ----------------------------------
//
// fsqr_lambda_max takes its buffers from the context's workspace, which grows
// by cudaMalloc on first use. Some callers cannot allocate at call time: a
// serving process whose device memory is reserved up front by its own pool
// (a caching allocator holding all free HBM), or one that cannot accept the
// device-wide synchronisation that cudaMalloc/cudaFree imply. For them the
// variant below runs the same kernels in the same order on buffers carved
// from one static device array that is part of the library image.

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[FSQR_NOALLOC_SCRATCH_BYTES];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoAllocMaxDevices] = {};

// Address of this device's copy of the array, looked up once per device with
// that device current (the caller has selected it).
int noalloc_base(fsqr_ctx *ctx, unsigned char **out) {
  if (ctx->device < 0 || ctx->device >= kNoAllocMaxDevices)
    return fail(ctx, FSQR_EINVAL, "device %d >= %d", ctx->device, kNoAllocMaxDevices);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[ctx->device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fail(ctx, FSQR_ECUDA, "cudaGetSymbolAddress of the static scratch: %s",
                  cudaGetErrorString(e));
    }
    g_noalloc_addr[ctx->device] = p;
  }
  *out = static_cast<unsigned char *>(g_noalloc_addr[ctx->device]);
  return FSQR_OK;
}

// Bump carving in 256-byte steps; with base == nullptr it only counts bytes.
struct Carve {
  unsigned char *base;
  size_t off = 0;
  template <class T>
  T *take(size_t count) {
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += (std::max<size_t>(count * sizeof(T), 1) + 255) / 256 * 256;
    return p;
  }
};

struct NoAllocBufs {
  double *mean, *sd, *a, *b, *q, *v, *vs, *s, *o;
  int *miss;
};

size_t noalloc_layout(unsigned char *base, int64_t n, int64_t P, NoAllocBufs *B) {
  Carve c{base};
  const size_t F = (size_t)(P - 1), npad = (size_t)pad16(n);
  B->mean = c.take<double>(F);
  B->sd = c.take<double>(F);
  B->a = c.take<double>((size_t)P);
  B->b = c.take<double>((size_t)P);
  B->s = c.take<double>((size_t)P);
  B->v = c.take<double>(npad);
  B->q = c.take<double>(1);
  B->vs = c.take<double>(1);
  B->o = c.take<double>(1);
  B->miss = c.take<int>(1);
  return c.off;
}

}  // namespace

extern "C" {

int fsqr_lambda_max_noalloc(fsqr_ctx *ctx, const fsqr_design *d, const double *y, double tau,
                            const double *omega, double *out) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  if (!y || !omega || !out) return fail(ctx, FSQR_EINVAL, "NULL argument");
  if (!(tau > 0.0 && tau < 1.0)) return fail(ctx, FSQR_EINVAL, "tau must be in (0,1)");
  TRY(check_design(ctx, d));
  Dsg X{};
  X.n = d->n;
  X.p = d->p;
  X.c = d->c;
  X.P = 1 + d->c + d->p;
  X.fmt = d->geno_format;
  X.geno = static_cast<const uint8_t *>(d->geno);
  X.ld = d->geno_ld;
  X.cov = d->cov;
  NoAllocBufs B;
  const size_t need = noalloc_layout(nullptr, X.n, X.P, &B);
  if (need > (size_t)FSQR_NOALLOC_SCRATCH_BYTES)
    return fail(ctx, FSQR_EINVAL,
                "n = %lld, P = %lld need %zu bytes of scratch; the static scratch holds %d "
                "(FSQR_NOALLOC_SCRATCH_BYTES): use fsqr_lambda_max",
                (long long)X.n, (long long)X.P, need, FSQR_NOALLOC_SCRATCH_BYTES);
  unsigned char *base = nullptr;
  TRY(noalloc_base(ctx, &base));
  noalloc_layout(base, X.n, X.P, &B);
  cudaStream_t st = ctx->stream;
  // The array still holds the previous call's bytes. Every buffer below is
  // fully written before it is read except the missing-entry counter, which
  // k_col_stats increments: it must start at zero.
  CK(cudaMemsetAsync(B.miss, 0, sizeof(int), st));
  LK(launch_col_stats(X, B.mean, B.sd, B.miss, st));
  const double *mean = d->col_mean ? d->col_mean : B.mean;
  const double *sd = d->col_sd ? d->col_sd : B.sd;
  LK(launch_affine(X, mean, sd, d->standardize, B.a, B.b, st));
  X.a = B.a;
  X.b = B.b;
  int hmiss = 0;
  CK(cudaMemcpyAsync(&hmiss, B.miss, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hmiss > 0)
    return fail(ctx, FSQR_EINVAL,
                "%d missing genotype entries: mean imputation of missing entries is not "
                "supported by this library",
                hmiss);
  const int64_t n = X.n, npad = pad16(n);
  int64_t k = (int64_t)ceil((double)n * tau);
  if (k < 1) k = 1;
  if (k > n) k = n;
  LK(launch_select(y, n, k, B.q, st));
  LK(launch_lmax_vec(y, n, npad, tau, B.q, B.v, st));
  LK(launch_sum_cols(B.v, n, npad, 1, B.vs, nullptr, st));
  Fits F = pass_fits(ctx, X);
  LK(launch_col_pass(A_XT, 1, X, F, 0, B.v, B.vs, B.s, nullptr, st));
  LK(launch_colmax_ratio(B.s, omega, X.P, (double)n, B.o, st));
  CK(cudaMemcpyAsync(out, B.o, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return FSQR_OK;
}

}  // extern "C"
