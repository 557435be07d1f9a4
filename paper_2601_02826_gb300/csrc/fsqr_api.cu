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

#include "fsqr_fixed.h"
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
  Dsg X{};
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
  X.mptr = nullptr;
  X.midx = nullptr;
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
  if (X.c > 0 || X.fmt == FSQR_DENSE_F64) {
    // non-finite dense values make the column statistics non-finite
    double *st3;
    TRY(wsget(ctx, "stat_chk", 3, &st3));
    LK(launch_vec_stats(mean, F, st3, ctx->stream));
    double h[3];
    CK(cudaMemcpyAsync(h, st3, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (!std::isfinite(h[0]) || !std::isfinite(h[2]))
      return fail(ctx, FSQR_ENUMERIC, "a covariate or dense feature column contains NaN or Inf");
  }
  if (hmiss > 0) {
    // mean imputation (Section 7.2): per stored column the ascending list of
    // its missing samples; int8 codes are read from a copy whose missing
    // codes are 0 (the E4M3 reading of the tensor-core passes needs 0/1/2)
    const int64_t pc = X.p;
    int *cnt;
    int64_t *mptr;
    TRY(wsget(ctx, "miss_cnt", (size_t)pc, &cnt));
    TRY(wsget(ctx, "miss_ptr", (size_t)pc + 1, &mptr));
    LK(launch_miss_count(X, cnt, ctx->stream));
    std::vector<int> hc((size_t)pc);
    std::vector<int64_t> hp((size_t)pc + 1, 0);
    CK(cudaMemcpyAsync(hc.data(), cnt, sizeof(int) * pc, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int64_t q = 0; q < pc; ++q) hp[q + 1] = hp[q] + hc[q];
    int32_t *midx;
    TRY(wsget(ctx, "miss_idx", (size_t)std::max<int64_t>(hp[pc], 1), &midx));
    CK(cudaMemcpyAsync(mptr, hp.data(), sizeof(int64_t) * (pc + 1), cudaMemcpyHostToDevice, ctx->stream));
    LK(launch_miss_fill(X, mptr, midx, ctx->stream));
    if (X.fmt == FSQR_INT8) {
      uint8_t *clean;
      TRY(wsget(ctx, "miss_geno", (size_t)(pc * X.ld), &clean));
      LK(launch_sanitize_int8(X, clean, ctx->stream));
      X.geno = clean;
    }
    X.mptr = mptr;
    X.midx = midx;
    CK(cudaStreamSynchronize(ctx->stream));
  }
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
  if (X.fmt == FSQR_DENSE_F64) {
    Fits F = pass_fits(ctx, X);
    LK(launch_col_pass(A_XT, 1, X, F, 0, v, vs, s, nullptr, ctx->stream));
  } else {  // int8 / 2-bit codes: exact integer products with v in 52-bit fixed point
    int2 *vq;
    double *vu;
    TRY(wsget(ctx, "lmax_vq", npad, &vq));
    TRY(wsget(ctx, "lmax_vu", 1, &vu));
    LK(launch_fix_seg(v, nullptr, nullptr, nullptr, npad, 1, 0, vq, vu, nullptr, ctx->stream));
    LK(launch_xtv_int(X, nullptr, 1, v, vq, vu, vs, npad, s, ctx->stream));
  }
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
  // int8 / 2-bit codes: both products exact in integers, the vectors in
  // 52-bit fixed point (v per split with its a_j, u per block)
  const bool exact = X.fmt != FSQR_DENSE_F64;
  int2 *qv = nullptr, *qu = nullptr;
  double *uv = nullptr, *cv = nullptr, *uu = nullptr;
  if (exact) {
    TRY(wsget(ctx, "pw_qv", P, &qv));
    TRY(wsget(ctx, "pw_uv", nsplit, &uv));
    TRY(wsget(ctx, "pw_cv", nsplit, &cv));
    TRY(wsget(ctx, "pw_qu", (size_t)G * npad, &qu));
    TRY(wsget(ctx, "pw_uu", G, &uu));
  }
  std::vector<double> lam(G, 0.0), res(G, 0.0), hq(G), hw(G);
  std::vector<char> frozen(G, 0);
  int left = G;
  for (int t = 1; t <= max_iter && left > 0; ++t) {
    if (exact) {
      LK(launch_fix_seg(v, X.a, X.b, d_splits, 0, nsplit, 1 + X.c, qv, uv, cv, ctx->stream));
      LK(launch_xv_blocks_int(X, v, d_splits, d_sob, G, nsplit, qv, uv, cv, U, npad, part, ctx->stream));
    } else {
      LK(launch_xv_blocks(X, v, d_splits, d_sob, G, nsplit, U, npad, part, ctx->stream));
    }
    if (X.mptr) LK(launch_miss_xv(X, v, d_bp, G, U, npad, ctx->stream));
    LK(launch_sum_cols(U, n, npad, G, usum, usq, ctx->stream));
    if (exact) {
      LK(launch_fix_seg(U, nullptr, nullptr, nullptr, npad, G, 0, qu, uu, nullptr, ctx->stream));
      LK(launch_xtv_int(X, d_bp, G, U, qu, uu, usum, npad, w, ctx->stream));
    } else {
      LK(launch_col_pass(A_XT_BLOCK, 1, X, F, 0, U, usum, w, nullptr, ctx->stream));
    }
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
  if (o->max_group < 0 || o->max_group > kWideMax)
    return fail(ctx, FSQR_EINVAL, "max_group must be in 0..32");
  if (o->eta)
    for (int g = 0; g < G; ++g)
      if (!(o->eta[g] > 0.0) || isinf(o->eta[g]))
        return fail(ctx, FSQR_EINVAL, "eta[%d] must be finite and > 0", g);
  if (!(o->eta_margin >= 0.0)) return fail(ctx, FSQR_EINVAL, "eta_margin must be >= 0");
  if (!(o->ridge >= 0.0) || isinf(o->ridge)) return fail(ctx, FSQR_EINVAL, "ridge must be finite and >= 0");
  if (o->screen != 0 && o->screen != 1) return fail(ctx, FSQR_EINVAL, "screen must be 0 or 1");
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

// The tensor-core passes run for int8 or 2-bit storage with at most 63
// covariates and sizes for which the integer arithmetic stays exact: a
// digit-product sum over n samples of |g t| <= 16 is a multiple of 2^-9
// below 2^24 * 2^-9 in FP32 when n <= 2^20. The X~ beta pass sums over the
// active columns only; it checks at run time that fewer than 2^19 are active
// (then its FP32 digit sums stay below 2^24 units and the recombined
// sum_j g_ij W_j, |W_j| < 2^43, below 2^63) and reports an error otherwise.
bool tc_eligible(const Dsg &X, int precision) {
  return precision == FSQR_MIXED && (X.fmt == FSQR_INT8 || X.fmt == FSQR_2BIT) && X.p > 0 && X.c <= 63 &&
         X.n <= ((int64_t)1 << 20) && X.p <= ((int64_t)1 << 20);
}

int solve_group(fsqr_ctx *ctx, const SolveEnv &E, const GroupSpec &gs) {
  const Dsg &X = E.pr->X;
  const int nb = gs.nb;
  const int NB = nb_template(nb);
  const int64_t n = X.n, npad = pad16(n), P = X.P;
  const bool mixed = E.o->precision == FSQR_MIXED || E.o->precision == FSQR_MIXED_SIMT;
  const bool tc = tc_eligible(X, E.o->precision) && NB <= 8;
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
  F.ridge = E.o->ridge;
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
    TRY(wsget(ctx, "g_err", 1, &d_err));
    CK(cudaMemsetAsync(dg, 0, (size_t)(nk * N * 128), st));
    CK(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    if (X.fmt == FSQR_2BIT) {  // packed 4 KB tiles, expanded in the column pass
      TRY(wsget(ctx, "g_xt2", (size_t)(ntile * nk * 4096), &xt));
      LK(launch_tile_x2(X, xt, nk, st));
    } else {
      TRY(wsget(ctx, "g_xt", (size_t)(ntile * nk * 16384), &xt));
      LK(launch_tile_x(X, xt, nk, st));
    }
    const int64_t maxkb = (P + 127) / 128;
    TRY(wsget(ctx, "g_scol", (size_t)(maxkb * 128), &scol));
    TRY(wsget(ctx, "g_wtile", (size_t)(maxkb * xbeta_tc_rows(NB) * 128), &wtile));
    TRY(wsget(ctx, "g_xbtick", (size_t)((n + 127) / 128), &F.xb_tick));
    CK(cudaMemsetAsync(F.xb_tick, 0, sizeof(unsigned) * (size_t)((n + 127) / 128), st));
    TRY(wsget(ctx, "g_tailpart", (size_t)std::max(1, tsc.rem * tsc.slices) * tc_tail_rows(NB, F.D) * 128,
              &tail_part));
    TRY(wsget(ctx, "g_tailtick", (size_t)std::max(1, tsc.rem), &tail_tick));
    CK(cudaMemsetAsync(tail_tick, 0, sizeof(unsigned) * (size_t)std::max(1, tsc.rem), st));
    const size_t smem = col_tc_smem(NB, F.D, F.T, X.fmt == FSQR_2BIT ? 1 : 0);
    if (smem > 200 * 1024)
      return fail(ctx, FSQR_EINVAL, "tensor-core column pass needs %zu B of shared memory", smem);
  }
  if (mixed) {
    TRY(wsget(ctx, "g_digits", (size_t)NB * std::max(F.D, 1) * F.n4p, &F.digits));
    TRY(wsget(ctx, "g_scale", kMaxNB, &F.scale));
    TRY(wsget(ctx, "g_xbipart", (size_t)kBMaxSplits * npad * NB, &F.xb_ipart));
    TRY(wsget(ctx, "g_awmax", (size_t)F.gridA * NB, &F.a_wmax));
  }
  if (X.mptr) {
    TRY(wsget(ctx, "g_qcorr", (size_t)npad * NB, &F.qcorr));
    CK(cudaMemsetAsync(F.qcorr, 0, sizeof(double) * npad * NB, st));
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
  if (F.qcorr) LK(launch_miss_xb(NB, X, F, 0, F.beta[0], st));
  LK(launch_vec(NB, X, F, 0, 1, st));

  // ---- the iteration as a captured graph of M steps
  const int K = F.K;
  const int M = K * std::max(1, (20 + K - 1) / K);
  const bool prof = ctx->prof;
  if (prof && !ctx->ev[0])
    for (int e = 0; e < 6; ++e) CK(cudaEventCreate(&ctx->ev[e]));
  // kernels per step: [quantize] col [check] (xprep + fused xbeta/vector | xbeta + vec)
  int per_graph = 1;  // the advance kernel
  for (int off = 0; off < M; ++off) per_graph += (mixed ? 1 : 0) + 3 + (off % K == 0 ? 1 : 0) + (F.qcorr ? 1 : 0);
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
      if (F.qcorr && ce == cudaSuccess) ce = launch_miss_xb(NB, X, F, off, nullptr, st);
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
  if (tc) ctx->pf.tc_groups += 1;
  else ctx->pf.simt_groups += 1;
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
    LK(launch_summary(NB, nb, n, P, E.y, F.z, F.r, bfin, E.omega, dtaus, dlams, schk_use, tc_use, E.o->ridge,
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

int predict_impl(fsqr_ctx *ctx, const Prep &pr, const double *beta, int B, double *out);

// One fit of a wide solve: its parameters, where its result goes and how it
// starts (cold, from the user's arrays, or from another fit's solution).
struct WideFit {
  double tau, lam, lamnorm;
  int fit;   // output index
  int from;  // -1 cold; >= 0 start from that fit's result (it must finish first)
  bool given;  // start from the user's arrays of this fit (FSQR_WARM_GIVEN / LEARNED)
};

// Wide slot scheduler (batched tau x lambda grid, tensor-core path): NB = 16
// or 32 slots share every X pass. The iteration runs as a captured CUDA
// graph of M steps; between replays the host reads the per-slot done flags,
// moves each finished fit's iterate to the user's arrays, and refills the
// slot with the next ready fit (a fit whose start is another fit's solution
// becomes ready when that fit finishes). Each fit keeps its own iteration
// count from the step at which it entered its slot, so the iterates of a fit
// are those of Algorithm 1 run alone; idle slots carry zero digits.
int solve_wide(fsqr_ctx *ctx, const SolveEnv &E, int NB, const std::vector<WideFit> &fits) {
  const Dsg &X = E.pr->X;
  const int64_t n = X.n, npad = pad16(n), P = X.P;
  const int nf = (int)fits.size();
  cudaStream_t st = ctx->stream;
  const double t0 = now_ms();

  Fits F{};
  F.nb = NB;
  F.n = n;
  F.npad = npad;
  F.y = E.y;
  F.ymax = E.ymax;
  F.omega = E.omega;
  F.block_ptr = E.d_bp;
  F.G = E.G;
  F.eta = E.d_eta;
  F.inv_eta = E.d_ieta;
  for (int b = 0; b < kMaxNB; ++b) { F.tau[b] = 0.5; F.lam[b] = 0.0; F.lamnorm[b] = 1.0; }
  F.mu = E.mu;
  F.sigma = E.mu / (double)(E.G + 1);
  F.tol = E.o->tol;
  F.ridge = E.o->ridge;
  F.K = E.o->check_every;
  F.max_iter = E.o->max_iter;
  F.mixed = 1;
  F.D = 7;
  F.dbits = 4;
  F.DW = 11;
  F.th_unit = ldexp(1.0, -28);
  F.xb_unit = ldexp(1.0, -44);
  F.n4p = npad / 4;
  F.colbound = E.pr->colbound;
  TcSchedule tsc{};
  col_tc_schedule(X.p, n, ctx->num_sms, &tsc);
  tsc.slices = 0;
  tsc.slots = tsc.grid;
  F.T = tsc.list_stride;
  F.gridA = tsc.grid;
  const int rows = (int)((n + 127) / 128);
  F.gridC = rows;
  if (wcol_smem(NB, F.T) > 227 * 1024)
    return fail(ctx, FSQR_EINVAL, "wide column pass needs %zu B of shared memory", wcol_smem(NB, F.T));
  TRY(wsget(ctx, "w_beta0", (size_t)P * NB, &F.beta[0]));
  TRY(wsget(ctx, "w_beta1", (size_t)P * NB, &F.beta[1]));
  TRY(wsget(ctx, "w_z", (size_t)npad * NB, &F.z));
  TRY(wsget(ctx, "w_theta", (size_t)npad * NB, &F.theta));
  TRY(wsget(ctx, "w_r", (size_t)npad * NB, &F.r));
  TRY(wsget(ctx, "w_arb", (size_t)F.gridA * NB, &F.a_rb));
  TRY(wsget(ctx, "w_act", (size_t)F.gridA * NB, &F.a_ct));
  TRY(wsget(ctx, "w_awmax", (size_t)F.gridA * NB, &F.a_wmax));
  TRY(wsget(ctx, "w_acnt", (size_t)F.gridA, &F.a_cnt));
  TRY(wsget(ctx, "w_alist", (size_t)F.gridA * F.T, &F.a_list));
  TRY(wsget(ctx, "w_metai", 4, &F.meta_i));
  TRY(wsget(ctx, "w_metad", 2 * kWideMax, &F.meta_d));
  TRY(wsget(ctx, "w_cpart0", (size_t)rows * NB * kCPartials, &F.c_part[0]));
  TRY(wsget(ctx, "w_cpart1", (size_t)rows * NB * kCPartials, &F.c_part[1]));
  TRY(wsget(ctx, "w_totc0", (size_t)kWideMax * kCPartials, &F.tot_c[0]));
  TRY(wsget(ctx, "w_totc1", (size_t)kWideMax * kCPartials, &F.tot_c[1]));
  TRY(wsget(ctx, "w_tota", (size_t)kWideMax * 3, &F.tot_a));
  TRY(wsget(ctx, "w_apre", (size_t)F.gridA + 1, &F.a_pre));
  TRY(wsget(ctx, "w_tick", 2, &F.tickets));
  TRY(wsget(ctx, "w_xbtick", (size_t)rows, &F.xb_tick));
  TRY(wsget(ctx, "w_done", kWideMax, &F.done));
  TRY(wsget(ctx, "w_ndone", 1, &F.n_done));
  TRY(wsget(ctx, "w_report", (size_t)kWideMax * kReport, &F.report));
  TRY(wsget(ctx, "w_scale", kWideMax, &F.scale));
  TRY(wsget(ctx, "w_xbipart", (size_t)16 * npad * NB, &F.xb_ipart));
  int *it_base;
  TRY(wsget(ctx, "w_itbase", 1, &it_base));
  F.it_base = it_base;
  double *d_tau, *d_lam, *d_lamnorm, *zero, *rfit;
  int *d_k0, *d_mask, *d_err, *scol;
  TRY(wsget(ctx, "w_tau", kWideMax, &d_tau));
  TRY(wsget(ctx, "w_lam", kWideMax, &d_lam));
  TRY(wsget(ctx, "w_lamnorm", kWideMax, &d_lamnorm));
  TRY(wsget(ctx, "w_k0", kWideMax, &d_k0));
  TRY(wsget(ctx, "w_mask", kWideMax, &d_mask));
  TRY(wsget(ctx, "w_zero", (size_t)std::max<int64_t>(P, npad), &zero));
  TRY(wsget(ctx, "w_rfit", (size_t)nf * n, &rfit));
  TRY(wsget(ctx, "g_err", 1, &d_err));
  F.w_tau = d_tau;
  F.w_lam = d_lam;
  F.w_lamnorm = d_lamnorm;
  F.w_k0 = d_k0;
  const int64_t nk = (n + 127) / 128, ntile = (X.p + 127) / 128, maxkb = (P + 127) / 128;
  uint8_t *dg, *xt, *wtile;
  TRY(wsget(ctx, "w_dg", (size_t)(nk * wide_rows(NB) * 128), &dg));
  TRY(wsget(ctx, "g_xt", (size_t)(ntile * nk * 16384), &xt));
  TRY(wsget(ctx, "g_scol", (size_t)(maxkb * 128), &scol));
  TRY(wsget(ctx, "w_wtile", (size_t)(maxkb * wide_xrows(NB) * 128), &wtile));
  double *xbtmp;
  TRY(wsget(ctx, "w_xbtmp", (size_t)npad, &xbtmp));
  if (X.mptr) {
    TRY(wsget(ctx, "w_qcorr", (size_t)npad * NB, &F.qcorr));
    CK(cudaMemsetAsync(F.qcorr, 0, sizeof(double) * npad * NB, st));
  }
  CK(cudaMemsetAsync(dg, 0, (size_t)(nk * wide_rows(NB) * 128), st));
  CK(cudaMemsetAsync(d_err, 0, sizeof(int), st));
  CK(cudaMemsetAsync(zero, 0, sizeof(double) * std::max<int64_t>(P, npad), st));
  CK(cudaMemsetAsync(F.xb_tick, 0, sizeof(unsigned) * rows, st));
  CK(cudaMemsetAsync(F.tickets, 0, 2 * sizeof(unsigned), st));
  CK(cudaMemsetAsync(F.tot_c[0], 0, sizeof(double) * kWideMax * kCPartials, st));
  CK(cudaMemsetAsync(F.tot_c[1], 0, sizeof(double) * kWideMax * kCPartials, st));
  CK(cudaMemsetAsync(F.tot_a, 0, sizeof(double) * kWideMax * 3, st));
  CK(cudaMemsetAsync(F.report, 0, sizeof(double) * kWideMax * kReport, st));
  CK(cudaMemsetAsync(F.beta[0], 0, sizeof(double) * P * NB, st));
  CK(cudaMemsetAsync(F.beta[1], 0, sizeof(double) * P * NB, st));
  CK(cudaMemsetAsync(F.z, 0, sizeof(double) * npad * NB, st));
  CK(cudaMemsetAsync(F.theta, 0, sizeof(double) * npad * NB, st));
  CK(cudaMemsetAsync(F.r, 0, sizeof(double) * npad * NB, st));
  CK(cudaMemsetAsync(it_base, 0, sizeof(int), st));
  CK(cudaMemsetAsync(F.n_done, 0, sizeof(int), st));
  LK(launch_tile_x(X, xt, nk, st));

  // host mirror of the per-slot state (pinned: done flags and reports come back every replay)
  double *hp;
  TRY(pinned(ctx, (size_t)kWideMax * kReport + 4 * kWideMax + 64, &hp));
  double *hrep = hp;
  int *hdone = reinterpret_cast<int *>(hp + kWideMax * kReport);
  std::vector<int> slot_fit(NB, -1), hk0(NB, 0), hmask(NB, 0);
  std::vector<double> htau(NB, 0.5), hlam(NB, 0.0), hlamn(NB, 1.0);
  std::vector<int> state(nf, 0);  // 0 waiting, 1 running, 2 finished
  std::vector<int> fit_pos(nf, 0);
  for (int q = 0; q < nf; ++q) fit_pos[q] = q;
  std::vector<int> pos_of_fit;  // output fit index -> position in fits
  {
    int mx = 0;
    for (const WideFit &w : fits) mx = std::max(mx, w.fit);
    pos_of_fit.assign(mx + 1, -1);
    for (int q = 0; q < nf; ++q) pos_of_fit[fits[q].fit] = q;
  }
  const int kIdle = 0x7fffffff;
  for (int b = 0; b < NB; ++b) hdone[b] = kIdle;
  int next = 0, finished = 0;
  int host_base = 0;
  bool timed_out = false;

  // fills the empty slots with ready fits at iteration host_base
  auto fill = [&]() -> int {
    const int par = host_base & 1;
    bool any = false;
    for (int b = 0; b < NB; ++b) {
      if (slot_fit[b] >= 0) continue;
      int pick = -1;
      for (int q = next; q < nf; ++q) {
        if (state[q] != 0) continue;
        const int src = fits[q].from;
        if (src >= 0 && (src >= (int)pos_of_fit.size() || pos_of_fit[src] < 0 || state[pos_of_fit[src]] != 2))
          continue;
        pick = q;
        break;
      }
      if (pick < 0) break;
      const WideFit &w = fits[pick];
      state[pick] = 1;
      while (next < nf && state[next] != 0) ++next;
      slot_fit[b] = pick;
      double *bs = F.beta[par] + b, *zs = F.z + b, *ts = F.theta + b, *rs = F.r + b;
      if (w.from >= 0) {
        const int sf = w.from;
        LK(launch_pack(E.beta + (int64_t)sf * P, P, bs, P, 1, NB, P, st));
        LK(launch_pack(E.z + (int64_t)sf * n, n, zs, n, 1, NB, npad, st));
        LK(launch_pack(E.theta + (int64_t)sf * n, n, ts, n, 1, NB, npad, st));
        LK(launch_pack(rfit + (int64_t)pos_of_fit[sf] * n, n, rs, n, 1, NB, npad, st));
      } else if (w.given) {
        const int f = w.fit;
        LK(launch_pack(E.beta + (int64_t)f * P, P, bs, P, 1, NB, P, st));
        LK(launch_pack(E.z + (int64_t)f * n, n, zs, n, 1, NB, npad, st));
        LK(launch_pack(E.theta + (int64_t)f * n, n, ts, n, 1, NB, npad, st));
        TRY(predict_impl(ctx, *E.pr, E.beta + (int64_t)f * P, 1, xbtmp));
        LK(launch_resid_slot(xbtmp, E.z + (int64_t)f * n, E.y, n, F.r, b, NB, st));
      } else {
        LK(launch_pack(zero, P, bs, P, 1, NB, P, st));
        LK(launch_pack(E.y, n, zs, n, 1, NB, npad, st));
        LK(launch_pack(zero, n, ts, n, 1, NB, npad, st));
        LK(launch_pack(zero, n, rs, n, 1, NB, npad, st));
      }
      htau[b] = w.tau;
      hlam[b] = w.lam;
      hlamn[b] = w.lamnorm;
      hk0[b] = host_base;
      hdone[b] = -1;
      hmask[b] = 1;
      any = true;
    }
    if (!any) return FSQR_OK;
    CK(cudaMemcpyAsync(d_tau, htau.data(), sizeof(double) * NB, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_lam, hlam.data(), sizeof(double) * NB, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_lamnorm, hlamn.data(), sizeof(double) * NB, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_k0, hk0.data(), sizeof(int) * NB, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_mask, hmask.data(), sizeof(int) * NB, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(F.done, hdone, sizeof(int) * NB, cudaMemcpyHostToDevice, st));
    LK(launch_slot_init(NB, F, par, d_mask, st));
    CK(cudaStreamSynchronize(st));  // the host arrays are reused by the next fill
    for (int b = 0; b < NB; ++b) hmask[b] = 0;
    return FSQR_OK;
  };
  TRY(fill());

  // ---- the iteration as a captured graph of M steps
  const int K = F.K;
  const int M = K * std::max(1, (20 + K - 1) / K);
  const bool prof = ctx->prof;
  if (prof && !ctx->ev[0])
    for (int e = 0; e < 6; ++e) CK(cudaEventCreate(&ctx->ev[e]));
  int per_graph = 1;
  for (int off = 0; off < M; ++off) per_graph += 4 + (off % K == 0 ? 1 : 0) + (F.qcorr ? 1 : 0);
  auto enqueue = [&](bool sample) -> cudaError_t {
    cudaError_t ce = cudaSuccess;
    for (int off = 0; off < M && ce == cudaSuccess; ++off) {
      const bool sm = sample && off == M - 1;
      ce = launch_wquant(NB, F, off, dg, st);
      if (sm && ce == cudaSuccess) ce = cudaEventRecord(ctx->ev[0], st);
      if (ce == cudaSuccess) ce = launch_wcol(NB, X, F, off, xt, dg, tsc.rounds, d_err, st);
      if (sm && ce == cudaSuccess) ce = cudaEventRecord(ctx->ev[1], st);
      if (off % K == 0 && ce == cudaSuccess) ce = launch_wcheck(NB, F, off, st);
      if (F.qcorr && ce == cudaSuccess) ce = launch_miss_xb(NB, X, F, off, nullptr, st);
      if (sm && ce == cudaSuccess) ce = cudaEventRecord(ctx->ev[2], st);
      if (ce == cudaSuccess) ce = launch_wxbeta(NB, X, F, off, 1, nullptr, scol, wtile, d_err, ctx->num_sms, st);
      if (sm && ce == cudaSuccess) ce = cudaEventRecord(ctx->ev[3], st);
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
    return fail(ctx, FSQR_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce != cudaSuccess ? ce : ee));
  }
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return fail(ctx, FSQR_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));

  std::vector<int> iters_of(nf, 0), status_of(nf, FSQR_OK);
  std::vector<double> rep_of((size_t)nf * kReport, 0.0);
  int64_t max_iter_sum = 0;
  for (int q = 0; q < nf; ++q) max_iter_sum += E.o->max_iter;
  const int64_t max_launch = max_iter_sum / M + 3 * (int64_t)nf + 8;
  int rc = FSQR_OK;
  int live = 0;
  for (int b = 0; b < NB; ++b) live += slot_fit[b] >= 0;
  for (int64_t l = 0; live > 0; ++l) {
    const bool sample = prof && (l % 4 == 0);
    ce = sample ? enqueue(true) : cudaGraphLaunch(exec, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(hdone, F.done, sizeof(int) * NB, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(hrep, F.report, sizeof(double) * NB * kReport, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
      rc = fail(ctx, FSQR_ECUDA, "wide iteration graph: %s", cudaGetErrorString(ce));
      break;
    }
    host_base += M;
    ctx->pf.kernel_launches += per_graph;
    if (sample) {
      float a = 0.f, b2 = 0.f;
      if (cudaEventElapsedTime(&a, ctx->ev[0], ctx->ev[1]) == cudaSuccess &&
          cudaEventElapsedTime(&b2, ctx->ev[2], ctx->ev[3]) == cudaSuccess) {
        ctx->pf.col_ms += a;
        ctx->pf.col_samples += 1;
        ctx->pf.xb_ms += b2;
        ctx->pf.xb_samples += 1;
      } else {
        cudaGetLastError();
      }
    }
    if (E.deadline_ms > 0 && now_ms() > E.deadline_ms) timed_out = true;
    // move finished fits out of their slots
    bool freed = false;
    for (int b = 0; b < NB; ++b) {
      const int q = slot_fit[b];
      if (q < 0) continue;
      const bool fin = hdone[b] >= 0 && hdone[b] != kIdle;
      if (!fin && !timed_out) continue;
      const int kf = fin ? hdone[b] : host_base;
      const int f = fits[q].fit;
      LK(launch_unpack(F.beta[kf & 1] + b, E.beta + (int64_t)f * P, P, P, 1, NB, st));
      LK(launch_unpack(F.z + b, E.z + (int64_t)f * n, n, n, 1, NB, st));
      LK(launch_unpack(F.theta + b, E.theta + (int64_t)f * n, n, n, 1, NB, st));
      LK(launch_unpack(F.r + b, rfit + (int64_t)q * n, n, n, 1, NB, st));
      for (int t = 0; t < kReport; ++t) rep_of[(size_t)q * kReport + t] = hrep[b * kReport + t];
      iters_of[q] = fin ? (int)hrep[b * kReport + 7] : host_base - hk0[b];
      status_of[q] = fin ? (int)hrep[b * kReport + 5] : FSQR_ETIMEOUT;
      state[q] = 2;
      ++finished;
      slot_fit[b] = -1;
      hdone[b] = kIdle;
      freed = true;
    }
    if (timed_out) break;
    if (freed) {
      CK(cudaMemcpyAsync(F.done, hdone, sizeof(int) * NB, cudaMemcpyHostToDevice, st));
      TRY(fill());
    }
    live = 0;
    for (int b = 0; b < NB; ++b) live += slot_fit[b] >= 0;
    if (l > max_launch) {
      rc = fail(ctx, FSQR_ECUDA, "wide iteration did not stop after %d steps", host_base);
      break;
    }
  }
  cudaGraphExecDestroy(exec);
  if (rc != FSQR_OK) return rc;
  {
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (herr != 0)
      return fail(ctx, FSQR_ECUDA, "wide tensor-core pass: a pipeline wait ran out of time (code %d)", herr);
  }
  if (!timed_out && finished < nf)
    return fail(ctx, FSQR_EINVAL, "%d fits could not start (a start refers to a fit outside the solve)",
                nf - finished);
  ctx->pf.iterations += host_base;
  ctx->pf.col_bytes = n * X.p + 8 * n * X.c + 2 * 8 * P * NB;
  ctx->pf.wide_groups += 1;
  const double t_solve = now_ms() - t0;

  // ---- per-fit reports: primal value, active count, duality gap (groups of 8)
  if (E.infos) {
    double *bfin, *zfin, *rfin, *thfin, *tcd, *tcs, *schk, *summ, *dtaus, *dlams;
    TRY(wsget(ctx, "r_bfin", (size_t)P * kMaxNB, &bfin));
    TRY(wsget(ctx, "r_zfin", (size_t)npad * kMaxNB, &zfin));
    TRY(wsget(ctx, "r_rfin", (size_t)npad * kMaxNB, &rfin));
    TRY(wsget(ctx, "r_thfin", (size_t)npad * kMaxNB, &thfin));
    TRY(wsget(ctx, "r_tc", (size_t)npad * kMaxNB, &tcd));
    TRY(wsget(ctx, "r_tcs", kMaxNB, &tcs));
    TRY(wsget(ctx, "r_schk", (size_t)P * kMaxNB, &schk));
    TRY(wsget(ctx, "r_summ", (size_t)kMaxNB * 8, &summ));
    TRY(wsget(ctx, "r_taus", kMaxNB, &dtaus));
    TRY(wsget(ctx, "r_lams", kMaxNB, &dlams));
    Fits Fx = pass_fits(ctx, X);
    for (int q0 = 0; q0 < nf; q0 += kMaxNB) {
      const int nb = std::min(kMaxNB, nf - q0);
      const int NB8 = nb_template(nb);
      double ht[kMaxNB], hl[kMaxNB];
      for (int u = 0; u < kMaxNB; ++u) {
        ht[u] = u < nb ? fits[q0 + u].tau : 0.5;
        hl[u] = u < nb ? fits[q0 + u].lam : 0.0;
      }
      CK(cudaMemsetAsync(bfin, 0, sizeof(double) * P * NB8, st));
      CK(cudaMemsetAsync(zfin, 0, sizeof(double) * npad * NB8, st));
      CK(cudaMemsetAsync(rfin, 0, sizeof(double) * npad * NB8, st));
      CK(cudaMemsetAsync(thfin, 0, sizeof(double) * npad * NB8, st));
      for (int u = 0; u < nb; ++u) {
        const int f = fits[q0 + u].fit;
        LK(launch_pack(E.beta + (int64_t)f * P, P, bfin + u, P, 1, NB8, P, st));
        LK(launch_pack(E.z + (int64_t)f * n, n, zfin + u, n, 1, NB8, npad, st));
        LK(launch_pack(E.theta + (int64_t)f * n, n, thfin + u, n, 1, NB8, npad, st));
        LK(launch_pack(rfit + (int64_t)(q0 + u) * n, n, rfin + u, n, 1, NB8, npad, st));
      }
      CK(cudaMemcpyAsync(dtaus, ht, sizeof ht, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(dlams, hl, sizeof hl, cudaMemcpyHostToDevice, st));
      const double *schk_use = nullptr, *tc_use = nullptr;
      if (E.gap_defined) {
        LK(launch_dual_point(NB8, thfin, n, npad, dtaus, nb, tcd, tcs, st));
        LK(launch_col_pass(A_XT, NB8, X, Fx, 0, tcd, tcs, schk, nullptr, st));
        schk_use = schk;
        tc_use = tcd;
      }
      LK(launch_summary(NB8, nb, n, P, E.y, zfin, rfin, bfin, E.omega, dtaus, dlams, schk_use, tc_use, E.o->ridge,
                        summ, st));
      double hs[kMaxNB * 8];
      CK(cudaMemcpyAsync(hs, summ, sizeof(double) * kMaxNB * 8, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int u = 0; u < nb; ++u) {
        const int q = q0 + u;
        fsqr_info &I = E.infos[fits[q].fit];
        const double *rp = &rep_of[(size_t)q * kReport];
        I.status = status_of[q];
        I.iters = iters_of[q];
        I.kkt = rp[0];
        I.r_p = rp[1];
        I.r_z = rp[2];
        I.r_beta = rp[3];
        I.r_1 = rp[4];
        I.primal = hs[u * 8 + 0] + hs[u * 8 + 1];
        I.active = (int64_t)hs[u * 8 + 2];
        if (E.gap_defined) {
          I.dual = hs[u * 8 + 3] * hs[u * 8 + 4];
          I.gap = (I.primal - I.dual) / (1.0 + fabs(I.primal) + fabs(I.dual));
        } else {
          I.dual = NAN;
          I.gap = NAN;
        }
        I.lambda = fits[q].lam;
        I.lambda_max = fits[q].lamnorm;
        I.mu = E.mu;
        I.t_solve_ms = t_solve;
      }
    }
  } else {
    CK(cudaStreamSynchronize(st));
  }
  return timed_out ? FSQR_ETIMEOUT : FSQR_OK;
}

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
  // the partition enters the key: eta_g and the per-block work depend on it
  uint64_t bph = 1469598103934665603ull;
  {
    std::vector<int64_t> hbp(E.G + 1);
    if (cudaMemcpy(hbp.data(), E.d_bp, sizeof(int64_t) * (E.G + 1), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(ctx, FSQR_ECUDA, "block partition read-back failed");
    for (int64_t v : hbp) bph = (bph ^ (uint64_t)v) * 1099511628211ull;
  }
  char key[200];
  snprintf(key, sizeof key, "%lld/%lld/%lld/%d/%d/%d/%d/%d/%d/%llx", (long long)X.n, (long long)X.p,
           (long long)X.c, X.fmt, o->precision, o->digits, B, o->warm, E.G, (unsigned long long)bph);
  auto it = ctx->tuned.find(key);
  if (it != ctx->tuned.end()) {
    *out = it->second;
    ctx->pf.tuned_group = it->second;
    return FSQR_OK;
  }
  std::vector<int> cand;
  for (int g : {1, 2, 3, 4, std::min(B, kMaxNB)})
    if (g <= B && (cand.empty() || g > cand.back())) cand.push_back(g);
  if (tc_eligible(X, o->precision) && X.fmt == FSQR_INT8) {  // wide slots (their fits run min(B, g) at a time)
    if (B > kMaxNB) cand.push_back(16);
    if (B > 16) cand.push_back(kWideMax);
  }
  const int gmax = std::min(B, cand.back());
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
    const int gf = std::min(g, B);
    std::vector<WideFit> wf;
    for (int q = 0; q < gf && g > kMaxNB; ++q) {
      const int t = q / n_lambda;
      WideFit w{};
      w.tau = taus[t];
      w.lam = lambdas[q];
      w.lamnorm = lmax[t] > 0.0 ? lmax[t] : 1.0;
      w.fit = q;
      w.from = -1;
      w.given = false;
      wf.push_back(w);
    }
    GroupSpec gs{};
    gs.nb = std::min(g, kMaxNB);
    for (int q = 0; q < gs.nb; ++q) {
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
      if (g > kMaxNB) TRY(solve_wide(ctx, E2, g, wf));
      else TRY(solve_group(ctx, E2, gs));
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

// lamnorm_in (host, n_tau; may be NULL): the lambda_max(tau) that divides R_b,
// in place of the one of omega (the reweighted fits of LLA keep the first
// fit's). eta_out (may be NULL): receives the eta_g used.
int fit_batch_impl(fsqr_ctx *ctx, const fsqr_design *Xd, const double *y, int n_tau,
                   const double *taus, int n_lambda, const double *lambdas, const double *omega,
                   const int64_t *block_ptr, int G, const fsqr_opts *opts, double *beta, double *z,
                   double *theta, fsqr_info *infos, const double *lamnorm_in = nullptr,
                   std::vector<double> *eta_out = nullptr) {
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
  if (opts->precision == FSQR_MIXED_SIMT && Xd && Xd->geno_format != FSQR_INT8)
    return fail(ctx, FSQR_EINVAL, "FSQR_MIXED_SIMT needs FSQR_INT8 genotype storage");
  if (opts->precision == FSQR_MIXED && Xd && Xd->geno_format == FSQR_DENSE_F64 && Xd->p > 0)
    return fail(ctx, FSQR_EINVAL, "mixed precision needs genotype (int8 or 2-bit) storage");
  Prep pr;
  TRY(prepare(ctx, Xd, &pr, opts->precision != FSQR_FP64));
  const Dsg &X = pr.X;
  const int64_t P = X.P, n = X.n;
  TRY(check_blocks(ctx, block_ptr, G, P));
  if (opts->precision == FSQR_MIXED && X.fmt == FSQR_2BIT && !tc_eligible(X, opts->precision))
    return fail(ctx, FSQR_EINVAL,
                "2-bit storage in FSQR_MIXED needs n, p <= 2^20 and at most 63 covariates; use FSQR_FP64");
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
  if (eta_out) *eta_out = eta;
  std::vector<double> lmax(n_tau);
  for (int t = 0; t < n_tau; ++t) {
    if (lamnorm_in) lmax[t] = lamnorm_in[t];
    else TRY(lambda_max_impl(ctx, pr, y, taus[t], omega, &lmax[t]));
  }
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
  E.gap_defined = ((P == 1) || (om[1] > 0.0)) && opts->ridge == 0.0;
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
  if (mg > kMaxNB && tc_eligible(X, opts->precision) && X.fmt == FSQR_INT8) {
    // wide slots: every fit streams through 16 or 32 slots of one solve
    std::vector<WideFit> wf;
    for (int t = 0; t < n_tau; ++t)
      for (int l = 0; l < n_lambda; ++l) {
        const int f = t * n_lambda + l;
        WideFit w{};
        w.tau = taus[t];
        w.lam = lambdas[f];
        w.lamnorm = lmax[t] > 0.0 ? lmax[t] : 1.0;
        w.fit = f;
        w.from = (opts->warm == FSQR_WARM_PATH && l > 0) ? f - 1 : -1;
        w.given = opts->warm == FSQR_WARM_GIVEN || opts->warm == FSQR_WARM_LEARNED;
        wf.push_back(w);
      }
    const int rcw = solve_wide(ctx, E, mg <= 16 ? 16 : kWideMax, wf);
    if (rcw != FSQR_OK && rcw != FSQR_ETIMEOUT) return rcw;
    int worstw = FSQR_OK;
    if (infos)
      for (int f = 0; f < B; ++f) {
        infos[f].t_setup_ms = t_setup;
        if (worstw == FSQR_OK && infos[f].status != FSQR_OK) worstw = infos[f].status;
      }
    return infos ? worstw : rcw;
  }
  mg = std::min(mg, kMaxNB);
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

// s_out (host, nf x P) = X~^T theta_b for nf fits whose theta sit at
// th + b*n (device, fit-major): full column passes, 8 fits at a time.
int full_xt(fsqr_ctx *ctx, const Prep &pr, const double *th, int nf, std::vector<double> &s_out) {
  const Dsg &X = pr.X;
  const int64_t n = X.n, npad = pad16(n), P = X.P;
  cudaStream_t st = ctx->stream;
  double *il, *sums, *s;
  TRY(wsget(ctx, "sc_thil", (size_t)npad * kMaxNB, &il));
  TRY(wsget(ctx, "sc_sums", kMaxNB, &sums));
  TRY(wsget(ctx, "sc_s", (size_t)P * kMaxNB, &s));
  s_out.assign((size_t)nf * P, 0.0);
  std::vector<double> h((size_t)P * kMaxNB);
  Fits Fx = pass_fits(ctx, X);
  for (int b0 = 0; b0 < nf; b0 += kMaxNB) {
    const int nb = std::min(kMaxNB, nf - b0);
    const int NB = nb_template(nb);
    const double *tb = th + (int64_t)b0 * n;
    CK(cudaMemsetAsync(il, 0, sizeof(double) * npad * NB, st));
    CK(cudaMemsetAsync(sums, 0, sizeof(double) * kMaxNB, st));
    LK(launch_pack(tb, n, il, n, nb, NB, npad, st));
    LK(launch_sum_cols(tb, n, n, nb, sums, nullptr, st));
    LK(launch_col_pass(A_XT, NB, X, Fx, 0, il, sums, s, nullptr, st));
    CK(cudaMemcpyAsync(h.data(), s, sizeof(double) * P * NB, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int b = 0; b < nb; ++b)
      for (int64_t j = 0; j < P; ++j) s_out[(size_t)(b0 + b) * P + j] = h[(size_t)j * NB + b];
  }
  return FSQR_OK;
}

// Sequential strong rule along each tau's lambda path (opts.screen with
// FSQR_WARM_PATH). At stage l, stored column j is left out of the fits of
// every tau when |s_j| < omega_j (2 lambda_l - lambda_{l-1}) for each tau,
// with s = X~^T theta of the tau's fit at lambda_{l-1} (at l = 0 the
// lambda_max direction, lambda_{-1} = lambda_max), and beta_j = 0 there. The
// stage's fits are solved on the kept columns only (same standardisation,
// blocks, eta and lambda_max), each from its predecessor's solution; then
// s = X~^T theta over ALL columns is checked: a left-out column with
// (|s_j| - lambda_j)_+ / lambda_max > tol is put back and the stage re-solved.
// So every returned fit meets the stop test on the full design.
int fit_path_screened(fsqr_ctx *ctx, const fsqr_design *Xd, const double *y, int n_tau, const double *taus,
                      int n_lambda, const double *lambdas, const double *omega, const int64_t *block_ptr, int G,
                      const fsqr_opts *opts, double *beta, double *z, double *theta, fsqr_info *infos) {
  const double t0 = now_ms();
  TRY(check_opts(ctx, opts, G));
  if (n_tau < 1 || n_lambda < 1 || !taus || !lambdas) return fail(ctx, FSQR_EINVAL, "bad tau/lambda grid");
  if (!y || !omega || !beta || !z || !theta) return fail(ctx, FSQR_EINVAL, "NULL array argument");
  if (n_tau > kWideMax) return fail(ctx, FSQR_EINVAL, "screening takes at most %d quantiles", kWideMax);
  Prep pr;
  TRY(prepare(ctx, Xd, &pr, opts->precision != FSQR_FP64));
  const Dsg &X = pr.X;
  const int64_t n = X.n, P = X.P, c = X.c, p = X.p, npad = pad16(n);
  TRY(check_blocks(ctx, block_ptr, G, P));
  cudaStream_t st = ctx->stream;
  double ymax, ysd;
  TRY(y_stats(ctx, y, n, &ymax, &ysd));
  const double mu = opts->mu > 0.0 ? opts->mu : 1.0 / ((double)n * (ysd > 0.0 ? ysd : 1.0));
  std::vector<double> eta(G);
  if (opts->eta) for (int g = 0; g < G; ++g) eta[g] = opts->eta[g];
  else TRY(eta_impl(ctx, pr, block_ptr, G, mu, opts->eta_margin, opts->power_iters, opts->power_tol, eta.data()));
  // lambda_max and its direction s_dir = X~^T v / n per tau
  std::vector<double> lmax(n_tau), sprev((size_t)n_tau * P), hom(P);
  for (int t = 0; t < n_tau; ++t) {
    LmaxDev L;
    TRY(lambda_max_dev(ctx, pr, y, taus[t], omega, &L));
    double lm;
    CK(cudaMemcpyAsync(&lm, L.o, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(sprev.data() + (size_t)t * P, L.s, sizeof(double) * P, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    lmax[t] = lm > 0.0 ? lm : 1.0;
    for (int64_t j = 0; j < P; ++j) sprev[(size_t)t * P + j] /= (double)n;
  }
  CK(cudaMemcpyAsync(hom.data(), omega, sizeof(double) * P, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  // work buffers
  int32_t *d_sel, *d_idx;
  uint8_t *g_red;
  double *m_red, *s_red, *om_red, *b_red, *z_st, *t_st;
  TRY(wsget(ctx, "sc_sel", (size_t)std::max<int64_t>(p, 1), &d_sel));
  TRY(wsget(ctx, "sc_idx", (size_t)P, &d_idx));
  TRY(wsget(ctx, "sc_geno", (size_t)std::max<int64_t>(p * Xd->geno_ld, 16), &g_red));
  TRY(wsget(ctx, "sc_mean", (size_t)(c + p), &m_red));
  TRY(wsget(ctx, "sc_sd", (size_t)(c + p), &s_red));
  TRY(wsget(ctx, "sc_om", (size_t)P, &om_red));
  TRY(wsget(ctx, "sc_beta", (size_t)n_tau * P, &b_red));
  TRY(wsget(ctx, "sc_z", (size_t)n_tau * n, &z_st));
  TRY(wsget(ctx, "sc_th", (size_t)n_tau * n, &t_st));
  std::vector<double> hbeta((size_t)P);
  std::vector<fsqr_info> st_info(n_tau);
  int worst = FSQR_OK;
  for (int l = 0; l < n_lambda; ++l) {
    std::vector<char> keep((size_t)p, 0);
    for (int t = 0; t < n_tau; ++t) {
      const int f = t * n_lambda + l;
      const double lam = lambdas[f], lprev = l ? lambdas[f - 1] : lmax[t];
      if (l) CK(cudaMemcpy(hbeta.data(), beta + (int64_t)(f - 1) * P, sizeof(double) * P, cudaMemcpyDeviceToHost));
      for (int64_t s = 0; s < p; ++s) {
        const int64_t j = 1 + c + s;
        if (hom[j] == 0.0 || fabs(sprev[(size_t)t * P + j]) >= hom[j] * (2.0 * lam - lprev) ||
            (l && hbeta[j] != 0.0))
          keep[s] = 1;
      }
    }
    for (int round = 0;; ++round) {
      // the reduced solve below re-prepares its own design in the same named
      // workspace (statistics, affine maps, missing lists): prepare the full
      // design again before its statistics and products are read
      if (l > 0 || round > 0) TRY(prepare(ctx, Xd, &pr, opts->precision != FSQR_FP64));
      std::vector<int32_t> sel, idx;
      for (int64_t j = 0; j <= c; ++j) idx.push_back((int32_t)j);
      for (int64_t s = 0; s < p; ++s)
        if (keep[s]) { sel.push_back((int32_t)s); idx.push_back((int32_t)(1 + c + s)); }
      const int64_t ns = (int64_t)sel.size(), Pr = 1 + c + ns;
      ctx->pf.screen_kept += ns * n_tau;
      ctx->pf.screen_total += p * n_tau;
      // reduced design: kept stored columns, the full design's statistics
      CK(cudaMemcpyAsync(d_idx, idx.data(), sizeof(int32_t) * Pr, cudaMemcpyHostToDevice, st));
      if (ns) CK(cudaMemcpyAsync(d_sel, sel.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, st));
      LK(launch_gather_cols(static_cast<const uint8_t *>(Xd->geno), Xd->geno_ld, d_sel, ns, g_red, st));
      if (c) {
        CK(cudaMemcpyAsync(m_red, pr.mean, sizeof(double) * c, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(s_red, pr.sd, sizeof(double) * c, cudaMemcpyDeviceToDevice, st));
      }
      LK(launch_index_copy(pr.mean + c, 0, d_sel, ns, 1, m_red + c, 0, 0, st));
      LK(launch_index_copy(pr.sd + c, 0, d_sel, ns, 1, s_red + c, 0, 0, st));
      LK(launch_index_copy(omega, 0, d_idx, Pr, 1, om_red, 0, 0, st));
      std::vector<int64_t> bpr(1, 0);
      std::vector<double> etar;
      {
        size_t q = 0;
        for (int g = 0; g < G; ++g) {
          int64_t cnt = 0;
          while (q < idx.size() && idx[q] < block_ptr[g + 1]) { ++cnt; ++q; }
          if (cnt) { bpr.push_back(bpr.back() + cnt); etar.push_back(eta[g]); }
        }
      }
      const int Gr = (int)etar.size();
      // starts: the predecessor's solution (round 0) or the stage's own last iterate
      for (int t = 0; t < n_tau; ++t) {
        const int f = t * n_lambda + l;
        const int src = (round == 0) ? (l ? f - 1 : -1) : f;
        if (src < 0) {
          CK(cudaMemsetAsync(b_red + (int64_t)t * Pr, 0, sizeof(double) * Pr, st));
          CK(cudaMemcpyAsync(z_st + (int64_t)t * n, y, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
          CK(cudaMemsetAsync(t_st + (int64_t)t * n, 0, sizeof(double) * n, st));
        } else {
          LK(launch_index_copy(beta + (int64_t)src * P, 0, d_idx, Pr, 1, b_red + (int64_t)t * Pr, 0, 0, st));
          CK(cudaMemcpyAsync(z_st + (int64_t)t * n, z + (int64_t)src * n, sizeof(double) * n,
                             cudaMemcpyDeviceToDevice, st));
          CK(cudaMemcpyAsync(t_st + (int64_t)t * n, theta + (int64_t)src * n, sizeof(double) * n,
                             cudaMemcpyDeviceToDevice, st));
        }
      }
      fsqr_design Xr = *Xd;
      Xr.p = ns;
      Xr.geno = ns ? g_red : nullptr;
      Xr.col_mean = m_red;
      Xr.col_sd = s_red;
      fsqr_opts o2 = *opts;
      if (opts->timeout_ms > 0) {  // one wall-clock budget for the whole path
        const double left = (double)opts->timeout_ms - (now_ms() - t0);
        o2.timeout_ms = (int64_t)std::max(1.0, left);
      }
      o2.warm = FSQR_WARM_GIVEN;
      o2.screen = 0;
      o2.eta = etar.data();
      o2.mu = mu;
      std::vector<double> lam_st(n_tau);
      for (int t = 0; t < n_tau; ++t) lam_st[t] = lambdas[t * n_lambda + l];
      memset(st_info.data(), 0, sizeof(fsqr_info) * n_tau);
      const int rc = fit_batch_impl(ctx, &Xr, y, n_tau, taus, 1, lam_st.data(), om_red, bpr.data(), Gr, &o2, b_red,
                                    z_st, t_st, st_info.data(), lmax.data(), nullptr);
      if (rc != FSQR_OK && rc != FSQR_ENOCONV && rc != FSQR_ETIMEOUT && rc != FSQR_ENUMERIC) return rc;
      // back to the full index space
      for (int t = 0; t < n_tau; ++t) {
        const int f = t * n_lambda + l;
        CK(cudaMemsetAsync(beta + (int64_t)f * P, 0, sizeof(double) * P, st));
        LK(launch_index_copy(b_red + (int64_t)t * Pr, 0, d_idx, Pr, 1, beta + (int64_t)f * P, 0, 1, st));
        CK(cudaMemcpyAsync(z + (int64_t)f * n, z_st + (int64_t)t * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(theta + (int64_t)f * n, t_st + (int64_t)t * n, sizeof(double) * n,
                           cudaMemcpyDeviceToDevice, st));
      }
      // the stop test's R_b over the left-out columns, on the full design
      TRY(prepare(ctx, Xd, &pr, opts->precision != FSQR_FP64));
      std::vector<double> sfull;
      TRY(full_xt(ctx, pr, t_st, n_tau, sfull));
      bool viol = false;
      for (int t = 0; t < n_tau; ++t) {
        const int f = t * n_lambda + l;
        double dmax = 0.0;
        for (int64_t s = 0; s < p; ++s) {
          if (keep[s]) continue;
          const int64_t j = 1 + c + s;
          const double d = fmax(fabs(sfull[(size_t)t * P + j]) - lambdas[f] * hom[j], 0.0) / lmax[t];
          if (d > opts->tol) { keep[s] = 1; viol = true; }
          dmax = fmax(dmax, d);
        }
        st_info[t].r_beta = fmax(st_info[t].r_beta, dmax);
        st_info[t].kkt = fmax(st_info[t].kkt, dmax);
        for (int64_t j = 0; j < P; ++j) sprev[(size_t)t * P + j] = sfull[(size_t)t * P + j];
      }
      if (!viol || round >= 8) {
        for (int t = 0; t < n_tau; ++t) {
          const int f = t * n_lambda + l;
          if (infos) {
            infos[f] = st_info[t];
            infos[f].t_setup_ms = 0.0;
            if (viol && infos[f].status == FSQR_OK) infos[f].status = FSQR_ENOCONV;
          }
          const int s_f = infos ? infos[f].status : FSQR_OK;
          if (worst == FSQR_OK && s_f != FSQR_OK) worst = s_f;
        }
        break;
      }
    }
  }
  if (infos)
    for (int f = 0; f < n_tau * n_lambda; ++f) infos[f].t_solve_ms = now_ms() - t0;
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
  if (X.mptr) {
    TRY(wsget(ctx, "p_qcorr", (size_t)npad * kMaxNB, &F.qcorr));
    CK(cudaMemsetAsync(F.qcorr, 0, sizeof(double) * npad * kMaxNB, st));
  }
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
    if (F.qcorr) LK(launch_miss_xb(NB, X, F, 0, bg, st));
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
  o->ridge = 0.0;
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
  if (opts && opts->screen) {
    if (opts->warm != FSQR_WARM_PATH) return fail(ctx, FSQR_EINVAL, "opts.screen needs FSQR_WARM_PATH");
    return fit_path_screened(ctx, X, y, n_tau, taus, n_lambda, lambdas, omega, block_ptr, G, opts, beta, z,
                             theta, infos);
  }
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

int fsqr_fit_lla(fsqr_ctx *ctx, const fsqr_design *X, const double *y, double tau, double lambda,
                 const double *omega, const int64_t *block_ptr, int G, int penalty, double a, int L,
                 const fsqr_opts *opts, double *beta, double *z, double *theta, double *lam_out,
                 fsqr_info *info) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  if (penalty != FSQR_PEN_SCAD && penalty != FSQR_PEN_MCP)
    return fail(ctx, FSQR_EINVAL, "penalty must be FSQR_PEN_SCAD or FSQR_PEN_MCP");
  if (!(a > (penalty == FSQR_PEN_SCAD ? 2.0 : 1.0)) || isinf(a))
    return fail(ctx, FSQR_EINVAL, "a must be finite and > %d for this penalty", penalty == FSQR_PEN_SCAD ? 2 : 1);
  if (L < 0) return fail(ctx, FSQR_EINVAL, "L must be >= 0");
  if (!(lambda > 0.0) || isinf(lambda)) return fail(ctx, FSQR_EINVAL, "lambda must be finite and > 0");
  if (!opts) return fail(ctx, FSQR_EINVAL, "opts is NULL");
  fsqr_info step{};
  std::vector<double> eta;
  // step 0: the weighted-l1 fit at lambda omega
  int rc = fit_batch_impl(ctx, X, y, 1, &tau, 1, &lambda, omega, block_ptr, G, opts, beta, z, theta, &step,
                          nullptr, &eta);
  if (rc != FSQR_OK && rc != FSQR_ENOCONV && rc != FSQR_ETIMEOUT) return rc;
  int iters = step.iters;
  const double lamnorm = step.lambda_max;
  const int64_t P = 1 + X->c + X->p;
  double *w;
  TRY(wsget(ctx, "lla_w", (size_t)P, &w));
  fsqr_opts o = *opts;
  o.eta = eta.data();
  o.warm = FSQR_WARM_GIVEN;
  o.max_group = 1;
  for (int l = 1; l <= L && (rc == FSQR_OK || rc == FSQR_ENOCONV); ++l) {
    // lambda omega'_j = omega_j p'_lambda(|beta~_j|), from the previous step's fit
    LK(launch_lla_weights(beta, omega, P, lambda, a, penalty, 1.0 / lambda, w, ctx->stream));
    rc = fit_batch_impl(ctx, X, y, 1, &tau, 1, &lambda, w, block_ptr, G, &o, beta, z, theta, &step, &lamnorm,
                        nullptr);
    if (rc != FSQR_OK && rc != FSQR_ENOCONV && rc != FSQR_ETIMEOUT) return rc;
    iters += step.iters;
  }
  if (lam_out) {
    if (L == 0) LK(launch_lla_weights(beta, omega, P, lambda, a, 0, 1.0, lam_out, ctx->stream));
    else LK(launch_lla_weights(w, nullptr, P, lambda, a, -1, lambda, lam_out, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  if (info) {
    *info = step;
    info->iters = iters;
  }
  return rc;
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
  LK(launch_summary(1, 1, n, P, y, ypad, xb, beta, omega, dt, dl, schk_use, tc_use, 0.0, summ, st));
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

int fsqr_path_stats(fsqr_ctx *ctx, const fsqr_design *Xd, const double *y, int B, const double *taus,
                    const double *beta, double *loss, int64_t *active, double *hbic) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  if (B < 1 || !y || !taus || !beta) return fail(ctx, FSQR_EINVAL, "B >= 1, y, taus and beta are required");
  for (int b = 0; b < B; ++b)
    if (!(taus[b] > 0.0 && taus[b] < 1.0)) return fail(ctx, FSQR_EINVAL, "tau must be in (0,1)");
  Prep pr;
  TRY(prepare(ctx, Xd, &pr, false));
  const int64_t n = pr.X.n, P = pr.X.P;
  double *q, *dt, *st;
  TRY(wsget(ctx, "ps_q", (size_t)B * n, &q));
  TRY(wsget(ctx, "ps_tau", (size_t)B, &dt));
  TRY(wsget(ctx, "ps_out", (size_t)2 * B, &st));
  TRY(predict_impl(ctx, pr, beta, B, q));
  CK(cudaMemcpyAsync(dt, taus, sizeof(double) * B, cudaMemcpyHostToDevice, ctx->stream));
  LK(launch_path_stats(q, y, dt, n, beta, P, B, st, ctx->stream));
  std::vector<double> h((size_t)2 * B);
  CK(cudaMemcpyAsync(h.data(), st, sizeof(double) * 2 * B, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  // HBIC with C_n = log p over the P - 1 candidate columns
  const double pen = (n > 1 ? log(log((double)n)) : 0.0) / (double)n * log((double)std::max<int64_t>(P - 1, 1));
  for (int b = 0; b < B; ++b) {
    if (loss) loss[b] = h[2 * b] / (double)n;
    if (active) active[b] = (int64_t)h[2 * b + 1];
    if (hbic) hbic[b] = log(h[2 * b]) + h[2 * b + 1] * pen;
  }
  return FSQR_OK;
}

int fsqr_interval_coverage(fsqr_ctx *ctx, const fsqr_design *Xd, const double *y, const double *beta_lo,
                           const double *beta_hi, double *coverage, double *width, int64_t *crossings) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  if (!y || !beta_lo || !beta_hi) return fail(ctx, FSQR_EINVAL, "y, beta_lo and beta_hi are required");
  Prep pr;
  TRY(prepare(ctx, Xd, &pr, false));
  const int64_t n = pr.X.n;
  double *q, *st;
  TRY(wsget(ctx, "cv_q", (size_t)2 * n, &q));
  TRY(wsget(ctx, "cv_out", 3, &st));
  TRY(predict_impl(ctx, pr, beta_lo, 1, q));
  TRY(predict_impl(ctx, pr, beta_hi, 1, q + n));
  LK(launch_coverage(q, q + n, y, n, st, ctx->stream));
  double h[3];
  CK(cudaMemcpyAsync(h, st, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (coverage) *coverage = h[0] / (double)n;
  if (width) *width = h[1] / (double)n;
  if (crossings) *crossings = (int64_t)h[2];
  return FSQR_OK;
}

int fsqr_wait_selftest(fsqr_ctx *ctx, int64_t budget_cycles, int arrive, int *wait_ok) {
  if (!ctx) return FSQR_EINVAL;
  TRY(enter(ctx));
  if (budget_cycles < 0 || budget_cycles > (int64_t)4000000000LL)
    return fail(ctx, FSQR_EINVAL, "budget_cycles must be in 0..4e9");
  int *d;
  TRY(wsget(ctx, "selftest", 2, &d));
  CK(cudaMemsetAsync(d, 0, 2 * sizeof(int), ctx->stream));
  LK(launch_wait_selftest((long long)budget_cycles, arrive ? 1 : 0, d, d + 1, ctx->stream));
  int h[2] = {0, 0};
  CK(cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (wait_ok) *wait_ok = h[1];
  if (h[0] != 0) return fail(ctx, FSQR_ETIMEOUT, "device wait ran out of its %lld-cycle budget (code %d)",
                             (long long)budget_cycles, h[0]);
  return FSQR_OK;
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
                "%d missing genotype entries: this entry point has no room for the per-column "
                "lists that mean imputation needs; use fsqr_lambda_max",
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
