// FS-QRPPA inner iteration kernels (Section 4, eq. fsppa_update, Algorithm 1).
//
// One iteration k of a group of NB fits is these launches on one stream:
//   [k_quantize]  theta^k -> int8 digit words            (mixed SIMT path only)
//   k_col         s = X~^T theta^k over every column, the stop-test distance
//                 for beta^k, and the block soft threshold of eq. beta_update
//                 -> beta^{k+1}, per-CTA lists of columns with beta^{k+1} != 0
//   [k_check]     stop test of the iterate w^k             (every K steps)
//   k_xbeta       partial sums of X~ beta^{k+1} over those columns only
//   k_vec         z^{k+1} (eq. z_update), r^{k+1}, theta^{k+1} (extrapolated
//                 dual step mu/(G+1)) and the reductions for the next test.
// The tensor-core path (k_tc.cu) replaces k_quantize, k_col and k_xbeta
// with its own kernels and applies the k_vec update inside its X~ beta pass.
// The G paper blocks survive as the per-block eta_g; the execution tiling
// (CTAs over contiguous column ranges) is independent of them.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "fsqr_device.cuh"
#include "fsqr_fixed.h"
#include "fsqr_internal.h"

namespace fsqr {

// ----------------------------------------------------------------- helpers

// Genotype code -> double without an FP64 conversion: 1 -> 1.0, 2 -> 2.0,
// anything else (0 or a missing code) -> 0.0.
__device__ __forceinline__ double g2d(uint32_t g) {
  uint32_t hi = (g == 1u) ? 0x3FF00000u : ((g == 2u) ? 0x40000000u : 0u);
  return __hiloint2double((int)hi, 0);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int block_of(const int64_t *__restrict__ bp, int G, int64_t j) {
  int lo = 0, hi = G;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(bp + mid) <= j) lo = mid; else hi = mid;
  }
  return lo;
}

// dist(s, lam * d|b|): |s - lam sign b| for b != 0, (|s| - lam)_+ for b = 0.
__device__ __forceinline__ double dist_l1(double s, double lam, double b) {
  if (b > 0.0) return fabs(s - lam);
  if (b < 0.0) return fabs(s + lam);
  return fmax(fabs(s) - lam, 0.0);
}


// Value of stored column entry (generic path, one sample).
__device__ __forceinline__ double stored_value(const Dsg &X, const uint8_t *col, int64_t i) {
  if (X.fmt == FSQR_DENSE_F64) return __ldg(reinterpret_cast<const double *>(col) + i);
  if (X.fmt == FSQR_INT8) return g2d(__ldg(col + i));
  uint32_t byte = __ldg(col + (i >> 2));
  return g2d((byte >> (2 * (i & 3))) & 3u);
}

__device__ __forceinline__ const uint8_t *col_ptr(const Dsg &X, int64_t j) {
  return X.geno + (j - 1 - X.c) * X.ld;
}

// ============================================================ column pass

// Generic per-column dot products (intercept, covariates, stored columns of
// any format): tot[b] = sum_i x_ij v_ib with v = vb (npad x NB interleaved).
template <int NB>
__device__ __forceinline__ void dot_generic(const Dsg &X, int64_t j, const double *__restrict__ vb,
                                            int lane, double *tot) {
#pragma unroll
  for (int b = 0; b < NB; ++b) tot[b] = 0.0;
  if (j == 0) return;  // intercept: a_0 = 0, its s comes from b_0 * sum(v)
  if (j <= X.c) {
    const double *cv = X.cov + (j - 1) * X.n;
    for (int64_t i = lane; i < X.n; i += 32) {
      double x = __ldg(cv + i);
#pragma unroll
      for (int b = 0; b < NB; ++b) tot[b] = fma(x, __ldg(vb + i * NB + b), tot[b]);
    }
  } else {
    const uint8_t *col = col_ptr(X, j);
    for (int64_t i = lane; i < X.n; i += 32) {
      double x = stored_value(X, col, i);
#pragma unroll
      for (int b = 0; b < NB; ++b) tot[b] = fma(x, __ldg(vb + i * NB + b), tot[b]);
    }
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) tot[b] = warp_sum(tot[b]);
}

// FP64 fast path: kACols consecutive stored columns, one warp, int8 codes.
template <int NB>
__device__ __forceinline__ void dot4_int8_f64(const Dsg &X, const uint8_t *const *cp,
                                              const double *__restrict__ vb, int lane,
                                              double (*tot)[NB]) {
  double acc[kACols][NB];
#pragma unroll
  for (int q = 0; q < kACols; ++q)
#pragma unroll
    for (int b = 0; b < NB; ++b) acc[q][b] = 0.0;
  const int64_t nch = (X.n + 15) >> 4;
  for (int64_t ch = lane; ch < nch; ch += 32) {
    uint4 gv[kACols];
#pragma unroll
    for (int q = 0; q < kACols; ++q) gv[q] = __ldcs(reinterpret_cast<const uint4 *>(cp[q]) + ch);
    const double *tp = vb + ch * 16 * NB;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        double tv[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) tv[b] = __ldg(tp + (4 * w + t) * NB + b);
#pragma unroll
        for (int q = 0; q < kACols; ++q) {
          uint32_t word = (w == 0) ? gv[q].x : (w == 1) ? gv[q].y : (w == 2) ? gv[q].z : gv[q].w;
          double gd = g2d((word >> (8 * t)) & 0xffu);
#pragma unroll
          for (int b = 0; b < NB; ++b) acc[q][b] = fma(gd, tv[b], acc[q][b]);
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kACols; ++q)
#pragma unroll
    for (int b = 0; b < NB; ++b) tot[q][b] = warp_sum(acc[q][b]);
}

// FP64 fast path for dense FP64 stored columns.
template <int NB>
__device__ __forceinline__ void dot4_dense_f64(const Dsg &X, const uint8_t *const *cp,
                                               const double *__restrict__ vb, int lane,
                                               double (*tot)[NB]) {
  double acc[kACols][NB];
#pragma unroll
  for (int q = 0; q < kACols; ++q)
#pragma unroll
    for (int b = 0; b < NB; ++b) acc[q][b] = 0.0;
  const int64_t nch = (X.n + 1) >> 1;
  for (int64_t ch = lane; ch < nch; ch += 32) {
    double2 xv[kACols];
#pragma unroll
    for (int q = 0; q < kACols; ++q) xv[q] = __ldcs(reinterpret_cast<const double2 *>(cp[q]) + ch);
    const bool tail = (2 * ch + 1 >= X.n);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      double tv[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) tv[b] = __ldg(vb + (2 * ch + t) * NB + b);
#pragma unroll
      for (int q = 0; q < kACols; ++q) {
        double x = (t == 0) ? xv[q].x : (tail ? 0.0 : xv[q].y);
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[q][b] = fma(x, tv[b], acc[q][b]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kACols; ++q)
#pragma unroll
    for (int b = 0; b < NB; ++b) tot[q][b] = warp_sum(acc[q][b]);
}

// Mixed fast path: exact integer dot products of int8 genotype codes with the
// D int8 digits of theta (DP4A, int32 accumulate), combined exactly in int64.
// Missing codes must not occur (the host rejects them for this path).
template <int NB, int D>
__device__ __forceinline__ void dot4_int8_digits(const Dsg &X, const uint8_t *const *cp,
                                                 const int32_t *__restrict__ sdig, int64_t n4p,
                                                 int lane, long long (*tot)[NB]) {
  int acc[kACols][NB][D];
#pragma unroll
  for (int q = 0; q < kACols; ++q)
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int d = 0; d < D; ++d) acc[q][b][d] = 0;
  const int64_t nch = (X.n + 15) >> 4;
  for (int64_t ch = lane; ch < nch; ch += 32) {
    uint4 cur[kACols];
#pragma unroll
    for (int q = 0; q < kACols; ++q) cur[q] = __ldcs(reinterpret_cast<const uint4 *>(cp[q]) + ch);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int4 tw = *reinterpret_cast<const int4 *>(sdig + (int64_t)(b * D + d) * n4p + 4 * ch);
#pragma unroll
        for (int q = 0; q < kACols; ++q) {
          int a = acc[q][b][d];
          a = __dp4a((int)cur[q].x, tw.x, a);
          a = __dp4a((int)cur[q].y, tw.y, a);
          a = __dp4a((int)cur[q].z, tw.z, a);
          a = __dp4a((int)cur[q].w, tw.w, a);
          acc[q][b][d] = a;
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kACols; ++q)
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      long long v = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) v += (long long)acc[q][b][d] << (7 * (D - 1 - d));
      tot[q][b] = warp_sum_ll(v);
    }
}

// The column pass. CTA c owns columns [c*T, min(P, (c+1)*T)); warp w takes
// groups of kACols consecutive columns starting at c*T + w*kACols.
//   A_PROX     : iteration step k = *it_base + off of the group F
//   A_XT       : s_out[j*NB+b] = x~_j^T v_b, v = vec, vsum[b] = sum_i v_ib
//   A_XT_BLOCK : NB = 1, column j uses v = vec + block(j)*npad, vsum[block(j)]
//   A_LIST     : lists and constant terms of beta_in, no data read
template <int NB, int MODE, int D>
__global__ void __launch_bounds__(kAThreads, ((D > 0 && NB * D <= 12) ? 2 : 1))
    k_col(Dsg X, Fits F, int off, const double *__restrict__ vec, const double *__restrict__ vsum,
          double *__restrict__ s_out, const double *__restrict__ beta_in) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = F.T;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j0 = (int64_t)blockIdx.x * T;
  const int64_t j1 = min(X.P, j0 + (int64_t)T);
  uint8_t *flags = smem;
  int32_t *sdig = reinterpret_cast<int32_t *>(smem + ((T + 15) & ~15));
  __shared__ double sS[kMaxNB];
  __shared__ double sScale[kMaxNB];
  __shared__ int sIdle[kMaxNB];
  __shared__ double red_rb[kAWarps][32];
  __shared__ double red_ct[kAWarps][32];
  __shared__ double red_wm[kAWarps][32];
  __shared__ int scan[kAThreads];

  int k = 0;
  const double *bcur = beta_in;
  double *bnxt = nullptr;
  if (MODE == A_PROX) {
    k = *F.it_base + off;
    bcur = F.beta[k & 1];
    bnxt = F.beta[(k & 1) ^ 1];
  }
  const double *vb = (MODE == A_PROX) ? F.theta : vec;
  if (threadIdx.x < NB) {
    const int b = threadIdx.x;
    double S = 0.0;
    if (MODE == A_PROX) {
      S = F.tot_c[k & 1][b * kCPartials + 2];
      sIdle[b] = (b >= F.nb) || (F.done[b] >= 0);
      sScale[b] = D ? F.scale[b] : 1.0;
    } else if (MODE == A_XT) {
      S = vsum[b];
      sIdle[b] = 0;
    } else if (MODE == A_LIST) {
      sIdle[b] = (b >= F.nb);
    } else {
      sIdle[b] = 0;
    }
    sS[b] = S;
  }
  if (MODE == A_PROX || MODE == A_LIST)
    for (int t = threadIdx.x; t < T; t += kAThreads) flags[t] = 0;
  if (D > 0) {  // stage the digit words of all NB fits
    const int64_t words = (int64_t)NB * D * F.n4p;
    const int4 *src = reinterpret_cast<const int4 *>(F.digits);
    int4 *dst = reinterpret_cast<int4 *>(sdig);
    for (int64_t t = threadIdx.x; t < words / 4; t += kAThreads) dst[t] = __ldcg(src + t);
  }
  __syncthreads();

  const int mycol = lane / NB, myb = lane % NB;
  const bool lane_has = lane < kACols * NB;
  double rbl = 0.0, ctl = 0.0, wml = 0.0;

  for (int64_t jg = j0 + warp * kACols; jg < j1; jg += kAWarps * kACols) {
    double tot[kACols][NB];
    if (MODE == A_LIST) {
#pragma unroll
      for (int q = 0; q < kACols; ++q)
#pragma unroll
        for (int b = 0; b < NB; ++b) tot[q][b] = 0.0;
    } else if (jg <= X.c || MODE == A_XT_BLOCK || (X.fmt == FSQR_2BIT && D == 0) ||
               (jg + kACols > j1 && X.fmt == FSQR_DENSE_F64)) {
#pragma unroll
      for (int q = 0; q < kACols; ++q) {
        const int64_t jq = jg + q;
        double t1[NB];
        if (jq < j1) {
          const double *vq = vb;
          if (MODE == A_XT_BLOCK) vq = vec + (int64_t)block_of(F.block_ptr, F.G, jq) * F.npad;
          dot_generic<NB>(X, jq, vq, lane, t1);
        } else {
#pragma unroll
          for (int b = 0; b < NB; ++b) t1[b] = 0.0;
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) tot[q][b] = t1[b];
      }
    } else {
      const uint8_t *cp[kACols];
#pragma unroll
      for (int q = 0; q < kACols; ++q) cp[q] = col_ptr(X, (jg + q < j1) ? jg + q : jg);
      if (D > 0) {
        long long it[kACols][NB];
        dot4_int8_digits<NB, (D > 0 ? D : 1)>(X, cp, sdig, F.n4p, lane, it);
#pragma unroll
        for (int q = 0; q < kACols; ++q)
#pragma unroll
          for (int b = 0; b < NB; ++b)
            tot[q][b] = (double)it[q][b] * (sScale[b] * ldexp(1.0, -7 * D));
      } else if (X.fmt == FSQR_DENSE_F64) {
        dot4_dense_f64<NB>(X, cp, vb, lane, tot);
      } else {
        dot4_int8_f64<NB>(X, cp, vb, lane, tot);
      }
    }

    // Epilogue: lane q*NB + b owns column jg+q and fit b.
    double mydot = 0.0;
#pragma unroll
    for (int q = 0; q < kACols; ++q)
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (lane == q * NB + b) mydot = tot[q][b];
    const int64_t jq = jg + mycol;
    bool act = false;
    if (lane_has && jq < j1) {
      const double aj = __ldg(X.a + jq), bj = __ldg(X.b + jq);
      // mean imputation: the missing entries of a stored column read as 0,
      // so their share b_j v_i of the constant part is taken back out
      if (MODE == A_XT) {
        const double mc = jq > X.c ? miss_dot(X, jq - 1 - X.c, vb, NB, myb) : 0.0;
        s_out[jq * NB + myb] = aj * mydot + bj * (sS[myb] - mc);
      } else if (MODE == A_XT_BLOCK) {
        const int g = block_of(F.block_ptr, F.G, jq);
        const double mc = jq > X.c ? miss_dot(X, jq - 1 - X.c, vec + (int64_t)g * F.npad, 1, 0) : 0.0;
        s_out[jq] = aj * mydot + bj * (__ldg(vsum + g) - mc);
      } else if (MODE == A_LIST) {
        const double bv = bcur[jq * NB + myb];
        if (!sIdle[myb]) {
          ctl = fma(bj, bv, ctl);
          act = (bv != 0.0) && jq >= 1;
          if (jq > X.c) wml = fmax(wml, fabs(aj * bv));
        }
      } else {  // A_PROX
        const double mc = jq > X.c ? miss_dot(X, jq - 1 - X.c, vb, NB, myb) : 0.0;
        const double s = aj * mydot + bj * (sS[myb] - mc);
        const double om = __ldg(F.omega + jq);
        const double lamj = F.lam[myb] * om;
        const double gj = F.ridge * om;  // elastic-net quadratic weight (0: weighted l1)
        const double bo = bcur[jq * NB + myb];
        if (!sIdle[myb]) {
          if (jq >= 1) rbl = fmax(rbl, dist_l1(gj == 0.0 ? s : s - gj * bo, lamj, bo));
          const int g = block_of(F.block_ptr, F.G, jq);
          const double eta = __ldg(F.eta + g);
          const double ie = gj == 0.0 ? __ldg(F.inv_eta + g) : 1.0 / (eta + gj);
          // eq. beta_update: (1/eta)[(eta b + s - lam)_+ - (-eta b - s - lam)_+]
          // (1/(eta + gamma_j) with the elastic-net term)
          const double av = eta * bo + s;
          const double bn = (fmax(av - lamj, 0.0) - fmax(-av - lamj, 0.0)) * ie;
          bnxt[jq * NB + myb] = bn;
          ctl = fma(bj, bn, ctl);
          act = (bn != 0.0) && jq >= 1;
          if (jq > X.c) wml = fmax(wml, fabs(aj * bn));
        }
      }
    }
    if (MODE == A_PROX || MODE == A_LIST) {
      const unsigned m = __ballot_sync(0xffffffffu, act);
      if (lane < kACols && jg + lane < j1) {
        const unsigned colmask = ((1u << NB) - 1u) << (lane * NB);
        if (m & colmask) flags[jg + lane - j0] = 1;
      }
    }
  }

  if (MODE != A_PROX && MODE != A_LIST) return;

  // Per-CTA reductions in a fixed order (deterministic).
  red_rb[warp][lane] = rbl;
  red_ct[warp][lane] = ctl;
  red_wm[warp][lane] = wml;
  __syncthreads();
  if (threadIdx.x < NB) {
    const int b = threadIdx.x;
    double m = 0.0, c = 0.0, wm = 0.0;
    for (int w = 0; w < kAWarps; ++w)
      for (int q = 0; q < kACols; ++q) {
        m = fmax(m, red_rb[w][q * NB + b]);
        c += red_ct[w][q * NB + b];
        wm = fmax(wm, red_wm[w][q * NB + b]);
      }
    F.a_rb[blockIdx.x * NB + b] = m;
    F.a_ct[blockIdx.x * NB + b] = c;
    if (F.a_wmax) F.a_wmax[blockIdx.x * NB + b] = wm;
  }
  // Ordered compaction of the active flags.
  const int per = (T + kAThreads - 1) / kAThreads;
  const int t0 = min(T, (int)threadIdx.x * per), t1 = min(T, t0 + per);
  int cnt = 0;
  for (int t = t0; t < t1; ++t) cnt += flags[t];
  scan[threadIdx.x] = cnt;
  __syncthreads();
  for (int o = 1; o < kAThreads; o <<= 1) {
    int v = (threadIdx.x >= (unsigned)o) ? scan[threadIdx.x - o] : 0;
    __syncthreads();
    scan[threadIdx.x] += v;
    __syncthreads();
  }
  int pos = scan[threadIdx.x] - cnt;
  int *lst = F.a_list + (int64_t)blockIdx.x * T;
  for (int t = t0; t < t1; ++t)
    if (flags[t]) lst[pos++] = (int)(j0 + t);
  if (threadIdx.x == kAThreads - 1) F.a_cnt[blockIdx.x] = scan[kAThreads - 1];
  col_finalize<NB>(F);
}

size_t col_pass_smem(int mode, const Fits &F, int NB) {
  size_t s = ((size_t)F.T + 15) & ~(size_t)15;
  if (mode == A_PROX && F.mixed) s += (size_t)NB * F.D * F.n4p * 4;
  return s;
}

// Largest dynamic shared memory opted in per instantiation of k_col.
template <int NB, int MODE, int D>
size_t g_col_opted = 48 * 1024;

template <int NB, int MODE, int D>
static cudaError_t col_pass_t(const Dsg &X, const Fits &F, int off, const double *vec,
                              const double *vsum, double *s_out, const double *beta_in,
                              cudaStream_t s) {
  const size_t smem = col_pass_smem(MODE, F, NB);
  auto kern = k_col<NB, MODE, D>;
  // The opt-in is raised outside graph capture (col_pass_occupancy runs
  // first with an upper bound); here it is only raised when still needed.
  if (smem > g_col_opted<NB, MODE, D>) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    g_col_opted<NB, MODE, D> = smem;
  }
  kern<<<F.gridA, kAThreads, smem, s>>>(X, F, off, vec, vsum, s_out, beta_in);
  return cudaGetLastError();
}

template <int NB>
static cudaError_t col_pass_nb(int mode, const Dsg &X, const Fits &F, int off, const double *vec,
                               const double *vsum, double *s_out, const double *beta_in,
                               cudaStream_t s) {
  switch (mode) {
    case A_PROX:
      if (!F.mixed) return col_pass_t<NB, A_PROX, 0>(X, F, off, vec, vsum, s_out, beta_in, s);
      if (F.D == 3) return col_pass_t<NB, A_PROX, 3>(X, F, off, vec, vsum, s_out, beta_in, s);
      if (F.D == 4) return col_pass_t<NB, A_PROX, 4>(X, F, off, vec, vsum, s_out, beta_in, s);
      if (F.D == 5) return col_pass_t<NB, A_PROX, 5>(X, F, off, vec, vsum, s_out, beta_in, s);
      return cudaErrorInvalidValue;
    case A_XT:
      return col_pass_t<NB, A_XT, 0>(X, F, off, vec, vsum, s_out, beta_in, s);
    case A_LIST:
      return col_pass_t<NB, A_LIST, 0>(X, F, off, vec, vsum, s_out, beta_in, s);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_col_pass(int mode, int NB, const Dsg &X, const Fits &F, int off,
                            const double *vec, const double *vsum, double *s_out,
                            const double *beta_in, cudaStream_t s) {
  if (mode == A_XT_BLOCK) return col_pass_t<1, A_XT_BLOCK, 0>(X, F, off, vec, vsum, s_out, beta_in, s);
  switch (NB) {
    case 1: return col_pass_nb<1>(mode, X, F, off, vec, vsum, s_out, beta_in, s);
    case 2: return col_pass_nb<2>(mode, X, F, off, vec, vsum, s_out, beta_in, s);
    case 3: return col_pass_nb<3>(mode, X, F, off, vec, vsum, s_out, beta_in, s);
    case 4: return col_pass_nb<4>(mode, X, F, off, vec, vsum, s_out, beta_in, s);
    case 8: return col_pass_nb<8>(mode, X, F, off, vec, vsum, s_out, beta_in, s);
    default: return cudaErrorInvalidValue;
  }
}

// ------------------------------------ X~^T u with exact integer products
//
// s_out[j] = x~_j^T u_g(j) for one vector per block (the power method's
// X~_g^T u_g; lambda_max with G = 1). u_g is given both in FP64 (u) and as
// 52-bit fixed point q_i = hi_i 2^26 + lo_i with unit[g] (k_fix_seg over the
// blocks' npad-long segments, so entries i >= n are 0). For stored int8 and
// 2-bit columns, sum_i x_ij q_i is exact in two int64 sums (codes 0/1/2, a
// missing code read as 0 and its share b_j u_i taken back out); one warp takes
// 4 consecutive columns of one block. The intercept, the covariates and the
// groups that straddle a block boundary or the end take the FP64 dot.
__global__ void __launch_bounds__(256) k_xtv_int(Dsg X, const int64_t *__restrict__ bp, int G,
                                                 const double *__restrict__ u, const int2 *__restrict__ q,
                                                 const double *__restrict__ unit, const double *__restrict__ usum,
                                                 int64_t npad, double *__restrict__ s_out) {
  const int lane = threadIdx.x & 31;
  const int64_t ngrp = (X.P + 3) >> 2;
  const int64_t nch = (X.n + 15) >> 4;  // 16-sample chunks; 16 nch <= npad
  for (int64_t gi = (int64_t)blockIdx.x * kAWarps + (threadIdx.x >> 5); gi < ngrp;
       gi += (int64_t)gridDim.x * kAWarps) {
    const int64_t j0 = gi * 4, j1 = min(X.P, j0 + 4);
    const int g0 = block_of(bp, G, j0);
    const bool fast = j0 > X.c && j1 - j0 == 4 && block_of(bp, G, j1 - 1) == g0 && X.fmt != FSQR_DENSE_F64;
    double d[4] = {0.0, 0.0, 0.0, 0.0};
    if (fast) {
      long long ahi[4] = {0, 0, 0, 0}, alo[4] = {0, 0, 0, 0};
      const int4 *qg = reinterpret_cast<const int4 *>(q + (int64_t)g0 * npad);
      const uint8_t *cp[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) cp[k] = col_ptr(X, j0 + k);
      for (int64_t ch = lane; ch < nch; ch += 32) {
        // codes of samples 16ch .. 16ch+15 as four 32-bit words per column
        uint32_t cw[4][4];
        if (X.fmt == FSQR_INT8) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint4 t = __ldcs(reinterpret_cast<const uint4 *>(cp[k]) + ch);
            const uint32_t tw[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int w = 0; w < 4; ++w) cw[k][w] = tw[w] & __vcmpleu4(tw[w], 0x02020202u);  // codes > 2 -> 0
          }
        } else {  // 2-bit: 16 samples in 4 bytes; widen to one byte per code, code 3 -> 0
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t t = __ldcs(reinterpret_cast<const unsigned *>(cp[k]) + ch);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              const uint32_t b = (t >> (8 * w)) & 0xffu;
              uint32_t e = (b & 3u) | ((b >> 2 & 3u) << 8) | ((b >> 4 & 3u) << 16) | ((b >> 6) << 24);
              cw[k][w] = e & ~__vcmpeq4(e, 0x03030303u);
            }
          }
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int4 qa = __ldg(qg + ch * 8 + 2 * w);      // samples 4w, 4w+1: (lo, hi), (lo, hi)
          const int4 qb = __ldg(qg + ch * 8 + 2 * w + 1);  // samples 4w+2, 4w+3
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t x = cw[k][w];
            const int c0 = (int)(x & 0xffu), c1 = (int)(x >> 8 & 0xffu), c2 = (int)(x >> 16 & 0xffu),
                      c3 = (int)(x >> 24);
            ahi[k] += (long long)c0 * qa.y + (long long)c1 * qa.w + (long long)c2 * qb.y + (long long)c3 * qb.w;
            alo[k] += (long long)c0 * qa.x + (long long)c1 * qa.z + (long long)c2 * qb.x + (long long)c3 * qb.z;
          }
        }
      }
      const double un = __ldg(unit + g0);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        d[k] = un * fma((double)warp_sum_ll(ahi[k]), 67108864.0, (double)warp_sum_ll(alo[k]));
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        double t = 0.0;
        if (j0 + k < j1) dot_generic<1>(X, j0 + k, u + (int64_t)block_of(bp, G, j0 + k) * npad, lane, &t);
        d[k] = t;
      }
    }
    if (lane < (int)(j1 - j0)) {
      const int64_t j = j0 + lane;
      const int g = block_of(bp, G, j);
      const double dj = lane == 0 ? d[0] : lane == 1 ? d[1] : lane == 2 ? d[2] : d[3];
      const double mc = j > X.c ? miss_dot(X, j - 1 - X.c, u + (int64_t)g * npad, 1, 0) : 0.0;
      s_out[j] = __ldg(X.a + j) * dj + __ldg(X.b + j) * (__ldg(usum + g) - mc);
    }
  }
}

cudaError_t launch_xtv_int(const Dsg &X, const int64_t *block_ptr, int G, const double *u, const int2 *q,
                           const double *unit, const double *usum, int64_t npad, double *s_out, cudaStream_t s) {
  if (X.P == 0) return cudaSuccess;
  const int64_t ngrp = (X.P + 3) >> 2;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (ngrp + kAWarps - 1) / kAWarps;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
  k_xtv_int<<<grid, kAThreads, 0, s>>>(X, block_ptr, G, u, q, unit, usum, npad, s_out);
  return cudaGetLastError();
}

// ============================================================= X~ beta

// Partial sums of X~ beta over the active columns listed by the column pass:
// CTA (rc, sp) covers rows [rc*kBRows, +kBRows) and the sp-th slice of the
// concatenated per-CTA lists. Only the slope part a_j x_ij beta_j is summed
// here; the constant part sum_j b_j beta_j comes from the column pass.
// CTA (0,0) also totals the constant terms and records the split count.
template <int NB>
__global__ void __launch_bounds__(kBThreads)
    k_xbeta(Dsg X, Fits F, int off, const double *__restrict__ beta_in) {
  extern __shared__ int spre[];  // gridA + 1 prefix sums
  const double *beta = beta_in;
  if (beta == nullptr) {
    const int k = *F.it_base + off;
    beta = F.beta[(k & 1) ^ 1];
  }
  // prefix of the per-CTA counts from the column pass's last CTA
  const int gA = F.gridA;
  for (int t = threadIdx.x; t <= gA; t += kBThreads) spre[t] = __ldcg(F.a_pre + t);
  __syncthreads();
  const int A = spre[gA];
  const int S = max(1, min(kBMaxSplits, A / kBMinColsPerSplit));
  if (blockIdx.x == 0 && blockIdx.y == 0) {
    if (threadIdx.x < NB) F.meta_d[threadIdx.x] = F.tot_a[threadIdx.x * 3 + 1];
    if (threadIdx.x == 0) { F.meta_i[0] = S; F.meta_i[1] = A; }
  }
  if ((int)blockIdx.y >= S) return;
  const int a0 = (int)((int64_t)A * blockIdx.y / S), a1 = (int)((int64_t)A * (blockIdx.y + 1) / S);
  const int64_t i0 = (int64_t)blockIdx.x * kBRows + (int64_t)threadIdx.x * kBRowsPerThread;
  double acc[kBRowsPerThread][NB];
#pragma unroll
  for (int r = 0; r < kBRowsPerThread; ++r)
#pragma unroll
    for (int b = 0; b < NB; ++b) acc[r][b] = 0.0;
  // first bucket containing a0
  int bk = 0;
  {
    int lo = 0, hi = gA;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (spre[mid] <= a0) lo = mid; else hi = mid;
    }
    bk = lo;
  }
  const bool rows_ok = i0 < X.n;
  for (int a = a0; a < a1; ++a) {
    while (a >= spre[bk + 1]) ++bk;
    const int64_t j = F.a_list[(int64_t)bk * F.T + (a - spre[bk])];
    const double aj = __ldg(X.a + j);
    double w[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) w[b] = aj * __ldg(beta + j * NB + b);
    if (!rows_ok) continue;
    double x[kBRowsPerThread];
    if (j <= X.c) {
      const double *cv = X.cov + (j - 1) * X.n;
#pragma unroll
      for (int r = 0; r < kBRowsPerThread; ++r) x[r] = (i0 + r < X.n) ? __ldg(cv + i0 + r) : 0.0;
    } else if (X.fmt == FSQR_INT8) {
      const uint2 g = __ldg(reinterpret_cast<const uint2 *>(col_ptr(X, j) + i0));
#pragma unroll
      for (int r = 0; r < kBRowsPerThread; ++r)
        x[r] = g2d(((r < 4 ? g.x : g.y) >> (8 * (r & 3))) & 0xffu);
    } else if (X.fmt == FSQR_2BIT) {
      const uint16_t g = __ldg(reinterpret_cast<const uint16_t *>(col_ptr(X, j) + (i0 >> 2)));
#pragma unroll
      for (int r = 0; r < kBRowsPerThread; ++r) x[r] = g2d((g >> (2 * r)) & 3u);
    } else {
      const double *cv = reinterpret_cast<const double *>(col_ptr(X, j));
#pragma unroll
      for (int r = 0; r < kBRowsPerThread; ++r) x[r] = (i0 + r < X.n) ? __ldg(cv + i0 + r) : 0.0;
    }
#pragma unroll
    for (int r = 0; r < kBRowsPerThread; ++r)
#pragma unroll
      for (int b = 0; b < NB; ++b) acc[r][b] = fma(x[r], w[b], acc[r][b]);
  }
  double *out = F.xb_part + (int64_t)blockIdx.y * F.npad * NB;
#pragma unroll
  for (int r = 0; r < kBRowsPerThread; ++r)
    if (i0 + r < F.npad)
#pragma unroll
      for (int b = 0; b < NB; ++b) out[(i0 + r) * NB + b] = acc[r][b];
}

// Mixed path: exact integer X~ beta over the active stored columns.
// w_jb = a_j beta_jb is rounded to a 7*DW-bit fixed-point integer W_jb with
// the per-fit scale 2^(E_b+1) (max_j |w_jb| < 2^E_b over the stored active
// columns, from the column pass's totals), split into DW balanced int8
// digits. For 4 active columns at a time each thread gathers the genotype
// bytes of its 2 rows and byte-transposes them so that one DP4A forms
// sum_{4 columns} g_ij * digit; per-digit int32 sums are combined exactly in
// int64 per (split, row, fit). The covariates and the constant term are
// added in FP64 by the vector kernel.
// CTA (rc, sp): rows [rc*512, +512) (256 threads x 2 rows), split sp of the
// concatenated active lists, staged kXIChunk columns at a time.
constexpr int kXIRows = 512;
constexpr int kDWMax = 6;
constexpr int kXIChunk = 512;
constexpr int kXIMaxSplits = 32;

template <int NB, int DW>
__global__ void __launch_bounds__(256, 2)
    k_xbeta_int(Dsg X, Fits F, int off, const double *__restrict__ beta_in) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  int *spre = reinterpret_cast<int *>(sm_raw);  // gridA + 1
  __shared__ double sInv[kMaxNB];
  const double *beta = beta_in;
  if (beta == nullptr) {
    const int k = *F.it_base + off;
    beta = F.beta[(k & 1) ^ 1];
  }
  const int gA = F.gridA;
  for (int t = threadIdx.x; t <= gA; t += blockDim.x) spre[t] = __ldcg(F.a_pre + t);
  if (threadIdx.x < NB) {
    const int b = threadIdx.x;
    const double m = F.tot_a[b * 3 + 2];
    int E = 0;
    if (m > 0.0) frexp(m, &E);
    const double scale = (m > 0.0) ? ldexp(1.0, E + 1) : 1.0;
    sInv[b] = ldexp(1.0, 7 * DW) / scale;
    if (blockIdx.x == 0 && blockIdx.y == 0) {
      F.meta_d[b] = F.tot_a[b * 3 + 1];
      F.meta_d[kMaxNB + b] = scale;
    }
  }
  __syncthreads();
  const int A = spre[gA];
  const int S = max(1, min(kXIMaxSplits, A / kBMinColsPerSplit));
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) { F.meta_i[0] = S; F.meta_i[1] = A; }
  if ((int)blockIdx.y >= S) return;
  const int a0 = (int)((int64_t)A * blockIdx.y / S), a1 = (int)((int64_t)A * (blockIdx.y + 1) / S);
  // per chunk: column of each slot (or -1) and the digit words Wd[g][b][d]
  // (byte q = digit of column q of group g)
  int *gcol = spre + gA + 1;
  uint32_t *wd = reinterpret_cast<uint32_t *>(gcol + kXIChunk);
  uint8_t *wb = reinterpret_cast<uint8_t *>(wd);
  const int64_t i0 = (int64_t)blockIdx.x * kXIRows + threadIdx.x * 2;
  int acc[2][NB][DW];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int d = 0; d < DW; ++d) acc[r][b][d] = 0;
  for (int c0 = a0; c0 < a1; c0 += kXIChunk) {
    const int cnt = min(kXIChunk, a1 - c0);
    const int ng = (cnt + 3) / 4;
    __syncthreads();  // previous chunk fully consumed
    for (int t = threadIdx.x; t < 4 * ng; t += blockDim.x) {
      int j = -1;
      if (t < cnt) {
        const int a = c0 + t;
        int lo = 0, hi = gA;  // bucket: spre[lo] <= a < spre[lo+1]
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (spre[mid] <= a) lo = mid; else hi = mid;
        }
        j = F.a_list[(int64_t)lo * F.T + (a - spre[lo])];
        if (j <= X.c) j = -1;  // covariates are summed in FP64 by k_vec
      }
      gcol[t] = j;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 4 * ng * NB; t += blockDim.x) {
      const int slot = t / NB, b = t - slot * NB;
      const int j = gcol[slot];
      long long W = 0;
      if (j >= 0) W = fixed_point(__ldg(X.a + j) * beta[(int64_t)j * NB + b] * sInv[b]);
      int dig[kDWMax];
#pragma unroll
      for (int d = DW - 1; d >= 1; --d) {
        const int tt = (int)(((W + 64) & 127) - 64);
        dig[d] = tt;
        W = (W - tt) >> 7;
      }
      dig[0] = (int)W;
      const int g = slot >> 2, q = slot & 3;
#pragma unroll
      for (int d = 0; d < DW; ++d) wb[(((size_t)g * NB + b) * DW + d) * 4 + q] = (uint8_t)(dig[d] & 0xff);
    }
    __syncthreads();
    if (i0 < X.n) {
      for (int g = 0; g < ng; ++g) {
        uint32_t c2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = gcol[4 * g + q];
          c2[q] = (j >= 0) ? (uint32_t)__ldg(reinterpret_cast<const uint16_t *>(X.geno + (j - 1 - X.c) * X.ld + i0)) : 0u;
        }
        // rows i0, i0+1 as (column 0..3) byte vectors
        const uint32_t x01 = c2[0] | (c2[1] << 16), x23 = c2[2] | (c2[3] << 16);
        const uint32_t rw0 = __byte_perm(x01, x23, 0x6420), rw1 = __byte_perm(x01, x23, 0x7531);
        const uint32_t *wg = wd + (size_t)g * NB * DW;
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int d = 0; d < DW; ++d) {
            const int wv = (int)wg[b * DW + d];
            acc[0][b][d] = __dp4a((int)rw0, wv, acc[0][b][d]);
            acc[1][b][d] = __dp4a((int)rw1, wv, acc[1][b][d]);
          }
      }
    }
  }
  long long *out = F.xb_ipart + (int64_t)blockIdx.y * F.npad * NB;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int64_t i = i0 + r;
    if (i < F.npad)
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        long long v = 0;
#pragma unroll
        for (int d = 0; d < DW; ++d) v += (long long)acc[r][b][d] << (7 * (DW - 1 - d));
        out[i * NB + b] = v;
      }
  }
}

// Shared memory of k_xbeta_int: prefix (gridA+1 ints), the column slots of
// one chunk and their digit words.
static size_t xbeta_int_smem(const Fits &F, int NB) {
  return (size_t)(F.gridA + 1) * 4 + (size_t)kXIChunk * 4 + (size_t)kXIChunk * NB * F.DW + 64;
}

template <int NB, int DW>
size_t g_xi_opted = 48 * 1024;

template <int NB, int DW>
static cudaError_t xbeta_int_t(const Dsg &X, const Fits &F, int off, const double *beta_in,
                               cudaStream_t s) {
  const size_t smem = xbeta_int_smem(F, NB);
  if (smem > g_xi_opted<NB, DW>) {
    cudaError_t e = cudaFuncSetAttribute(k_xbeta_int<NB, DW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    g_xi_opted<NB, DW> = smem;
  }
  dim3 grid((unsigned)((X.n + kXIRows - 1) / kXIRows), kXIMaxSplits);
  k_xbeta_int<NB, DW><<<grid, 256, smem, s>>>(X, F, off, beta_in);
  return cudaGetLastError();
}

template <int NB>
static cudaError_t xbeta_t(const Dsg &X, const Fits &F, int off, const double *beta_in,
                           cudaStream_t s) {
  if (F.mixed) {
    if (F.DW == 6) return xbeta_int_t<NB, 6>(X, F, off, beta_in, s);
    return cudaErrorInvalidValue;
  }
  dim3 grid((unsigned)((X.n + kBRows - 1) / kBRows), kBMaxSplits);
  size_t smem = (size_t)(F.gridA + 1) * sizeof(int);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_xbeta<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_xbeta<NB><<<grid, kBThreads, smem, s>>>(X, F, off, beta_in);
  return cudaGetLastError();
}

cudaError_t launch_xbeta(int NB, const Dsg &X, const Fits &F, int off, const double *beta_in,
                         cudaStream_t s) {
  switch (NB) {
    case 1: return xbeta_t<1>(X, F, off, beta_in, s);
    case 2: return xbeta_t<2>(X, F, off, beta_in, s);
    case 3: return xbeta_t<3>(X, F, off, beta_in, s);
    case 4: return xbeta_t<4>(X, F, off, beta_in, s);
    case 8: return xbeta_t<8>(X, F, off, beta_in, s);
    default: return cudaErrorInvalidValue;
  }
}

// ================================================== quantise theta (mixed)

// theta^k_b / scale_b rounded to a 7D-bit fixed-point integer X, written as D
// balanced base-128 digits t_0..t_{D-1} (X = sum_d t_d 128^{D-1-d}, each in
// [-64, 64]) packed four samples per int32 word. scale_b = 2^(E+1) with
// max_i |theta_ib| < 2^E, so |X| <= 2^(7D-1).
template <int NB>
__global__ void __launch_bounds__(256) k_quantize(Fits F, int off) {
  const int k = *F.it_base + off;
  __shared__ double sInv[kMaxNB];
  if (threadIdx.x < NB) {
    const int b = threadIdx.x;
    const double m = F.tot_c[k & 1][b * kCPartials + 3];
    int E = 0;
    if (m > 0.0) frexp(m, &E);  // m = f 2^E, f in [0.5, 1)
    const double scale = (m > 0.0) ? ldexp(1.0, E + 1) : 1.0;
    sInv[b] = ldexp(1.0, 7 * F.D) / scale;
    if (blockIdx.x == 0) F.scale[b] = scale;
  }
  __syncthreads();
  const int64_t rows = 4 * F.n4p;  // == npad
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = (int)(g / rows);
  const int64_t i = g - (int64_t)b * rows;
  const bool ok = b < NB;
  long long Xq = 0;
  if (ok) Xq = fixed_point(F.theta[i * NB + b] * sInv[b]);
  int dig[6];
#pragma unroll
  for (int d = 5; d >= 0; --d) {
    if (d < F.D) {
      if (d == 0) {
        dig[0] = (int)Xq;
      } else {
        const int t = (int)(((Xq + 64) & 127) - 64);
        dig[d] = t;
        Xq = (Xq - t) >> 7;
      }
    } else {
      dig[d] = 0;
    }
  }
  // pack four consecutive samples (lanes 4m..4m+3 of the same fit)
  const int lane = threadIdx.x & 31;
  const int base = lane & ~3;
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    if (d >= F.D) break;
    const unsigned byte = (unsigned)(dig[d] & 0xff);
    unsigned word = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) word |= __shfl_sync(0xffffffffu, byte, base + q) << (8 * q);
    if (ok && (lane & 3) == 0) F.digits[(int64_t)(b * F.D + d) * F.n4p + (i >> 2)] = (int32_t)word;
  }
}

cudaError_t launch_quantize(int NB, const Fits &F, int off, cudaStream_t s) {
  const int64_t total = (int64_t)NB * 4 * F.n4p;
  const unsigned grid = (unsigned)((total + 255) / 256);
  switch (NB) {
    case 1: k_quantize<1><<<grid, 256, 0, s>>>(F, off); break;
    case 2: k_quantize<2><<<grid, 256, 0, s>>>(F, off); break;
    case 3: k_quantize<3><<<grid, 256, 0, s>>>(F, off); break;
    case 4: k_quantize<4><<<grid, 256, 0, s>>>(F, off); break;
    case 8: k_quantize<8><<<grid, 256, 0, s>>>(F, off); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ============================================================ stop test

// Stop test of the iterate w^k (k = *it_base + off, a multiple of K):
// combines the column pass's R_b partials with the vector kernel's partials
// of w^k. A fit stops when KKT <= tol, when k >= max_iter, or on NaN.
template <int NB>
__global__ void __launch_bounds__(32) k_check(Fits F, int off) {
  const int k = *F.it_base + off;
  const int b = threadIdx.x;
  if (b >= F.nb || F.done[b] >= 0) return;
  const double *tc = F.tot_c[k & 1] + b * kCPartials;
  const double rb = F.tot_a[b * 3 + 0];
  double bound = 0.0;
  if (F.mixed) {
    // |s_j error| <= a_j sum_i x_ij |theta_i - theta^_i| <= colbound * half an ulp;
    // the X~ beta rounding bound is already inside the r_p partials
    bound = 0.5 * F.colbound * F.scale[b] * F.th_unit;
  }
  const double R_p = tc[0] / (1.0 + F.ymax);
  const double R_z = tc[1];
  const double R_b = (rb + bound) / F.lamnorm[b];
  const double R_1 = fabs(tc[2]);
  const double kkt = fmax(fmax(R_p, R_z), fmax(R_b, R_1));
  // fmax drops a NaN operand, so each residual is tested: a NaN iterate
  // reaches at least the sum of theta behind R_1
  const bool bad = isnan(R_p) || isnan(R_z) || isnan(R_b) || isnan(R_1) || isinf(kkt);
  double *rep = F.report + b * kReport;
  rep[0] = kkt; rep[1] = R_p; rep[2] = R_z; rep[3] = R_b; rep[4] = R_1;
  rep[6] = bound / F.lamnorm[b];
  rep[7] = k;
  if (bad || kkt <= F.tol || k >= F.max_iter) {
    rep[5] = bad ? FSQR_ENUMERIC : (kkt <= F.tol ? FSQR_OK : FSQR_ENOCONV);
    F.done[b] = k;
    atomicAdd(F.n_done, 1);
  }
}

cudaError_t launch_check(int NB, const Fits &F, int off, cudaStream_t s) {
  switch (NB) {
    case 1: k_check<1><<<1, 32, 0, s>>>(F, off); break;
    case 2: k_check<2><<<1, 32, 0, s>>>(F, off); break;
    case 3: k_check<3><<<1, 32, 0, s>>>(F, off); break;
    case 4: k_check<4><<<1, 32, 0, s>>>(F, off); break;
    case 8: k_check<8><<<1, 32, 0, s>>>(F, off); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ====================================================== vector update

// Thread per (sample i, fit b). init = 1: r^0 = X~ beta^0 + z^0 - y and the
// partials of w^0 only. Otherwise, for fits still running:
//   z^{k+1} = (v - tau/(n mu))_+ - (-v - (1-tau)/(n mu))_+,  v = z^k + theta^k/mu
//   r^{k+1} = X~ beta^{k+1} + z^{k+1} - y
//   theta^{k+1} = theta^k - mu/(G+1) (2 r^{k+1} - r^k)
// and the partials (max |r|, max dist(n theta, d rho(z)), sum theta,
// max |theta|) of w^{k+1} for the next stop test and quantisation.
template <int NB>
__global__ void __launch_bounds__(kCThreads) k_vec(Dsg X, Fits F, int off, int init) {
  __shared__ double red[kCPartials][256];
  const int k = init ? 0 : (*F.it_base + off);
  const int64_t i = (int64_t)blockIdx.x * kCThreads + threadIdx.x;
  const int S = F.meta_i[0];
  const int64_t nrows = F.n;
  const bool row = i < nrows;
  double p[NB][kCPartials];
  bool run[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    run[b] = (b < F.nb) && (init || F.done[b] < 0);
#pragma unroll
    for (int q = 0; q < kCPartials; ++q) p[b][q] = 0.0;
  }
  if (row) {
    double xb[NB], xb_err[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) { xb[b] = F.meta_d[b]; xb_err[b] = 0.0; }
    if (F.mixed) {
      // exact integer slope part of the stored columns, then the covariates
      long long V[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) V[b] = 0;
      // all split partials are loaded before any is added (no serial latency)
      for (int sp0 = 0; sp0 < S; sp0 += 8) {
        long long v[8][NB];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const long long *src = F.xb_ipart + ((int64_t)(sp0 + u) * F.npad + i) * NB;
#pragma unroll
          for (int b = 0; b < NB; ++b) v[u][b] = (sp0 + u < S) ? __ldcg(src + b) : 0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int b = 0; b < NB; ++b) V[b] += v[u][b];
      }
      const double *bt = F.beta[init ? 0 : ((k & 1) ^ 1)];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const double unit = F.meta_d[kMaxNB + b] * F.xb_unit;
        xb_err[b] = (double)F.meta_i[1] * unit;
        xb[b] += (double)V[b] * unit;
      }
#pragma unroll 4
      for (int64_t j = 1; j <= X.c; ++j) {
        const double x = __ldg(X.cov + (j - 1) * X.n + i), aj = __ldg(X.a + j);
#pragma unroll
        for (int b = 0; b < NB; ++b) xb[b] = fma(aj * __ldg(bt + j * NB + b), x, xb[b]);
      }
    } else {
#pragma unroll 8
      for (int sp = 0; sp < S; ++sp) {
        const double *src = F.xb_part + ((int64_t)sp * F.npad + i) * NB;
#pragma unroll
        for (int b = 0; b < NB; ++b) xb[b] += __ldcg(src + b);
      }
    }
    const double yi = __ldg(F.y + i);
    const double nmu = (double)nrows * F.mu;
    if (F.qcorr)
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        xb[b] += F.qcorr[i * NB + b];
        F.qcorr[i * NB + b] = 0.0;
      }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (!run[b]) continue;
      const int64_t ib = i * NB + b;
      const double tau = F.tau[b];
      if (init) {
        const double zi = F.z[ib], ti = F.theta[ib];
        const double ri = xb[b] + zi - yi;
        F.r[ib] = ri;
        p[b][0] = fabs(ri) + xb_err[b];
        p[b][1] = dist_pinball((double)nrows * ti, zi, tau);
        p[b][2] = ti;
        p[b][3] = fabs(ti);
      } else {
        row_update(F, ib, tau, nmu, (double)nrows, xb[b], xb_err[b], yi, F.z[ib], F.theta[ib], F.r[ib],
                   p[b]);
      }
    }
  }
  const int par = init ? 0 : ((k + 1) & 1);
  const int ops[4] = {0, 0, 1, 0};
#pragma unroll
  for (int b = 0; b < NB; ++b) {
#pragma unroll
    for (int q = 0; q < kCPartials; ++q) red[q][threadIdx.x] = p[b][q];
    __syncthreads();
    tree_reduce<4>(red, ops, kCThreads);
    if (threadIdx.x == 0 && run[b]) {
      double *cp = F.c_part[par] + (blockIdx.x * NB + b) * kCPartials;
      cp[0] = red[0][0]; cp[1] = red[1][0]; cp[2] = red[2][0]; cp[3] = red[3][0];
    }
    __syncthreads();
  }
  vec_finalize<NB>(F, par, F.gridC);
}

cudaError_t launch_vec(int NB, const Dsg &X, const Fits &F, int off, int init, cudaStream_t s) {
  const unsigned grid = (unsigned)F.gridC;
  switch (NB) {
    case 1: k_vec<1><<<grid, kCThreads, 0, s>>>(X, F, off, init); break;
    case 2: k_vec<2><<<grid, kCThreads, 0, s>>>(X, F, off, init); break;
    case 3: k_vec<3><<<grid, kCThreads, 0, s>>>(X, F, off, init); break;
    case 4: k_vec<4><<<grid, kCThreads, 0, s>>>(X, F, off, init); break;
    case 8: k_vec<8><<<grid, kCThreads, 0, s>>>(X, F, off, init); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

__global__ void k_advance(int *it_base, int M) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *it_base += M;
}

cudaError_t launch_advance(int *it_base, int M, cudaStream_t s) {
  k_advance<<<1, 32, 0, s>>>(it_base, M);
  return cudaGetLastError();
}

// X~ beta of the last k_xbeta pass: out[b*ldo + i] for b < nb, i < n.
template <int NB>
__global__ void k_gather_xb(Fits F, double *out, int64_t ldo, int nb, int64_t n) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = g / NB;
  const int b = (int)(g - i * NB);
  if (i >= n || b >= nb) return;
  const int S = F.meta_i[0];
  double xb = F.meta_d[b];
  for (int sp = 0; sp < S; ++sp) xb += F.xb_part[((int64_t)sp * F.npad + i) * NB + b];
  if (F.qcorr) {
    xb += F.qcorr[i * NB + b];
    F.qcorr[i * NB + b] = 0.0;
  }
  out[(int64_t)b * ldo + i] = xb;
}

cudaError_t launch_gather_xb(int NB, const Fits &F, double *out, int64_t ldo, int nb,
                             cudaStream_t s) {
  const int64_t rows = F.n;
  const unsigned grid = (unsigned)((rows * NB + 255) / 256);
  switch (NB) {
    case 1: k_gather_xb<1><<<grid, 256, 0, s>>>(F, out, ldo, nb, rows); break;
    case 2: k_gather_xb<2><<<grid, 256, 0, s>>>(F, out, ldo, nb, rows); break;
    case 3: k_gather_xb<3><<<grid, 256, 0, s>>>(F, out, ldo, nb, rows); break;
    case 4: k_gather_xb<4><<<grid, 256, 0, s>>>(F, out, ldo, nb, rows); break;
    case 8: k_gather_xb<8><<<grid, 256, 0, s>>>(F, out, ldo, nb, rows); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace fsqr

namespace fsqr {

// Resident CTAs per SM of the iteration's column kernel for this group shape.
template <int NB, int D>
static int occ_one(size_t smem) {
  int nblk = 0;
  // raises the shared-memory opt-in before any graph capture
  if (smem > g_col_opted<NB, A_PROX, D>) {
    if (cudaFuncSetAttribute(k_col<NB, A_PROX, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    g_col_opted<NB, A_PROX, D> = smem;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, k_col<NB, A_PROX, D>, kAThreads, smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nblk;
}

template <int NB>
static int occ_nb(int mixed, int D, size_t smem) {
  if (!mixed) return occ_one<NB, 0>(smem);
  if (D == 3) return occ_one<NB, 3>(smem);
  if (D == 4) return occ_one<NB, 4>(smem);
  if (D == 5) return occ_one<NB, 5>(smem);
  return 0;
}

int col_pass_occupancy(int NB, int mixed, int D, size_t smem) {
  switch (NB) {
    case 1: return occ_nb<1>(mixed, D, smem);
    case 2: return occ_nb<2>(mixed, D, smem);
    case 3: return occ_nb<3>(mixed, D, smem);
    case 4: return occ_nb<4>(mixed, D, smem);
    case 8: return occ_nb<8>(mixed, D, smem);
    default: return 0;
  }
}

}  // namespace fsqr

namespace fsqr {

// Mean imputation in X~ beta: a missing entry (i, j) of a stored column
// reads as code 0, which the slope/constant split turns into b_j; so
// qcorr[i*NB + b] -= b_j beta_jb for the missing samples of every active
// stored column (the active list of the column pass). Warps stride over the
// active positions; atomic FP64 adds (the few corrections of one sample are
// added in no fixed order).
__global__ void __launch_bounds__(256) k_miss_xb(Dsg X, Fits F, int NB, int off, const double *__restrict__ beta_in) {
  const double *beta = beta_in;
  if (beta == nullptr) {
    const int k = *F.it_base + off;
    beta = F.beta[(k & 1) ^ 1];
  }
  const int gA = F.gridA;
  const int A = __ldcg(F.a_pre + gA);
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t a = w0; a < A; a += nw) {
    int lo = 0, hi = gA;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldcg(F.a_pre + mid) <= a) lo = mid; else hi = mid;
    }
    const int64_t j = F.a_list[(int64_t)lo * F.T + (a - __ldcg(F.a_pre + lo))];
    if (j <= X.c) continue;  // intercept and covariates have no missing entries
    const int64_t s = j - 1 - X.c;
    const double bj = X.b[j];
    const int64_t e0 = X.mptr[s], e1 = X.mptr[s + 1];
    for (int b = 0; b < NB; ++b) {
      const double c = -bj * beta[j * NB + b];
      if (c == 0.0) continue;
      for (int64_t e = e0 + lane; e < e1; e += 32) atomicAdd(F.qcorr + (int64_t)X.midx[e] * NB + b, c);
    }
  }
}

cudaError_t launch_miss_xb(int NB, const Dsg &X, const Fits &F, int off, const double *beta_in, cudaStream_t s) {
  if (X.mptr == nullptr || F.qcorr == nullptr) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_miss_xb<<<std::max(1, sms) * 4, 256, 0, s>>>(X, F, NB, off, beta_in);
  return cudaGetLastError();
}

}  // namespace fsqr
