// Setup and reporting kernels of the FS-QRPPA path: column statistics
// (standardisation, Section 7), lambda_max (penalty path), the power method
// for eta_g (Section 4), state packing, and the final primal value and
// duality gap of each fit (the stop test's secondary measure).
#include <math.h>
#include <stdint.h>

#include "fsqr_fixed.h"
#include "fsqr_internal.h"

namespace fsqr {

namespace {

__device__ __forceinline__ double g2d_s(uint32_t g) {
  uint32_t hi = (g == 1u) ? 0x3FF00000u : ((g == 2u) ? 0x40000000u : 0u);
  return __hiloint2double((int)hi, 0);
}

// Block-wide reductions for blockDim.x a power of two <= 1024.
__device__ double block_sum(double v, double *sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < (unsigned)o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

__device__ double block_max(double v, double *sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < (unsigned)o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

__device__ double block_min(double v, double *sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < (unsigned)o) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

__device__ long long block_sum_ll(long long v, long long *sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < (unsigned)o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  long long r = sh[0];
  __syncthreads();
  return r;
}

}  // namespace

// ------------------------------------------------------------ column stats

// Mean and population sd over observed entries of feature f (covariates then
// stored columns), one CTA of 256 threads per feature. Integer genotype
// moments are accumulated exactly in int64.
__global__ void __launch_bounds__(256) k_col_stats(Dsg X, double *mean, double *sd, int *missing) {
  __shared__ double shd[256];
  __shared__ long long shl[256];
  const int64_t f = blockIdx.x;
  const int64_t n = X.n;
  if (f < X.c) {
    const double *cv = X.cov + f * n;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += cv[i];
    const double m = block_sum(s, shd) / (double)n;
    double q = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const double d = cv[i] - m;
      q += d * d;
    }
    const double v = block_sum(q, shd) / (double)n;
    if (threadIdx.x == 0) { mean[f] = m; sd[f] = sqrt(v); }
    return;
  }
  const uint8_t *col = X.geno + (f - X.c) * X.ld;
  if (X.fmt == FSQR_DENSE_F64) {
    const double *cv = reinterpret_cast<const double *>(col);
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += cv[i];
    const double m = block_sum(s, shd) / (double)n;
    double q = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const double d = cv[i] - m;
      q += d * d;
    }
    const double v = block_sum(q, shd) / (double)n;
    if (threadIdx.x == 0) { mean[f] = m; sd[f] = sqrt(v); }
    return;
  }
  long long c1 = 0, s1 = 0, s2 = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    uint32_t g;
    if (X.fmt == FSQR_INT8) g = col[i];
    else g = (col[i >> 2] >> (2 * (i & 3))) & 3u;
    if (g <= 2u) { c1 += 1; s1 += g; s2 += g * g; }
  }
  c1 = block_sum_ll(c1, shl);
  s1 = block_sum_ll(s1, shl);
  s2 = block_sum_ll(s2, shl);
  if (threadIdx.x == 0) {
    if (c1 < n) atomicAdd(missing, (int)min((long long)(n - c1), (long long)1 << 30));
    if (c1 == 0) { mean[f] = 0.0; sd[f] = 0.0; return; }
    const double m = (double)s1 / (double)c1;
    // population variance (c1*s2 - s1^2)/c1^2, numerator exact in int64
    const long long num = c1 * s2 - s1 * s1;
    mean[f] = m;
    sd[f] = sqrt((double)num) / (double)c1;
  }
}

cudaError_t launch_col_stats(const Dsg &X, double *mean, double *sd, int *missing, cudaStream_t s) {
  const int64_t F = X.c + X.p;
  if (F == 0) return cudaSuccess;
  k_col_stats<<<(unsigned)F, 256, 0, s>>>(X, mean, sd, missing);
  return cudaGetLastError();
}

// a_j, b_j of x~_ij = a_j x_ij + b_j: intercept (0, 1); standardised
// (1/sd, -mean/sd), constant columns (0, 0); raw (1, 0).
__global__ void k_affine(int64_t P, const double *mean, const double *sd, int standardize,
                         double *a, double *b) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  if (j == 0) { a[0] = 0.0; b[0] = 1.0; return; }
  if (!standardize) { a[j] = 1.0; b[j] = 0.0; return; }
  const double s = sd[j - 1];
  const double aj = (s > 0.0) ? 1.0 / s : 0.0;
  a[j] = aj;
  b[j] = -mean[j - 1] * aj;
}

cudaError_t launch_affine(const Dsg &X, const double *mean, const double *sd, int standardize,
                          double *a, double *b, cudaStream_t s) {
  k_affine<<<(unsigned)((X.P + 255) / 256), 256, 0, s>>>(X.P, mean, sd, standardize, a, b);
  return cudaGetLastError();
}

// max over stored columns of a_j * sum_i x_ij (= a_j n mean_j for 0/1/2 codes
// without missing entries): the l1 weight in the mixed-precision error bound.
__global__ void k_colbound(Dsg X, const double *mean, double *out) {
  __shared__ double sh[256];
  double m = 0.0;
  for (int64_t j = 1 + X.c + threadIdx.x; j < X.P; j += blockDim.x)
    m = fmax(m, X.a[j] * (double)X.n * mean[j - 1]);
  m = block_max(m, sh);
  if (threadIdx.x == 0) *out = m;
}

cudaError_t launch_colbound(const Dsg &X, const double *mean, double *out, cudaStream_t s) {
  k_colbound<<<1, 256, 0, s>>>(X, mean, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------- vector stats

// out3 = {sum v, sum v^2, max |v|} (one CTA).
__global__ void k_vec_stats(const double *v, int64_t n, double *out3) {
  __shared__ double sh[1024];
  double s = 0.0, q = 0.0, m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = v[i];
    s += x;
    q += x * x;
    m = fmax(m, fabs(x));
  }
  s = block_sum(s, sh);
  q = block_sum(q, sh);
  m = block_max(m, sh);
  if (threadIdx.x == 0) { out3[0] = s; out3[1] = q; out3[2] = m; }
}

cudaError_t launch_vec_stats(const double *v, int64_t n, double *out3, cudaStream_t s) {
  k_vec_stats<<<1, 1024, 0, s>>>(v, n, out3);
  return cudaGetLastError();
}

// sums[g] = sum_i v[g*ldv + i], sqsums[g] = sum_i v^2 (one CTA per vector).
__global__ void k_sum_cols(const double *v, int64_t n, int64_t ldv, double *sums, double *sqsums) {
  __shared__ double sh[512];
  const double *x = v + (int64_t)blockIdx.x * ldv;
  double s = 0.0, q = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    s += x[i];
    q += x[i] * x[i];
  }
  s = block_sum(s, sh);
  q = block_sum(q, sh);
  if (threadIdx.x == 0) {
    if (sums) sums[blockIdx.x] = s;
    if (sqsums) sqsums[blockIdx.x] = q;
  }
}

cudaError_t launch_sum_cols(const double *v, int64_t n, int64_t ldv, int nvec, double *sums,
                            double *sqsums, cudaStream_t s) {
  if (nvec <= 0) return cudaSuccess;
  k_sum_cols<<<nvec, 512, 0, s>>>(v, n, ldv, sums, sqsums);
  return cudaGetLastError();
}

// ------------------------------------------------------------ lambda_max

// k-th smallest (1-based) of y by an 8-pass radix select over the
// order-preserving 64-bit keys of the doubles (one CTA).
__device__ __forceinline__ unsigned long long dkey(double x) {
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void __launch_bounds__(1024) k_select(const double *y, int64_t n, int64_t k, double *out) {
  __shared__ unsigned int hist[256];
  __shared__ unsigned long long sPrefix;
  __shared__ long long sK;
  if (threadIdx.x == 0) { sPrefix = 0ull; sK = k; }
  __syncthreads();
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 56 - 8 * pass;
    for (int t = threadIdx.x; t < 256; t += blockDim.x) hist[t] = 0u;
    __syncthreads();
    const unsigned long long pre = sPrefix;
    const unsigned long long mask = (pass == 0) ? 0ull : (~0ull << (shift + 8));
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const unsigned long long key = dkey(y[i]);
      if ((key & mask) == pre) atomicAdd(&hist[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long kk = sK;
      int d = 0;
      for (; d < 256; ++d) {
        if (kk <= (long long)hist[d]) break;
        kk -= hist[d];
      }
      if (d > 255) d = 255;
      sK = kk;
      sPrefix = pre | ((unsigned long long)d << shift);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const unsigned long long key = sPrefix;
    const unsigned long long u = (key >> 63) ? (key & 0x7fffffffffffffffull) : ~key;
    *out = __longlong_as_double((long long)u);
  }
}

cudaError_t launch_select(const double *y, int64_t n, int64_t k, double *out, cudaStream_t s) {
  k_select<<<1, 1024, 0, s>>>(y, n, k, out);
  return cudaGetLastError();
}

// v_i = tau - 1{y_i < q} for i < n, 0 on the padding rows.
__global__ void k_lmax_vec(const double *y, int64_t n, int64_t npad, double tau, const double *q,
                           double *v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  v[i] = (i < n) ? (tau - ((y[i] < *q) ? 1.0 : 0.0)) : 0.0;
}

cudaError_t launch_lmax_vec(const double *y, int64_t n, int64_t npad, double tau, const double *q,
                            double *v, cudaStream_t s) {
  k_lmax_vec<<<(unsigned)((npad + 255) / 256), 256, 0, s>>>(y, n, npad, tau, q, v);
  return cudaGetLastError();
}

// out = max_{j>=1, omega_j>0} |s_j| / (scale omega_j), 0 if no such column.
__global__ void k_colmax_ratio(const double *s_col, const double *omega, int64_t P, double scale,
                               double *out) {
  __shared__ double sh[1024];
  double m = 0.0;
  for (int64_t j = 1 + threadIdx.x; j < P; j += blockDim.x) {
    const double w = omega[j];
    if (w > 0.0) m = fmax(m, fabs(s_col[j]) / (scale * w));
  }
  m = block_max(m, sh);
  if (threadIdx.x == 0) *out = m;
}

cudaError_t launch_colmax_ratio(const double *s_col, const double *omega, int64_t P, double scale,
                                double *out, cudaStream_t s) {
  k_colmax_ratio<<<1, 1024, 0, s>>>(s_col, omega, P, scale, out);
  return cudaGetLastError();
}

// --------------------------------------------------------- power method

// v_j = 1/sqrt(p_g) for j in block g.
__global__ void k_power_init(double *v, const int64_t *bp, int G, int64_t P) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  int lo = 0, hi = G;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (bp[mid] <= j) lo = mid; else hi = mid;
  }
  v[j] = 1.0 / sqrt((double)(bp[lo + 1] - bp[lo]));
}

cudaError_t launch_power_init(double *v, const int64_t *block_ptr, int G, int64_t P, cudaStream_t s) {
  k_power_init<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(v, block_ptr, G, P);
  return cudaGetLastError();
}

// Per block g: wnorm[g] = ||w_g||, then v_g = w_g / ||w_g|| (v_g = 0 if the
// norm is 0). One CTA per block.
__global__ void k_power_step(const double *w, const int64_t *bp, double *v, double *wnorm) {
  __shared__ double sh[512];
  const int g = blockIdx.x;
  const int64_t j0 = bp[g], j1 = bp[g + 1];
  double q = 0.0;
  for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) q += w[j] * w[j];
  const double nw = sqrt(block_sum(q, sh));
  if (threadIdx.x == 0) wnorm[g] = nw;
  for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) v[j] = (nw > 0.0) ? w[j] / nw : 0.0;
}

cudaError_t launch_power_step(const double *w, const int64_t *block_ptr, int G, int64_t P,
                              double *v, double *wnorm, cudaStream_t s) {
  (void)P;
  k_power_step<<<G, 512, 0, s>>>(w, block_ptr, v, wnorm);
  return cudaGetLastError();
}

// u_g = X~_g v_g for every block g at once. CTA (rc, sp) sums the columns of
// split sp (a range inside one block, from the split table) over its rows;
// a second kernel adds the splits of each block in order.
__global__ void __launch_bounds__(256) k_xv_split(Dsg X, const double *v, const int64_t *splits,
                                                  double *part, int64_t npad) {
  const int sp = blockIdx.y;
  const int64_t ja = splits[2 * sp], jb = splits[2 * sp + 1];
  const int64_t i0 = (int64_t)blockIdx.x * 2048 + threadIdx.x * 8;
  double acc[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) acc[r] = 0.0;
  if (i0 < X.n) {
    for (int64_t j = ja; j < jb; ++j) {
      const double aj = X.a[j], bj = X.b[j], vj = v[j];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int64_t i = i0 + r;
        if (i >= X.n) break;
        double x;
        if (j == 0) x = 0.0;
        else if (j <= X.c) x = X.cov[(j - 1) * X.n + i];
        else {
          const uint8_t *col = X.geno + (j - 1 - X.c) * X.ld;
          if (X.fmt == FSQR_DENSE_F64) x = reinterpret_cast<const double *>(col)[i];
          else if (X.fmt == FSQR_INT8) x = g2d_s(col[i]);
          else x = g2d_s((col[i >> 2] >> (2 * (i & 3))) & 3u);
        }
        acc[r] = fma(fma(aj, x, bj), vj, acc[r]);
      }
    }
  }
  double *out = part + (int64_t)sp * npad;
#pragma unroll
  for (int r = 0; r < 8; ++r)
    if (i0 + r < npad) out[i0 + r] = (i0 + r < X.n) ? acc[r] : 0.0;
}

__global__ void k_xv_reduce(const double *part, const int *split_of_block, int G, int64_t npad,
                            double *u) {
  const int64_t g = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  double s = 0.0;
  for (int sp = split_of_block[g]; sp < split_of_block[g + 1]; ++sp) s += part[(int64_t)sp * npad + i];
  u[g * npad + i] = s;
}

// splits: device table of 2*nsplit column bounds, split_of_block: G+1 offsets.
cudaError_t launch_xv_blocks(const Dsg &X, const double *v, const int64_t *splits,
                             const int *split_of_block, int G, int nsplit, double *u,
                             int64_t npad, double *part, cudaStream_t s) {
  dim3 g1((unsigned)((X.n + 2047) / 2048), (unsigned)nsplit);
  k_xv_split<<<g1, 256, 0, s>>>(X, v, splits, part, npad);
  dim3 g2((unsigned)((npad + 255) / 256), (unsigned)G);
  k_xv_reduce<<<g2, 256, 0, s>>>(part, split_of_block, G, npad, u);
  return cudaGetLastError();
}

// ------------------------------- exact integer products for the setup passes
//
// The power method and lambda_max multiply the stored codes (0, 1, 2) by a
// vector. As FP64 SIMT passes they run at the GB300's FP64 rate, far below
// HBM. Here the vector is rounded once, per segment, to 52-bit fixed point:
// w_k = q_k unit_s with unit_s = 2^(e-52), 2^e > max_s |w_k|, and
// q_k = hi_k 2^26 + lo_k, 0 <= lo_k < 2^26. Sums of code * hi and code * lo
// are exact in int64 (|sum| < 2^48 for n, column ranges <= 2^20) and become
// one FP64 value per output: the rounding is that of one FP64 operation on
// the result, and the vector's own rounding is 2^-53 relative to its largest
// entry.

// Segment s covers x[bounds[2s] .. bounds[2s+1]), or x[s*seglen .. +seglen)
// when bounds is NULL. Entries below `first` get
// q = 0 (columns taken in FP64 by the caller). w_k = x_k * mult_k (mult NULL:
// 1). Also cst[s] = sum over the quantised entries of cmul_k x_k (cmul,
// cst NULL: none). One CTA of 256 threads per segment, fixed-order sums.
__global__ void __launch_bounds__(256) k_fix_seg(const double *x, const double *mult, const double *cmul,
                                                 const int64_t *bounds, int64_t seglen, int64_t first, int2 *q,
                                                 double *unit, double *cst) {
  __shared__ double sh[256];
  const int sg = blockIdx.x;
  const int64_t k0 = bounds ? bounds[2 * sg] : (int64_t)sg * seglen;
  const int64_t k1 = bounds ? bounds[2 * sg + 1] : k0 + seglen;
  double m = 0.0, c = 0.0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += 256) {
    if (k < first) continue;
    const double w = mult ? x[k] * mult[k] : x[k];
    m = fmax(m, fabs(w));
    if (cmul) c = fma(cmul[k], x[k], c);
  }
  m = block_max(m, sh);
  if (cst) {
    c = block_sum(c, sh);
    if (threadIdx.x == 0) cst[sg] = c;
  }
  // 2^e > m: ilogb(m) = floor(log2 m) for finite m > 0
  const int e = (m > 0.0 && m <= 1.0e300) ? ilogb(m) + 1 : 0;
  if (threadIdx.x == 0) unit[sg] = (m > 0.0 && m <= 1.0e300) ? ldexp(1.0, e - 52) : 0.0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += 256) {
    long long v = 0;
    if (k >= first && m > 0.0 && m <= 1.0e300) {
      const double t = ldexp(mult ? x[k] * mult[k] : x[k], 52 - e);  // |t| < 2^52
      v = (fabs(t) <= 4503599627370496.0) ? __double2ll_rn(t) : 0LL;
    }
    const long long hi = v >> 26;  // arithmetic shift: floor
    q[k] = make_int2((int)(v - (hi << 26)), (int)hi);
  }
}

cudaError_t launch_fix_seg(const double *x, const double *mult, const double *cmul, const int64_t *bounds,
                           int64_t seglen, int nseg, int64_t first, int2 *q, double *unit, double *cst,
                           cudaStream_t s) {
  if (nseg <= 0) return cudaSuccess;
  k_fix_seg<<<nseg, 256, 0, s>>>(x, mult, cmul, bounds, seglen, first, q, unit, cst);
  return cudaGetLastError();
}

// u_g = X~_g v_g with exact integer products over the stored columns (int8 or
// 2-bit codes; a missing code reads as 0 and k_miss_xv takes its share back
// out). The split table and the layout of `part` are those of k_xv_split;
// q/unit/cst are k_fix_seg's output over the splits (mult = a, cmul = b,
// first = c + 1), so that stored column j adds x_ij q_j unit + b_j v_j.
// The intercept and the covariates (j <= c) stay in FP64. Thread: 8 samples.
__global__ void __launch_bounds__(256) k_xv_int(Dsg X, const double *v, const int64_t *splits, const int2 *q,
                                                const double *unit, const double *cst, double *part,
                                                int64_t npad) {
  const int sp = blockIdx.y;
  const int64_t ja = splits[2 * sp], jb = splits[2 * sp + 1];
  const int64_t i0 = (int64_t)blockIdx.x * 2048 + threadIdx.x * 8;
  long long ahi[8], alo[8];
  double acc[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    ahi[r] = 0;
    alo[r] = 0;
    acc[r] = 0.0;
  }
  if (i0 < X.n) {
    int64_t j = ja;
    for (; j < jb && j <= X.c; ++j) {  // intercept (x~ = b_0) and covariates, FP64
      const double aj = X.a[j], bj = X.b[j], vj = v[j];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int64_t i = i0 + r;
        if (i >= X.n) break;
        const double x = (j == 0) ? 0.0 : X.cov[(j - 1) * X.n + i];
        acc[r] = fma(fma(aj, x, bj), vj, acc[r]);
      }
    }
    if (X.fmt == FSQR_INT8) {
      // i0 is a multiple of 8 and i0 + 8 <= pad16(n) <= ld: one aligned 8-byte load
      for (; j < jb; ++j) {
        const int2 qj = __ldg(q + j);
        const uint2 cw = __ldcs(reinterpret_cast<const uint2 *>(X.geno + (j - 1 - X.c) * X.ld + i0));
        // codes above 2 (missing) read as 0
        const uint32_t w0 = cw.x & __vcmpleu4(cw.x, 0x02020202u);
        const uint32_t w1 = cw.y & __vcmpleu4(cw.y, 0x02020202u);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int cd = (int)(((r < 4 ? w0 : w1) >> (8 * (r & 3))) & 0xffu);
          ahi[r] += (long long)cd * qj.y;
          alo[r] += (long long)cd * qj.x;
        }
      }
    } else if (X.fmt == FSQR_2BIT) {
      // 8 samples = 2 bytes at byte i0/4, inside ld (ld >= 2 ceil(n/8))
      for (; j < jb; ++j) {
        const int2 qj = __ldg(q + j);
        const uint32_t cw = __ldcs(reinterpret_cast<const unsigned short *>(X.geno + (j - 1 - X.c) * X.ld + (i0 >> 2)));
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          int cd = (int)((cw >> (2 * r)) & 3u);
          cd = (cd == 3) ? 0 : cd;
          ahi[r] += (long long)cd * qj.y;
          alo[r] += (long long)cd * qj.x;
        }
      }
    }
  }
  const double un = unit[sp], cs = cst[sp];
  double *out = part + (int64_t)sp * npad;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int64_t i = i0 + r;
    if (i < npad)
      out[i] = (i < X.n) ? fma(un, fma((double)ahi[r], 67108864.0, (double)alo[r]), cs + acc[r]) : 0.0;
  }
}

cudaError_t launch_xv_blocks_int(const Dsg &X, const double *v, const int64_t *splits, const int *split_of_block,
                                 int G, int nsplit, const int2 *q, const double *unit, const double *cst, double *u,
                                 int64_t npad, double *part, cudaStream_t s) {
  dim3 g1((unsigned)((X.n + 2047) / 2048), (unsigned)nsplit);
  k_xv_int<<<g1, 256, 0, s>>>(X, v, splits, q, unit, cst, part, npad);
  dim3 g2((unsigned)((npad + 255) / 256), (unsigned)G);
  k_xv_reduce<<<g2, 256, 0, s>>>(part, split_of_block, G, npad, u);
  return cudaGetLastError();
}

// ----------------------------------------------------------- state layout

// dst[j*NB + q] = src[q*lds + j] for q < nb and j < len, 0 for len <= j <
// dst_rows; slots q >= nb are left untouched (callers pass dst + slot with
// nb = 1 to fill one slot of an interleaved array).
__global__ void k_pack(const double *src, int64_t lds, double *dst, int64_t len, int nb, int NB,
                       int64_t dst_rows) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= dst_rows * nb) return;
  const int64_t j = g / nb;
  const int q = (int)(g - j * nb);
  dst[j * NB + q] = (j < len) ? src[(int64_t)q * lds + j] : 0.0;
}

cudaError_t launch_pack(const double *src, int64_t lds, double *dst, int64_t len, int nb, int NB,
                        int64_t dst_rows, cudaStream_t s) {
  const int64_t tot = dst_rows * nb;
  if (tot == 0) return cudaSuccess;
  k_pack<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, lds, dst, len, nb, NB, dst_rows);
  return cudaGetLastError();
}

// dst[q*lds + j] = src[j*NB + q] for q < nb, j < len.
__global__ void k_unpack(const double *src, double *dst, int64_t lds, int64_t len, int nb, int NB) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= len * nb) return;
  const int q = (int)(g / len);
  const int64_t j = g - (int64_t)q * len;
  dst[(int64_t)q * lds + j] = src[j * NB + q];
}

cudaError_t launch_unpack(const double *src, double *dst, int64_t lds, int64_t len, int nb, int NB,
                          cudaStream_t s) {
  const int64_t tot = len * nb;
  if (tot == 0) return cudaSuccess;
  k_unpack<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, dst, lds, len, nb, NB);
  return cudaGetLastError();
}

__global__ void k_fill(double *p, double v, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

cudaError_t launch_fill(double *p, double v, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, v, n);
  return cudaGetLastError();
}

// Cold start beta = 0, z = y, theta = 0 for the group's live fits; resets the
// per-fit status and the iteration counter.
__global__ void k_init_state(Fits F, int NB, int cold) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g == 0) {
    *const_cast<int *>(F.it_base) = 0;
    *F.n_done = 0;
  }
  if (g < NB) F.done[g] = (g < F.nb) ? -1 : 0;
  if (!cold) return;
  if (g < F.npad * NB) {
    const int64_t i = g / NB;
    const int q = (int)(g - i * NB);
    F.z[g] = (q < F.nb && i < F.n) ? F.y[i] : 0.0;
    F.theta[g] = 0.0;
  }
}

cudaError_t launch_init_state(int NB, const Fits &F, int nb, int warm, cudaStream_t s) {
  (void)nb;
  const int64_t tot = F.npad * NB;
  k_init_state<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(F, NB, warm == FSQR_WARM_NONE);
  return cudaGetLastError();
}

// ------------------------------------------------------- final reporting

// theta_check_b = clip(theta_b - c, [(tau_b-1)/n, tau_b/n]) with the shift c
// found by bisection so that the entries sum to 0 (one CTA per fit).
__global__ void __launch_bounds__(512) k_dual_point(const double *theta, int64_t n, int64_t npad,
                                                    const double *taus, int NB, double *out,
                                                    double *sums) {
  __shared__ double sh[512];
  const int b = blockIdx.x;
  const double tau = taus[b];
  const double lo_b = (tau - 1.0) / (double)n, hi_b = tau / (double)n;
  double mn = INFINITY, mx = -INFINITY;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double t = theta[i * NB + b];
    mn = fmin(mn, t);
    mx = fmax(mx, t);
  }
  mn = block_min(mn, sh);
  mx = block_max(mx, sh);
  double a = mn - hi_b, c2 = mx - lo_b;
  for (int it = 0; it < 200; ++it) {
    const double c = 0.5 * (a + c2);
    double f = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
      f += fmin(fmax(theta[i * NB + b] - c, lo_b), hi_b);
    f = block_sum(f, sh);
    if (f > 0.0) a = c; else c2 = c;
    if (c2 - a <= 0.0) break;
  }
  const double c = 0.5 * (a + c2);
  double tot = 0.0;
  for (int64_t i = threadIdx.x; i < npad; i += blockDim.x) {
    const double v = (i < n) ? fmin(fmax(theta[i * NB + b] - c, lo_b), hi_b) : 0.0;
    out[i * NB + b] = v;
    tot += v;
  }
  tot = block_sum(tot, sh);
  if (threadIdx.x == 0) sums[b] = tot;
}

cudaError_t launch_dual_point(int NB, const double *theta, int64_t n, int64_t npad,
                              const double *taus, int nb, double *out, double *sums,
                              cudaStream_t s) {
  k_dual_point<<<nb, 512, 0, s>>>(theta, n, npad, taus, NB, out, sums);
  return cudaGetLastError();
}

// out = min_{j>=1} omega_j (+inf when P == 1).
__global__ void k_min_omega(const double *omega, int64_t P, double *out) {
  __shared__ double sh[1024];
  double m = INFINITY;
  for (int64_t j = 1 + threadIdx.x; j < P; j += blockDim.x) m = fmin(m, omega[j]);
  m = block_min(m, sh);
  if (threadIdx.x == 0) *out = m;
}

cudaError_t launch_min_omega(const double *omega, int64_t P, double *out, cudaStream_t s) {
  k_min_omega<<<1, 1024, 0, s>>>(omega, P, out);
  return cudaGetLastError();
}

// Per fit b (one CTA): out[b*8 + ...] = {loss, penalty, active, alpha, y.tc}
//   loss    = (1/n) sum_i rho_tau(z_i - r_i)   (z - r = y - X~ beta)
//   penalty = sum_j lam_b omega_j |beta_j| (+ ridge/2 sum_j omega_j beta_j^2)
//   active  = #{j >= 1 : beta_j != 0}
//   alpha   = min(1, min_{j>=1} lam_j / |s_j|) for s = X~^T theta_check (if s)
//   y.tc    = sum_i y_i theta_check_i (if tc)
__global__ void __launch_bounds__(512) k_summary(int NB, int64_t n, int64_t P, const double *y,
                                                 const double *z, const double *r,
                                                 const double *beta, const double *omega,
                                                 const double *taus, const double *lams,
                                                 const double *s_chk, const double *tc, double ridge,
                                                 double *out) {
  __shared__ double sh[512];
  const int b = blockIdx.x;
  const double tau = taus[b], lam = lams[b];
  double loss = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double u = z[i * NB + b] - r[i * NB + b];
    loss += (tau - (u < 0.0 ? 1.0 : 0.0)) * u;
  }
  loss = block_sum(loss, sh) / (double)n;
  double pen = 0.0, act = 0.0, al = INFINITY;
  for (int64_t j = threadIdx.x; j < P; j += blockDim.x) {
    const double bj = beta[j * NB + b];
    const double lj = lam * omega[j];
    pen += lj * fabs(bj) + 0.5 * ridge * omega[j] * bj * bj;
    if (j >= 1 && bj != 0.0) act += 1.0;
    if (s_chk && j >= 1) {
      const double sa = fabs(s_chk[j * NB + b]);
      if (sa > 0.0) al = fmin(al, lj / sa);
    }
  }
  pen = block_sum(pen, sh);
  act = block_sum(act, sh);
  al = block_min(al, sh);
  double ytc = 0.0;
  if (tc) {
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) ytc += y[i] * tc[i * NB + b];
    ytc = block_sum(ytc, sh);
  }
  if (threadIdx.x == 0) {
    out[b * 8 + 0] = loss;
    out[b * 8 + 1] = pen;
    out[b * 8 + 2] = act;
    out[b * 8 + 3] = fmin(1.0, al);
    out[b * 8 + 4] = ytc;
  }
}

cudaError_t launch_summary(int NB, int nb, int64_t n, int64_t P, const double *y, const double *z,
                           const double *r, const double *beta, const double *omega,
                           const double *taus, const double *lams, const double *s_chk,
                           const double *tc, double ridge, double *out, cudaStream_t s) {
  k_summary<<<nb, 512, 0, s>>>(NB, n, P, y, z, r, beta, omega, taus, lams, s_chk, tc, ridge, out);
  return cudaGetLastError();
}

// Stop-test residuals of a given iterate (fsqr_kkt): needs X~ beta (xb),
// s = X~^T theta, one fit. out = {R_p, R_z, R_b_unnormalised, R_1}.
__global__ void __launch_bounds__(512) k_kkt_given(int64_t n, int64_t P, const double *y,
                                                   const double *xb, const double *z,
                                                   const double *theta, const double *s,
                                                   const double *beta, const double *omega,
                                                   double tau, double lam, double *out) {
  __shared__ double sh[512];
  double rp = 0.0, rz = 0.0, st = 0.0, ym = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    rp = fmax(rp, fabs(y[i] - xb[i] - z[i]));
    ym = fmax(ym, fabs(y[i]));
    const double t = (double)n * theta[i];
    const double zi = z[i];
    double d;
    if (zi > 0.0) d = fabs(t - tau);
    else if (zi < 0.0) d = fabs(t - (tau - 1.0));
    else d = fmax(fmax(tau - 1.0 - t, t - tau), 0.0);
    rz = fmax(rz, d);
    st += theta[i];
  }
  double rb = 0.0;
  for (int64_t j = 1 + threadIdx.x; j < P; j += blockDim.x) {
    const double sj = s[j], bj = beta[j], lj = lam * omega[j];
    double d;
    if (bj > 0.0) d = fabs(sj - lj);
    else if (bj < 0.0) d = fabs(sj + lj);
    else d = fmax(fabs(sj) - lj, 0.0);
    rb = fmax(rb, d);
  }
  rp = block_max(rp, sh);
  ym = block_max(ym, sh);
  rz = block_max(rz, sh);
  st = block_sum(st, sh);
  rb = block_max(rb, sh);
  if (threadIdx.x == 0) {
    out[0] = rp / (1.0 + ym);
    out[1] = rz;
    out[2] = rb;
    out[3] = fabs(st);
  }
}

cudaError_t launch_kkt_given(int64_t n, int64_t P, const double *y, const double *xb,
                             const double *z, const double *theta, const double *s,
                             const double *beta, const double *omega, double tau, double lam,
                             double *out, cudaStream_t st) {
  k_kkt_given<<<1, 512, 0, st>>>(n, P, y, xb, z, theta, s, beta, omega, tau, lam, out);
  return cudaGetLastError();
}

// Original-scale coefficients: b_j a_j for j >= 1 (a_j = 1/sd_j or 0), and
// b_0 + sum_j b_j(offset) beta_j for the intercept (one CTA per vector).
__global__ void __launch_bounds__(512) k_back_transform(Dsg X, const double *beta, double *out) {
  __shared__ double sh[512];
  const double *bv = beta + (int64_t)blockIdx.x * X.P;
  double *ov = out + (int64_t)blockIdx.x * X.P;
  double c = 0.0;
  for (int64_t j = 1 + threadIdx.x; j < X.P; j += blockDim.x) {
    ov[j] = X.a[j] * bv[j];
    c += X.b[j] * bv[j];
  }
  c = block_sum(c, sh);
  if (threadIdx.x == 0) ov[0] = bv[0] + c;
}

cudaError_t launch_back_transform(const Dsg &X, const double *beta, int B, double *out,
                                  cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_back_transform<<<B, 512, 0, s>>>(X, beta, out);
  return cudaGetLastError();
}

}  // namespace fsqr

namespace fsqr {

// Penalty weights of an LLA step (Section 6, Algorithm 2), out[0] = 0 and
// for j >= 1:
//   type FSQR_PEN_SCAD: omega_j p'(|src_j|) scale, p' of eq. scad (a > 2)
//   type FSQR_PEN_MCP:  omega_j p'(|src_j|) scale, p' of eq. mcp  (a > 1)
//   type 0:             omega_j lam scale (the weighted-l1 weights)
//   type -1:            src_j scale
__global__ void k_lla_weights(const double *src, const double *omega, int64_t P, double lam, double a, int type,
                              double scale, double *out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  if (j == 0) { out[0] = 0.0; return; }
  double v;
  if (type == FSQR_PEN_SCAD || type == FSQR_PEN_MCP) {
    const double t = fabs(src[j]);
    double d;
    if (type == FSQR_PEN_SCAD) d = (t <= lam) ? lam : ((t < a * lam) ? (a * lam - t) / (a - 1.0) : 0.0);
    else d = (t <= a * lam) ? lam - t / a : 0.0;
    v = omega[j] * d * scale;
  } else if (type == 0) {
    v = omega[j] * lam * scale;
  } else {
    v = src[j] * scale;
  }
  out[j] = v;
}

cudaError_t launch_lla_weights(const double *src, const double *omega, int64_t P, double lam, double a, int type,
                               double scale, double *out, cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  k_lla_weights<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(src, omega, P, lam, a, type, scale, out);
  return cudaGetLastError();
}

}  // namespace fsqr

namespace fsqr {

// Model selection along a path (Section 7), one CTA per fit b:
//   out[2b]     = sum_i rho_{tau_b}(y_i - q_{b,i})   (q = X~ beta_b, row b*n)
//   out[2b + 1] = #{j >= 1 : beta_{b,j} != 0}
__global__ void __launch_bounds__(512) k_path_stats(const double *q, const double *y, const double *taus, int64_t n,
                                                    const double *beta, int64_t P, double *out) {
  __shared__ double sh[512];
  const int b = blockIdx.x;
  const double tau = taus[b];
  double loss = 0.0, act = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double u = y[i] - q[(int64_t)b * n + i];
    loss += (tau - (u < 0.0 ? 1.0 : 0.0)) * u;
  }
  for (int64_t j = 1 + threadIdx.x; j < P; j += blockDim.x) act += (beta[(int64_t)b * P + j] != 0.0) ? 1.0 : 0.0;
  loss = block_sum(loss, sh);
  act = block_sum(act, sh);
  if (threadIdx.x == 0) {
    out[2 * b] = loss;
    out[2 * b + 1] = act;
  }
}

cudaError_t launch_path_stats(const double *q, const double *y, const double *taus, int64_t n, const double *beta,
                              int64_t P, int B, double *out, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_path_stats<<<B, 512, 0, s>>>(q, y, taus, n, beta, P, out);
  return cudaGetLastError();
}

// Prediction intervals [q_lo, q_hi] (Section 7.1): out = {number of samples
// with q_lo <= y <= q_hi and q_lo <= q_hi, sum of q_hi - q_lo, number of
// crossings q_lo > q_hi} (one CTA, fixed-order reduction).
__global__ void __launch_bounds__(1024) k_coverage(const double *qlo, const double *qhi, const double *y, int64_t n,
                                                   double *out) {
  __shared__ double sh[1024];
  double cov = 0.0, wid = 0.0, cr = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double lo = qlo[i], hi = qhi[i], yi = y[i];
    cov += (lo <= hi && lo <= yi && yi <= hi) ? 1.0 : 0.0;
    wid += hi - lo;
    cr += (lo > hi) ? 1.0 : 0.0;
  }
  cov = block_sum(cov, sh);
  wid = block_sum(wid, sh);
  cr = block_sum(cr, sh);
  if (threadIdx.x == 0) {
    out[0] = cov;
    out[1] = wid;
    out[2] = cr;
  }
}

cudaError_t launch_coverage(const double *qlo, const double *qhi, const double *y, int64_t n, double *out,
                            cudaStream_t s) {
  k_coverage<<<1, 1024, 0, s>>>(qlo, qhi, y, n, out);
  return cudaGetLastError();
}

}  // namespace fsqr

namespace fsqr {

// ------------------------------------------- missing genotype entries
// (mean imputation of Section 7.2: a missing entry takes the column mean,
// i.e. standardised value 0)

__device__ __forceinline__ bool is_missing(const Dsg &X, const uint8_t *col, int64_t i) {
  if (X.fmt == FSQR_INT8) return col[i] > 2u;
  if (X.fmt == FSQR_2BIT) return ((col[i >> 2] >> (2 * (i & 3))) & 3u) == 3u;
  return false;
}

// One warp per stored column: cnt[s] = number of missing samples.
__global__ void k_miss_count(Dsg X, int *cnt) {
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= X.p) return;
  const uint8_t *col = X.geno + s * X.ld;
  int c = 0;
  for (int64_t i = lane; i < X.n; i += 32) c += is_missing(X, col, i) ? 1 : 0;
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) cnt[s] = c;
}

cudaError_t launch_miss_count(const Dsg &X, int *cnt, cudaStream_t s) {
  if (X.p == 0) return cudaSuccess;
  const int64_t threads = X.p * 32;
  k_miss_count<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(X, cnt);
  return cudaGetLastError();
}

// One warp per stored column: the missing samples in ascending order.
__global__ void k_miss_fill(Dsg X, const int64_t *mptr, int32_t *midx) {
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= X.p) return;
  const uint8_t *col = X.geno + s * X.ld;
  int64_t pos = mptr[s];
  for (int64_t i0 = 0; i0 < X.n; i0 += 32) {
    const int64_t i = i0 + lane;
    const bool m = i < X.n && is_missing(X, col, i);
    const unsigned bal = __ballot_sync(0xffffffffu, m);
    if (m) midx[pos + __popc(bal & ((1u << lane) - 1u))] = (int32_t)i;
    pos += __popc(bal);
  }
}

cudaError_t launch_miss_fill(const Dsg &X, const int64_t *mptr, int32_t *midx, cudaStream_t s) {
  if (X.p == 0) return cudaSuccess;
  const int64_t threads = X.p * 32;
  k_miss_fill<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(X, mptr, midx);
  return cudaGetLastError();
}

// dst: a copy of the int8 stored columns (same ld) with missing codes set to 0.
__global__ void k_sanitize_int8(Dsg X, uint8_t *dst) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // one 16-byte chunk
  const int64_t per = X.ld / 16;
  if (g >= X.p * per) return;
  const uint4 v = reinterpret_cast<const uint4 *>(X.geno)[g];
  uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t o = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const uint32_t byte = (w[q] >> (8 * t)) & 0xffu;
      o |= (byte <= 2u ? byte : 0u) << (8 * t);
    }
    w[q] = o;
  }
  reinterpret_cast<uint4 *>(dst)[g] = make_uint4(w[0], w[1], w[2], w[3]);
}

cudaError_t launch_sanitize_int8(const Dsg &X, uint8_t *dst, cudaStream_t s) {
  const int64_t chunks = X.p * (X.ld / 16);
  if (chunks == 0) return cudaSuccess;
  k_sanitize_int8<<<(unsigned)((chunks + 255) / 256), 256, 0, s>>>(X, dst);
  return cudaGetLastError();
}

// One warp per stored column j of block g: u[g*npad + i] -= b_j v_j at its
// missing samples (atomic FP64 adds: the order of the few corrections per
// sample is not fixed).
__global__ void k_miss_xv(Dsg X, const double *v, const int64_t *block_ptr, int G, double *u, int64_t npad) {
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= X.p) return;
  const int64_t j = 1 + X.c + s;
  const double c = -X.b[j] * v[j];
  if (c == 0.0) return;
  int lo = 0, hi = G;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (block_ptr[mid] <= j) lo = mid; else hi = mid;
  }
  double *ug = u + (int64_t)lo * npad;
  for (int64_t e = X.mptr[s] + lane; e < X.mptr[s + 1]; e += 32) atomicAdd(ug + X.midx[e], c);
}

cudaError_t launch_miss_xv(const Dsg &X, const double *v, const int64_t *block_ptr, int G, double *u,
                           int64_t npad, cudaStream_t s) {
  if (X.p == 0 || X.mptr == nullptr) return cudaSuccess;
  const int64_t threads = X.p * 32;
  k_miss_xv<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(X, v, block_ptr, G, u, npad);
  return cudaGetLastError();
}

}  // namespace fsqr

namespace fsqr {

// ------------------------------------------------ screening (strong rule)

// dst column q = src column sel[q] (ld bytes each, 16-byte chunks).
__global__ void k_gather_cols(const uint8_t *src, int64_t ld, const int32_t *sel, int64_t nsel, uint8_t *dst) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = ld / 16;
  if (g >= nsel * per) return;
  const int64_t q = g / per, c = g - q * per;
  reinterpret_cast<uint4 *>(dst + q * ld)[c] = reinterpret_cast<const uint4 *>(src + (int64_t)sel[q] * ld)[c];
}

cudaError_t launch_gather_cols(const uint8_t *src, int64_t ld, const int32_t *sel, int64_t nsel, uint8_t *dst,
                               cudaStream_t s) {
  const int64_t chunks = nsel * (ld / 16);
  if (chunks == 0) return cudaSuccess;
  k_gather_cols<<<(unsigned)((chunks + 255) / 256), 256, 0, s>>>(src, ld, sel, nsel, dst);
  return cudaGetLastError();
}

// dst[b*ldd + q] = src[b*lds + idx[q]] for b < nb, q < m (gather) or, with
// scatter = 1, dst[b*ldd + idx[q]] = src[b*lds + q].
__global__ void k_index_copy(const double *src, int64_t lds, const int32_t *idx, int64_t m, int nb, double *dst,
                             int64_t ldd, int scatter) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= m * nb) return;
  const int b = (int)(g / m);
  const int64_t q = g - (int64_t)b * m;
  if (scatter) dst[b * ldd + idx[q]] = src[b * lds + q];
  else dst[b * ldd + q] = src[b * lds + idx[q]];
}

cudaError_t launch_index_copy(const double *src, int64_t lds, const int32_t *idx, int64_t m, int nb, double *dst,
                              int64_t ldd, int scatter, cudaStream_t s) {
  if (m * nb == 0) return cudaSuccess;
  k_index_copy<<<(unsigned)((m * nb + 255) / 256), 256, 0, s>>>(src, lds, idx, m, nb, dst, ldd, scatter);
  return cudaGetLastError();
}

}  // namespace fsqr
