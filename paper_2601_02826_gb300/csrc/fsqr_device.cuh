// Device helpers shared by the column passes (SIMT and tensor core) and the
// vector kernel: the last CTA of a pass turns the per-CTA partials into the
// totals the next kernels read, in a fixed order (deterministic).
#pragma once

#include "fsqr_internal.h"

namespace fsqr {

// Fixed-order (deterministic) tree reduction of n = 2^m shared-memory values
// per array, for `cnt` arrays at once; ops[q] = 0 max, 1 sum. Every thread of
// the block must call it. Result in v[q][0].
template <int NQ>
__device__ __forceinline__ void tree_reduce(double (*v)[256], const int (&ops)[NQ], int n) {
  for (int o = n >> 1; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const double a = v[q][threadIdx.x], b = v[q][threadIdx.x + o];
        v[q][threadIdx.x] = ops[q] ? a + b : fmax(a, b);
      }
    }
    __syncthreads();
  }
}

// Called by every thread of every CTA of a column pass after the CTA wrote
// a_rb, a_ct, a_wmax and a_cnt. The last CTA to finish writes
//   tot_a[b*3 + 0] = max over CTAs of a_rb     (stop-test distance)
//   tot_a[b*3 + 1] = sum over CTAs of a_ct     (constant term of X~ beta)
//   tot_a[b*3 + 2] = max over CTAs of a_wmax   (scale of the integer X~ beta)
//   a_pre[0..gridA] = exclusive prefix of a_cnt (a_pre[gridA] = total)
template <int NB>
__device__ void col_finalize(const Fits &F) {
  __shared__ unsigned s_ticket;
  __shared__ double s_red[3][256];
  __shared__ int s_scan[256];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = atomicAdd(&F.tickets[0], 1u);
  __syncthreads();
  if (s_ticket != gridDim.x - 1) return;
  __threadfence();
  const int nt = min((int)blockDim.x, 256);  // a power of two
  const int t = threadIdx.x;
  const int gA = F.gridA;
  for (int b = 0; b < NB; ++b) {
    double rb = 0.0, ct = 0.0, wm = 0.0;
    if (t < nt)
#pragma unroll 4
      for (int c = t; c < gA; c += nt) {
        rb = fmax(rb, __ldcg(F.a_rb + c * NB + b));
        ct += __ldcg(F.a_ct + c * NB + b);
        if (F.a_wmax) wm = fmax(wm, __ldcg(F.a_wmax + c * NB + b));
      }
    if (t < nt) { s_red[0][t] = rb; s_red[1][t] = ct; s_red[2][t] = wm; }
    __syncthreads();
    const int ops[3] = {0, 1, 0};
    tree_reduce<3>(s_red, ops, nt);
    if (t == 0) {
      F.tot_a[b * 3 + 0] = s_red[0][0];
      F.tot_a[b * 3 + 1] = s_red[1][0];
      F.tot_a[b * 3 + 2] = s_red[2][0];
    }
    __syncthreads();
  }
  // exclusive prefix of the per-CTA active counts, in chunks of nt
  int carry = 0;
  for (int c0 = 0; c0 < gA; c0 += nt) {
    const int c = c0 + t;
    const int v = (t < nt && c < gA) ? __ldcg(F.a_cnt + c) : 0;
    if (t < nt) s_scan[t] = v;
    __syncthreads();
    for (int o = 1; o < nt; o <<= 1) {
      int u = (t < nt && t >= o) ? s_scan[t - o] : 0;
      __syncthreads();
      if (t < nt) s_scan[t] += u;
      __syncthreads();
    }
    if (t < nt && c < gA) F.a_pre[c] = carry + s_scan[t] - v;
    carry += s_scan[nt - 1];
    __syncthreads();
  }
  if (t == 0) {
    F.a_pre[gA] = carry;
    F.tickets[0] = 0u;
  }
}

// sum of v[i*NB + b] over the missing samples i of stored column s (0-based);
// 0 when the design has no missing entries.
__device__ __forceinline__ double miss_dot(const Dsg &X, int64_t s, const double *v, int NB, int b) {
  if (X.mptr == nullptr) return 0.0;
  double acc = 0.0;
  const int64_t e1 = X.mptr[s + 1];
  for (int64_t e = X.mptr[s]; e < e1; ++e) acc += v[(int64_t)X.midx[e] * NB + b];
  return acc;
}

// Fixed-point integer of v (already scaled): v rounded to the nearest
// integer. Finite iterates always give |v| < 2^44 here; a NaN or infinite
// iterate gives 0, so that digit extraction stays in range while the stop
// test reports the non-finite value.
__device__ __forceinline__ long long fixed_point(double v) {
  return (fabs(v) < 4.0e18) ? __double2ll_rn(v) : 0LL;
}

// dist(t, d rho_tau(z)): {tau} for z > 0, {tau-1} for z < 0, [tau-1, tau] at 0.
__device__ __forceinline__ double dist_pinball(double t, double z, double tau) {
  if (z > 0.0) return fabs(t - tau);
  if (z < 0.0) return fabs(t - (tau - 1.0));
  return fmax(fmax(tau - 1.0 - t, t - tau), 0.0);
}

// One sample of one fit, given q = x~_i^T beta^{k+1} (with its rounding
// bound qerr) and the old z, theta, r:
//   z^{k+1} = (v - tau/(n mu))_+ - (-v - (1-tau)/(n mu))_+,  v = z^k + theta^k/mu
//   r^{k+1} = q + z^{k+1} - y_i
//   theta^{k+1} = theta^k - mu/(G+1) (2 r^{k+1} - r^k)
// stores them at index ib and returns the stop-test partials of w^{k+1}.
__device__ __forceinline__ void row_update(const Fits &F, int64_t ib, double tau, double nmu, double n,
                                           double q, double qerr, double yi, double zo, double th,
                                           double ro, double *p) {
  const double v = zo + th / F.mu;
  // eq. z_update
  const double zn = fmax(v - tau / nmu, 0.0) - fmax(-v - (1.0 - tau) / nmu, 0.0);
  // eq. fsppa_update, theta line: extrapolated dual step of size mu/(G+1)
  const double rn = q + zn - yi;
  const double tn = th - F.sigma * (2.0 * rn - ro);
  F.z[ib] = zn;
  F.theta[ib] = tn;
  F.r[ib] = rn;
  p[0] = fabs(rn) + qerr;
  p[1] = dist_pinball(n * tn, zn, tau);
  p[2] = tn;
  p[3] = fabs(tn);
}

// Vector-pass counterpart: totals of the nparts per-CTA partials of the
// iterate of the given parity, tot_c[par][b*4 + q] (q: max |r|, max dist,
// sum theta, max |theta|). Called by the gridDim.x CTAs that wrote partials.
template <int NB>
__device__ void vec_finalize(const Fits &F, int par, int nparts) {
  __shared__ unsigned s_ticket;
  __shared__ double s_red[kCPartials][256];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = atomicAdd(&F.tickets[1], 1u);
  __syncthreads();
  if (s_ticket != gridDim.x - 1) return;
  __threadfence();
  const int nt = min((int)blockDim.x, 256);
  const int t = threadIdx.x;
  const double *cp = F.c_part[par];
  for (int b = 0; b < NB; ++b) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    if (t < nt)
#pragma unroll 4
      for (int c = t; c < nparts; c += nt) {
        const double *p = cp + (c * NB + b) * kCPartials;
        a0 = fmax(a0, __ldcg(p + 0));
        a1 = fmax(a1, __ldcg(p + 1));
        a2 += __ldcg(p + 2);
        a3 = fmax(a3, __ldcg(p + 3));
      }
    if (t < nt) { s_red[0][t] = a0; s_red[1][t] = a1; s_red[2][t] = a2; s_red[3][t] = a3; }
    __syncthreads();
    const int ops[4] = {0, 0, 1, 0};
    tree_reduce<4>(s_red, ops, nt);
    if (t == 0) {
      double *o = F.tot_c[par] + b * kCPartials;
      o[0] = s_red[0][0]; o[1] = s_red[1][0]; o[2] = s_red[2][0]; o[3] = s_red[3][0];
    }
    __syncthreads();
  }
  if (t == 0) F.tickets[1] = 0u;
}

}  // namespace fsqr
