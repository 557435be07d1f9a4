// Wide groups of the tensor-core iteration: NB = 16 or 32 fit slots share
// every pass over X (the batched tau x lambda grid).
//
// The arithmetic is that of k_tc.cu (exact integer digit products, FP64
// state, Algorithm 1 step by step); what changes is the width:
//   * theta of every slot is split into 7 balanced base-16 E4M3 digits, at
//     rows 8b .. 8b+6 of the digit matrix (row 8b+7 stays zero), so the MMA
//     has N = 8 NB rows (128 or 256) and a 16-column TMEM load holds exactly
//     two slots;
//   * the epilogue walks the accumulator two slots at a time and reduces the
//     per-slot stop-test partials with warp shuffles into shared memory, so
//     no per-thread array grows with NB;
//   * the per-slot parameters (tau, lambda, lambda_max, the iteration at which
//     the fit entered its slot) are device arrays: the host refills a slot
//     with the next fit between replays of the captured iteration graph.
// A slot is idle while done[b] >= 0: its digits are zero and no state of it
// is written.
#include <cuda.h>
#include <math.h>
#include <stdint.h>

#include "fsqr_device.cuh"
#include "fsqr_internal.h"
#include "sm103_ops.cuh"

namespace fsqr {

using namespace sm103;

// E4M3 encodings of the integers -8..8 (index t + 8).
__constant__ uint8_t kWE4M3[17] = {0xD0, 0xCE, 0xCC, 0xCA, 0xC8, 0xC4, 0xC0, 0xB8, 0x00,
                                   0x38, 0x40, 0x44, 0x48, 0x4A, 0x4C, 0x4E, 0x50};

template <int NB>
struct WShape {
  static constexpr int D = 7;                      // theta digits per slot
  static constexpr int N = 8 * NB;                 // digit rows (128 or 256)
  static constexpr int ACC = N <= 128 ? 4 : 2;     // TMEM accumulators (ACC * N = 512 columns)
  static constexpr int STAGES = N <= 128 ? 6 : 4;  // 32 KB or 48 KB stages
  static constexpr int A_BYTES = 128 * 128;
  static constexpr int B_BYTES = N * 128;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int THREADS = 256;
};

// X~ beta weights: 11 base-16 digits per slot, rows 11b + d; NH MMAs of
// NX rows each cover the 11 NB rows, accumulating at TMEM columns 256 h.
template <int NB>
struct WXShape {
  static constexpr int DW = 11;
  static constexpr int NR = DW * NB;               // 176 or 352
  static constexpr int NH = NR > 256 ? 2 : 1;
  static constexpr int NX = NR / NH;               // 176
  static constexpr int LAG = NB > 16 ? 1 : 2;      // blocks in flight per thread
  static constexpr int STAGES = LAG + 2;
  static constexpr int A_BYTES = 128 * 128;
  static constexpr int B_BYTES = NR * 128;
  static constexpr int BUF = A_BYTES + B_BYTES;
};

__device__ __forceinline__ double wdist(double s, double lam, double b) {
  if (b > 0.0) return fabs(s - lam);
  if (b < 0.0) return fabs(s + lam);
  return fmax(fabs(s) - lam, 0.0);
}

__device__ __forceinline__ int wblock_of(const int64_t *__restrict__ bp, int G, int64_t j) {
  int lo = 0, hi = G;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(bp + mid) <= j) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ double wmax32(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double wsum32(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------ theta digits

// theta^k of every live slot / scale_b rounded to a 28-bit fixed-point
// integer and split into 7 balanced base-16 digits (E4M3 bytes) at rows
// 8b .. 8b+6 of the swizzled digit tiles; idle slots get zero digits.
template <int NB>
__global__ void __launch_bounds__(256) k_wquant(Fits F, int off, uint8_t *dg) {
  constexpr int N = WShape<NB>::N;
  const int k = *F.it_base + off;
  __shared__ double sInv[NB];
  if (threadIdx.x < NB) {
    const int b = threadIdx.x;
    const double m = F.tot_c[k & 1][b * kCPartials + 3];
    int E = 0;
    if (m > 0.0) frexp(m, &E);
    const double scale = (m > 0.0) ? ldexp(1.0, E + 1) : 1.0;
    sInv[b] = (F.done[b] < 0) ? ldexp(1.0, 28) / scale : 0.0;
    if (blockIdx.x == 0) F.scale[b] = scale;
  }
  __syncthreads();
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = (int)(g / F.npad);
  const int64_t i = g - (int64_t)b * F.npad;
  if (b >= NB) return;
  long long Xq = fixed_point(F.theta[i * NB + b] * sInv[b]);
  int dig[7];
#pragma unroll
  for (int d = 6; d >= 1; --d) {
    const int t = (int)(((Xq + 8) & 15) - 8);
    dig[d] = t;
    Xq = (Xq - t) >> 4;
  }
  dig[0] = (int)Xq;
  const int64_t kc = i >> 7;
  const int c = (int)((i & 127) >> 4), bt = (int)(i & 15);
#pragma unroll
  for (int d = 0; d < 7; ++d) {
    const int r = 8 * b + d;
    dg[kc * (N * 128) + r * 128 + ((c ^ (r & 7)) << 4) + bt] = kWE4M3[dig[d] + 8];
  }
}

// --------------------------------------------------------------- column pass

// s_j = x~_j^T theta^k for every slot and column, the beta prox (eq.
// beta_update), the stop-test distance of beta^k and the active list of
// beta^{k+1}. Persistent, one CTA per SM: CTA c takes the 128-column tiles
// c, c + grid, ... (the leftover tiles of a partial last round go to CTAs
// 0 .. rem-1). Roles: warp 0 bulk-copy producer, warp 1 MMA issuer, warps
// 2-5 epilogue (one tile column per thread), warps 6-7 the FP64 dense
// columns j <= c.
template <int NB>
__global__ void __launch_bounds__(256, 1)
    k_wcol(Dsg X, Fits F, int off, const uint8_t *__restrict__ xt, const uint8_t *__restrict__ dgt,
           int rounds, int *err) {
  using Sh = WShape<NB>;
  constexpr int N = Sh::N;
  constexpr int S = Sh::STAGES;
  constexpr int kAcc = Sh::ACC;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[S], empty[S], accf[kAcc], acce[kAcc], drain;
  __shared__ uint32_t tmem_base;
  __shared__ double sS[NB], sScale[NB], sLam[NB];
  __shared__ float sSf[NB], sScalef[NB], sLamf[NB];
  __shared__ int sIdle[NB];
  __shared__ double s_part[4][NB][3];  // per epilogue warp: max dist, sum b_j beta_j, max |a_j beta_j|
  __shared__ double s_dpart[NB][3];    // the dense columns' share
  __shared__ double s_dot[2][NB];
  __shared__ int scan[Sh::THREADS];
  __shared__ int s_dense_act[64];
  __shared__ int s_ndense;

  const uint32_t base_u32 = smem_u32(smem_raw);
  uint8_t *ring = smem_raw + (((base_u32 + 1023u) & ~1023u) - base_u32);
  uint8_t *flags = ring + S * Sh::STAGE_BYTES;
  const int T = F.T;
  const int TF = 128 * (rounds + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = *F.it_base + off;
  const bool chk = (k % F.K) == 0;  // a stop-test step
  const double *bcur = F.beta[k & 1];
  double *bnxt = F.beta[(k & 1) ^ 1];
  const int64_t ntiles = (X.p + 127) / 128;
  const int rem = (int)(ntiles - (int64_t)rounds * gridDim.x);
  const int R = rounds + ((int)blockIdx.x < rem ? 1 : 0);
  const int nk = (int)((X.n + 127) / 128);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int a = 0; a < kAcc; ++a) { mbar_init(&accf[a], 1); mbar_init(&acce[a], 128); }
    mbar_init(&drain, 1);
    fence_mbar_init();
    s_ndense = 0;
  }
  if (threadIdx.x < NB) {
    const int b = threadIdx.x;
    sS[b] = F.tot_c[k & 1][b * kCPartials + 2];
    sIdle[b] = F.done[b] >= 0;
    sScale[b] = F.scale[b] * ldexp(1.0, -28);
    sLam[b] = F.w_lam[b];
    sSf[b] = (float)sS[b];
    sScalef[b] = (float)sScale[b];
    sLamf[b] = (float)sLam[b];
  }
  for (int t = threadIdx.x; t < 4 * NB * 3; t += Sh::THREADS) (&s_part[0][0][0])[t] = 0.0;
  for (int t = threadIdx.x; t < NB * 3; t += Sh::THREADS) (&s_dpart[0][0])[t] = 0.0;
  for (int t = threadIdx.x; t < TF; t += Sh::THREADS) flags[t] = 0;
  if (warp == 1) tmem_alloc(&tmem_base, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    // ---------------------------------------------------------- bulk-copy producer
    if (lane == 0) {
      int it = 0;
      for (int lt = 0; lt < R; ++lt) {
        const int tile = (int)blockIdx.x + lt * (int)gridDim.x;
        for (int kc = 0; kc < nk; ++kc, ++it) {
          const int s = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, err, kErrEmpty)) goto producer_done;
          uint8_t *sa = ring + s * Sh::STAGE_BYTES;
          mbar_arrive_expect_tx(&full[s], Sh::STAGE_BYTES);
          bulk_load(sa, xt + ((int64_t)tile * nk + kc) * Sh::A_BYTES, Sh::A_BYTES, &full[s]);
          bulk_load(sa + Sh::A_BYTES, dgt + (int64_t)kc * Sh::B_BYTES, Sh::B_BYTES, &full[s]);
        }
      }
    producer_done:;
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_f32acc(0u, 128u, (uint32_t)N);
      int it = 0;
      for (int lt = 0; lt < R; ++lt) {
        const int ab = lt % kAcc;
        const uint32_t aph = (uint32_t)(lt / kAcc) & 1u;
        if (!mbar_wait(&acce[ab], aph ^ 1u, err, kErrAccEmpty)) break;
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(ab * N);
        bool ok = true;
        for (int kc = 0; kc < nk; ++kc, ++it) {
          const int s = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          if (!mbar_wait(&full[s], ph, err, kErrFull)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(ring + s * Sh::STAGE_BYTES);
          const uint64_t ad = sdesc_k128(sa), bd = sdesc_k128(sa + Sh::A_BYTES);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma_f8(dt, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc, (kc != 0 || kk != 0) ? 1u : 0u);
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&accf[ab]);
      }
      mma_commit(&drain);
      mbar_wait(&drain, 0u, err, kErrFull);
    }
  } else if (warp >= 6) {
    // --------------------------------------------------- dense columns (FP64)
    const int dl = threadIdx.x - 192;  // 0..63
    for (int64_t j = blockIdx.x; j <= X.c; j += gridDim.x) {
      double dot[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) dot[b] = 0.0;
      if (j >= 1) {
        const double *cv = X.cov + (j - 1) * X.n;
        for (int64_t i = dl; i < X.n; i += 64) {
          const double x = __ldg(cv + i);
#pragma unroll
          for (int b = 0; b < NB; ++b) dot[b] = fma(x, F.theta[i * NB + b], dot[b]);
        }
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) dot[b] = wsum32(dot[b]);
      if (lane == 0)
#pragma unroll
        for (int b = 0; b < NB; ++b) s_dot[warp - 6][b] = dot[b];
      asm volatile("bar.sync 1, 64;" ::: "memory");
      if (dl == 0) {
        const double aj = X.a[j], bj = X.b[j], om = F.omega[j];
        const int g = wblock_of(F.block_ptr, F.G, j);
        const double gj = F.ridge * om;  // elastic-net quadratic weight (0: weighted l1)
        const double eta = F.eta[g], ie = gj == 0.0 ? F.inv_eta[g] : 1.0 / (F.eta[g] + gj);
        bool act = false;
        for (int b = 0; b < NB; ++b) {
          if (sIdle[b]) continue;
          const double s = aj * (s_dot[0][b] + s_dot[1][b]) + bj * sS[b];
          const double lamj = sLam[b] * om;
          const double bo = bcur[j * NB + b];
          if (j >= 1) s_dpart[b][0] = fmax(s_dpart[b][0], wdist(gj == 0.0 ? s : s - gj * bo, lamj, bo));
          const double av = eta * bo + s;
          const double bn = (fmax(av - lamj, 0.0) - fmax(-av - lamj, 0.0)) * ie;
          bnxt[j * NB + b] = bn;
          s_dpart[b][1] = fma(bj, bn, s_dpart[b][1]);
          act = act || (bn != 0.0 && j >= 1);
        }
        if (act) s_dense_act[s_ndense++] = (int)j;
      }
      asm volatile("bar.sync 1, 64;" ::: "memory");
    }
  } else {
    // -------------------------------------------------------------- epilogue
    const int q = warp & 3;           // TMEM lane quarter of this warp
    const int m = q * 32 + lane;      // tile row = column within the tile
    for (int lt = 0; lt < R; ++lt) {
      const int ab = lt % kAcc;
      const uint32_t aph = (uint32_t)(lt / kAcc) & 1u;
      const int tile = blockIdx.x + lt * gridDim.x;
      const int64_t sidx = (int64_t)tile * 128 + m;
      const bool live = sidx < X.p;
      const int64_t j = 1 + X.c + (live ? sidx : 0);
      const double aj = __ldg(X.a + j), bj = __ldg(X.b + j);
      const double om = __ldg(F.omega + j);
      const double gj = F.ridge * om;  // elastic-net quadratic weight (0: weighted l1)
      const int g = wblock_of(F.block_ptr, F.G, j);
      const double eta = __ldg(F.eta + g);
      const double ie = gj == 0.0 ? __ldg(F.inv_eta + g) : 1.0 / (eta + gj);
      // FP32 copies for the pre-test below; 1 - 2^-20 keeps the threshold
      // below the FP64 lambda_j whatever the two FP32 roundings did
      const float ajf = (float)aj, bjf = (float)bj, omf = (float)om * (1.0f - 9.5367431640625e-7f);
      const bool screen = live && X.mptr == nullptr;
      if (!mbar_wait(&accf[ab], aph, err, kErrAccFull)) break;
      tc_fence_after();
      bool act = false;
      for (int cc = 0; cc < NB / 2; ++cc) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * N + 16 * cc), r);
        tmem_wait_ld();
        const double2 bo2 = live ? *reinterpret_cast<const double2 *>(bcur + j * NB + 2 * cc)
                                 : make_double2(0.0, 0.0);
        double bn2[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int b = 2 * cc + h;
          long long V = 0;
#pragma unroll
          for (int d = 0; d < 7; ++d) V = V * 16 + (long long)__float2int_rn(__uint_as_float(r[8 * h + d]) * 512.0f);
          const double bo = h ? bo2.y : bo2.x;
          double rb = 0.0, ct = 0.0, wm = 0.0;
          bn2[h] = bo;
          // Exact FP32 pre-test (FP64 runs at a small fraction of the FP32
          // rate on this part): with beta_j = 0 and |s_j| < lambda_j the
          // FP64 step gives beta_j^{k+1} = 0 and a zero stop-test distance.
          // Each of the five FP32 roundings in s32 is within 2^-24 of its
          // operands, so |s - s32| <= 2^-21 (|t1| + |t2|) bounds the error.
          bool zero = false;
          if (screen && bo == 0.0 && !sIdle[b]) {
            const float t1 = ajf * ((float)V * sScalef[b]), t2 = bjf * sSf[b];
            const float s32 = t1 + t2;
            const float e32 = (fabsf(t1) + fabsf(t2)) * 4.76837158203125e-7f;
            zero = fabsf(s32) + e32 < sLamf[b] * omf;
          }
          float wmf = 0.0f;
          if (zero) {
            bn2[h] = 0.0;
          } else if (live && !sIdle[b]) {
            // mean imputation: missing entries read as 0, so their b_j theta_i is taken back out
            const double mc = X.mptr ? miss_dot(X, sidx, F.theta, NB, b) : 0.0;
            const double s = aj * ((double)V * sScale[b]) + bj * (sS[b] - mc);
            const double lamj = sLam[b] * om;
            // the stop test reads the distance only at its own steps
            if (chk) rb = wdist(gj == 0.0 ? s : s - gj * bo, lamj, bo);
            // eq. beta_update: the soft threshold of av at lamj, over eta_g (+ gamma_j)
            const double av = eta * bo + s;
            const double bn = fabs(av) > lamj ? copysign(fabs(av) - lamj, av) * ie : 0.0;
            bn2[h] = bn;
            ct = bj * bn;
            act = act || (bn != 0.0);
            // max |a_j beta_j| only sets the power-of-two scale of the X~ beta
            // digits: rounded up to FP32 it stays an upper bound
            wmf = __double2float_ru(fabs(aj * bn));
          }
          // the warp's partials (skipped when every lane's are zero)
          if (__any_sync(0xffffffffu, rb != 0.0 || ct != 0.0 || wmf != 0.0f)) {
            if (chk) rb = wmax32(rb);
            ct = wsum32(ct);
#pragma unroll
            for (int o = 16; o; o >>= 1) wmf = fmaxf(wmf, __shfl_xor_sync(0xffffffffu, wmf, o));
            wm = (double)wmf;
            if (lane == 0) {
              s_part[q][b][0] = fmax(s_part[q][b][0], rb);
              s_part[q][b][1] += ct;
              s_part[q][b][2] = fmax(s_part[q][b][2], wm);
            }
          }
        }
        // idle slots keep their (unused) next-iterate entries untouched
        if (live) {
          if (!sIdle[2 * cc] && !sIdle[2 * cc + 1])
            *reinterpret_cast<double2 *>(bnxt + j * NB + 2 * cc) = make_double2(bn2[0], bn2[1]);
          else if (!sIdle[2 * cc])
            bnxt[j * NB + 2 * cc] = bn2[0];
          else if (!sIdle[2 * cc + 1])
            bnxt[j * NB + 2 * cc + 1] = bn2[1];
        }
      }
      tc_fence_before();
      mbar_arrive(&acce[ab]);
      if (act) flags[lt * 128 + m] = 1;
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
  // per-CTA partials in a fixed order
  if (threadIdx.x < NB) {
    const int b = threadIdx.x;
    double rb = s_dpart[b][0], ct = 0.0, wm = 0.0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      rb = fmax(rb, s_part[w][b][0]);
      ct += s_part[w][b][1];
      wm = fmax(wm, s_part[w][b][2]);
    }
    ct += s_dpart[b][1];
    F.a_rb[blockIdx.x * NB + b] = rb;
    F.a_ct[blockIdx.x * NB + b] = ct;
    F.a_wmax[blockIdx.x * NB + b] = wm;
  }
  // ordered compaction of the active flags (local tile order), then the
  // active dense columns
  const int per = (TF + Sh::THREADS - 1) / Sh::THREADS;
  const int t0 = min(TF, (int)threadIdx.x * per), t1 = min(TF, t0 + per);
  int cnt = 0;
  for (int t = t0; t < t1; ++t) cnt += flags[t];
  scan[threadIdx.x] = cnt;
  __syncthreads();
  for (int o = 1; o < Sh::THREADS; o <<= 1) {
    int v = (threadIdx.x >= (unsigned)o) ? scan[threadIdx.x - o] : 0;
    __syncthreads();
    scan[threadIdx.x] += v;
    __syncthreads();
  }
  int pos = scan[threadIdx.x] - cnt;
  int *lst = F.a_list + (int64_t)blockIdx.x * T;
  for (int t = t0; t < t1; ++t)
    if (flags[t]) {
      const int64_t tile = blockIdx.x + (int64_t)(t >> 7) * gridDim.x;
      lst[pos++] = (int)(1 + X.c + tile * 128 + (t & 127));
    }
  if (threadIdx.x == Sh::THREADS - 1) {
    int tot = scan[Sh::THREADS - 1];
    for (int d = 0; d < s_ndense; ++d) lst[tot++] = s_dense_act[d];
    F.a_cnt[blockIdx.x] = tot;
  }
  col_finalize<NB>(F);
}


// ---------------------------------------------------------------- stop test

// Stop test of the iterate w^k of every running slot (k a multiple of K,
// at least one step after the fit entered its slot): KKT = max(R_p, R_z,
// R_b, R_1) with the rounding bound of the digit products added to R_b;
// the slot stops at KKT <= tol, after max_iter of its own steps, or on NaN.
template <int NB>
__global__ void __launch_bounds__(32) k_wcheck(Fits F, int off) {
  const int k = *F.it_base + off;
  const int b = threadIdx.x + 32 * blockIdx.x;
  if (b >= NB || F.done[b] >= 0) return;
  const int k0 = F.w_k0[b];
  if (k <= k0) return;
  const double *tc = F.tot_c[k & 1] + b * kCPartials;
  const double rb = F.tot_a[b * 3 + 0];
  const double lamnorm = F.w_lamnorm[b];
  const double bound = 0.5 * F.colbound * F.scale[b] * F.th_unit;
  const double R_p = tc[0] / (1.0 + F.ymax);
  const double R_z = tc[1];
  const double R_b = (rb + bound) / lamnorm;
  const double R_1 = fabs(tc[2]);
  const double kkt = fmax(fmax(R_p, R_z), fmax(R_b, R_1));
  const bool bad = isnan(R_p) || isnan(R_z) || isnan(R_b) || isnan(R_1) || isinf(kkt);
  double *rep = F.report + b * kReport;
  rep[0] = kkt; rep[1] = R_p; rep[2] = R_z; rep[3] = R_b; rep[4] = R_1;
  rep[6] = bound / lamnorm;
  rep[7] = k - k0;
  if (bad || kkt <= F.tol || k - k0 >= F.max_iter) {
    rep[5] = bad ? FSQR_ENUMERIC : (kkt <= F.tol ? FSQR_OK : FSQR_ENOCONV);
    F.done[b] = k;
    atomicAdd(F.n_done, 1);
  }
}

// ------------------------------------------------------------ slot set-up

// Partials of the current iterate (z, theta, r) of each masked slot:
// tot_c[par][b*4 + q] = max |r_i|, max_i dist(n theta_i, d rho_tau(z_i)),
// sum theta_i, max |theta_i| (fixed-order reductions; one CTA per slot).
template <int NB>
__global__ void __launch_bounds__(256) k_slot_init(Fits F, int par, const int *__restrict__ mask) {
  const int b = blockIdx.x;
  if (b >= NB || mask[b] == 0) return;
  __shared__ double red[kCPartials][256];
  const double tau = F.w_tau[b];
  const double n = (double)F.n;
  double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
  for (int64_t i = threadIdx.x; i < F.n; i += 256) {
    const double zi = F.z[i * NB + b], ti = F.theta[i * NB + b], ri = F.r[i * NB + b];
    p0 = fmax(p0, fabs(ri));
    p1 = fmax(p1, dist_pinball(n * ti, zi, tau));
    p2 += ti;
    p3 = fmax(p3, fabs(ti));
  }
  red[0][threadIdx.x] = p0;
  red[1][threadIdx.x] = p1;
  red[2][threadIdx.x] = p2;
  red[3][threadIdx.x] = p3;
  __syncthreads();
  const int ops[4] = {0, 0, 1, 0};
  tree_reduce<4>(red, ops, 256);
  if (threadIdx.x < kCPartials) F.tot_c[par][b * kCPartials + threadIdx.x] = red[threadIdx.x][0];
}

// ------------------------------------------------------------ X~ beta (wide)

// One thread per active position of the union list: its stored column and
// the 11 base-16 digits of w_jb = a_j beta_jb / scale_b * 2^44 of every
// running slot, as the byte image of a K-major swizzled operand tile (rows
// 11b + d) per block of 128 active positions.
template <int NB>
__global__ void __launch_bounds__(128)
    k_wxprep(Dsg X, Fits F, int off, const double *__restrict__ beta_in, int split_cap, int *__restrict__ scol,
             uint8_t *__restrict__ wtile, int *err) {
  using Sh = WXShape<NB>;
  extern __shared__ int spre[];  // gridA + 1
  __shared__ double sInv[NB];
  const double *beta = beta_in;
  if (beta == nullptr) {
    const int k = *F.it_base + off;
    beta = F.beta[(k & 1) ^ 1];
  }
  const int gA = F.gridA;
  int A = __ldcg(F.a_pre + gA);
  if (A >= (1 << 19)) {  // the exact integer sums need fewer than 2^19 active columns
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(err, 0, 5);
    A = 0;
  }
  const int nkb = (A + 127) / 128;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    F.meta_i[0] = max(1, min(16, min(nkb, split_cap)));
    F.meta_i[1] = A;
  }
  if (threadIdx.x < NB) {
    const int b = threadIdx.x;
    const double m = F.tot_a[b * 3 + 2];
    int E = 0;
    if (m > 0.0) frexp(m, &E);
    const double scale = (m > 0.0) ? ldexp(1.0, E + 1) : 1.0;
    sInv[b] = (F.done[b] < 0) ? ldexp(1.0, 44) / scale : 0.0;
    if (blockIdx.x == 0) {
      F.meta_d[b] = F.tot_a[b * 3 + 1];
      F.meta_d[kWideMax + b] = scale;
    }
  }
  if ((int)blockIdx.x >= nkb) return;
  for (int t = threadIdx.x; t <= gA; t += 128) spre[t] = __ldcg(F.a_pre + t);
  __syncthreads();
  const int t = threadIdx.x, ch = t >> 4, bt = t & 15;
  for (int kb = blockIdx.x; kb < nkb; kb += gridDim.x) {
    const int a = kb * 128 + t;
    int j = -1;
    if (a < A) {
      int lo = 0, hi = gA;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (spre[mid] <= a) lo = mid; else hi = mid;
      }
      j = F.a_list[(int64_t)lo * F.T + (a - spre[lo])];
      if (j <= X.c) j = -1;  // covariates are summed in FP64 by the vector update
    }
    scol[a] = (j >= 0) ? (int)(j - 1 - X.c) : (int)X.p;
    uint8_t *tile = wtile + (int64_t)kb * Sh::B_BYTES;
    const double aj = (j >= 0) ? __ldg(X.a + j) : 0.0;
    for (int b = 0; b < NB; ++b) {
      long long W = (j >= 0) ? fixed_point(aj * beta[(int64_t)j * NB + b] * sInv[b]) : 0;
      int dig[11];
#pragma unroll
      for (int d = 10; d >= 1; --d) {
        const int tt = (int)(((W + 8) & 15) - 8);
        dig[d] = tt;
        W = (W - tt) >> 4;
      }
      dig[0] = (int)W;
#pragma unroll
      for (int d = 0; d < 11; ++d) {
        const int r = b * 11 + d;
        tile[r * 128 + ((ch ^ (r & 7)) << 4) + bt] = kWE4M3[dig[d] + 8];
      }
    }
  }
}

// CTA (rt, sp): samples [128 rt, +128) over the active blocks of split sp,
// as k_xbeta_tc: 16-byte asynchronous copies of the active columns' sample
// runs (MN-major operand), a bulk copy of the block's weight-digit tile, NH
// MMAs of NX rows each into TMEM. The last split CTA of a row tile sums the
// splits' exact int64 partials and applies the vector update of every
// running slot (eq. z_update, the extrapolated theta step) with the
// stop-test partials; the last row tile writes the totals.
template <int NB>
__global__ void __launch_bounds__(128)
    k_wxbeta(Dsg X, Fits F, int off, int fuse, const int *__restrict__ scol, const uint8_t *__restrict__ wtile,
             int *err) {
  using Sh = WXShape<NB>;
  constexpr int ST = Sh::STAGES;
  constexpr int LAG = Sh::LAG;
  constexpr int TMEM_COLS = Sh::NR <= 256 ? 256 : 512;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[ST], empty[ST], dbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_last;
  __shared__ double s_red[4][NB][kCPartials];
  __shared__ double sTau[NB];
  __shared__ int sRun[NB];
  const uint32_t base_u32 = smem_u32(smem_raw);
  uint8_t *ring = smem_raw + (((base_u32 + 1023u) & ~1023u) - base_u32);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int A = F.meta_i[1];
  const int nkb = (A + 127) / 128;
  const int S = F.meta_i[0];
  if ((int)blockIdx.y >= S) return;
  const int kb0 = (int)((int64_t)nkb * blockIdx.y / S), kb1 = (int)((int64_t)nkb * (blockIdx.y + 1) / S);
  const bool has = kb1 > kb0;
  const int64_t i0 = (int64_t)blockIdx.x * 128;
  const int64_t i = i0 + tid;
  const bool row = i < F.n;
  long long *out = F.xb_ipart + (int64_t)blockIdx.y * F.npad * NB;

  long long V[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) V[b] = 0;
  if (has) {
    if (tid == 0) {
      for (int q = 0; q < ST; ++q) { mbar_init(&full[q], 128); mbar_init(&empty[q], 1); }
      mbar_init(&dbar, 1);
      fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&tmem_base, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = idesc_f32acc_amn(0u, 128u, (uint32_t)Sh::NX);
    const int c = tid & 7, kr = tid >> 3;
    const int64_t s0 = i0 + 16 * c;
    const uint32_t valid = s0 < F.n ? (uint32_t)(F.n - s0 < 16 ? F.n - s0 : 16) : 0u;
    const int nb = kb1 - kb0;
    bool ok = true;
    // iteration it: copy block it into its stage; release block it - LAG
    // (whose copies by this thread have landed) to the MMA issuer
    for (int it = 0; it < nb + LAG && ok; ++it) {
      if (it < nb) {
        const int s = it % ST;
        if (!mbar_wait(&empty[s], ((uint32_t)(it / ST) & 1u) ^ 1u, err, kErrEmpty)) { ok = false; break; }
        uint8_t *stage = ring + s * Sh::BUF;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int kk = 16 * e + kr;
          const int idx = __ldg(scol + (int64_t)(kb0 + it) * 128 + kk);
          uint8_t *dst = stage + kk * 128 + ((c ^ (kk & 7)) << 4);
          if (valid > 0 && idx < X.p)
            cp_async16(dst, X.geno + (int64_t)idx * X.ld + s0, valid);
          else
            *reinterpret_cast<int4 *>(dst) = make_int4(0, 0, 0, 0);
        }
        if (tid == 0) {
          mbar_expect_tx(&full[s], Sh::B_BYTES);
          bulk_load(stage + Sh::A_BYTES, wtile + (int64_t)(kb0 + it) * Sh::B_BYTES, Sh::B_BYTES, &full[s]);
        }
      }
      cp_async_commit();
      const int rt = it - LAG;
      if (rt >= 0 && rt < nb) {
        cp_async_wait<LAG>();
        fence_proxy_async();
        const int s = rt % ST;
        const uint32_t ph = (uint32_t)(rt / ST) & 1u;
        mbar_arrive(&full[s]);
        if (tid == 0) {
          if (!mbar_wait(&full[s], ph, err, kErrFull)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(ring + s * Sh::BUF);
          const uint64_t ad = sdesc_mn128(sa);
#pragma unroll
          for (int h = 0; h < Sh::NH; ++h) {
            const uint64_t bd = sdesc_k128(sa + Sh::A_BYTES + h * Sh::NX * 128);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              mma_f8(tmem + (uint32_t)(h * 256), ad + (uint64_t)(q * 256), bd + (uint64_t)(q * 2), idesc,
                     (rt | q) != 0 ? 1u : 0u);
          }
          mma_commit(&empty[s]);
        }
      }
    }
    cp_async_wait<0>();
    if (tid == 0) mma_commit(&dbar);
    __syncwarp();
    const bool done = mbar_wait(&dbar, 0u, err, kErrAccFull) && ok;
    tc_fence_after();
    // TMEM lane = sample row; half h of the slots starts at column 256 h,
    // where column 11 b' + d holds digit d of slot NB/NH h + b'
#pragma unroll
    for (int h = 0; h < Sh::NH; ++h) {
#pragma unroll
      for (int cc = 0; cc < Sh::NX / 16; ++cc) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(256 * h + 16 * cc), r);
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int col = 16 * cc + e;
          const int b = (NB / Sh::NH) * h + col / 11;
          V[b] = V[b] * 16 + (long long)__float2int_rn(__uint_as_float(r[e]) * 512.0f);
        }
      }
    }
    if (!done)
#pragma unroll
      for (int b = 0; b < NB; ++b) V[b] = 0;
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
      tc_fence_after();
      tmem_dealloc(tmem, TMEM_COLS);
    }
  }

  if (!fuse || S > 1) {
    if (i < F.npad)
#pragma unroll
      for (int b = 0; b < NB; ++b) out[i * NB + b] = V[b];
  }
  if (!fuse) return;

  // ---- fused vector update: the last split CTA of this row tile
  if (S > 1) {
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&F.xb_tick[blockIdx.x], 1u) == (unsigned)(S - 1)) ? 1 : 0;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (row) {
#pragma unroll
      for (int b = 0; b < NB; ++b) V[b] = 0;
      for (int sp = 0; sp < S; ++sp) {
        const long long *src = F.xb_ipart + ((int64_t)sp * F.npad + i) * NB;
#pragma unroll
        for (int b = 0; b < NB; ++b) V[b] += __ldcg(src + b);
      }
    }
    if (tid == 0) F.xb_tick[blockIdx.x] = 0u;
  }
  const int k = *F.it_base + off;
  if (tid < NB) {
    sTau[tid] = F.w_tau[tid];
    sRun[tid] = F.done[tid] < 0;
  }
  __syncthreads();
  const double *bt = F.beta[(k & 1) ^ 1];
  const double nmu = (double)F.n * F.mu;
  const double yi = row ? __ldg(F.y + i) : 0.0;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    double p[kCPartials] = {0.0, 0.0, 0.0, 0.0};
    double qc = 0.0;
    if (row && F.qcorr) {
      qc = F.qcorr[i * NB + b];
      F.qcorr[i * NB + b] = 0.0;
    }
    if (row && sRun[b]) {
      double cv = qc;
      for (int64_t j = 1; j <= X.c; ++j)
        cv = fma(__ldg(X.a + j) * bt[j * NB + b], __ldg(X.cov + (j - 1) * X.n + i), cv);
      const double unit = F.meta_d[kWideMax + b] * F.xb_unit;
      const double q = F.meta_d[b] + (double)V[b] * unit + cv;
      const int64_t ib = i * NB + b;
      row_update(F, ib, sTau[b], nmu, (double)F.n, q, (double)A * unit, yi, F.z[ib], F.theta[ib], F.r[ib], p);
    }
    p[0] = wmax32(p[0]);
    p[1] = wmax32(p[1]);
    p[2] = wsum32(p[2]);
    p[3] = wmax32(p[3]);
    if (lane == 0)
#pragma unroll
      for (int qq = 0; qq < kCPartials; ++qq) s_red[warp][b][qq] = p[qq];
  }
  __syncthreads();
  const int par = (k + 1) & 1;
  if (tid < NB) {
    const int b = tid;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      a0 = fmax(a0, s_red[w][b][0]);
      a1 = fmax(a1, s_red[w][b][1]);
      a2 += s_red[w][b][2];
      a3 = fmax(a3, s_red[w][b][3]);
    }
    double *cp = F.c_part[par] + (blockIdx.x * NB + b) * kCPartials;
    cp[0] = a0; cp[1] = a1; cp[2] = a2; cp[3] = a3;
  }
  vec_finalize<NB>(F, par, (int)gridDim.x);
}

// r[i NB + slot] = xb_i + z_i - y_i: the residual of a given start (rows
// i < n; padding rows stay 0).
__global__ void k_resid_slot(const double *__restrict__ xb, const double *__restrict__ z,
                             const double *__restrict__ y, int64_t n, double *r, int slot, int NB) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i * NB + slot] = xb[i] + z[i] - y[i];
}

cudaError_t launch_resid_slot(const double *xb, const double *z, const double *y, int64_t n, double *r, int slot,
                              int NB, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_resid_slot<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xb, z, y, n, r, slot, NB);
  return cudaGetLastError();
}

// ------------------------------------------------------------------- host

bool wide_ok(int NB) { return NB == 16 || NB == 32; }
int wide_rows(int NB) { return 8 * NB; }
int wide_xrows(int NB) { return 11 * NB; }

size_t wcol_smem(int NB, int T) {
  const size_t stage = 128 * 128 + (size_t)8 * NB * 128;
  const size_t stages = NB <= 16 ? 6 : 4;
  return stages * stage + 1024 + (size_t)T + 16;
}

size_t wxbeta_smem(int NB) {
  const size_t lag = NB > 16 ? 1 : 2;
  return (lag + 2) * (128 * 128 + (size_t)11 * NB * 128) + 1024 + 16;
}

template <int NB>
static cudaError_t wcol_t(const Dsg &X, const Fits &F, int off, const uint8_t *xt, const uint8_t *dgt, int rounds,
                          int *err, cudaStream_t s) {
  static size_t opted = 0;
  const size_t smem = wcol_smem(NB, F.T);
  if (smem > opted) {
    cudaError_t e = cudaFuncSetAttribute(k_wcol<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    opted = smem;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_wcol<NB><<<std::max(1, sms), 256, smem, s>>>(X, F, off, xt, dgt, rounds, err);
  return cudaGetLastError();
}

cudaError_t launch_wcol(int NB, const Dsg &X, const Fits &F, int off, const uint8_t *xt, const uint8_t *dgt,
                        int rounds, int *err, cudaStream_t s) {
  if (NB == 16) return wcol_t<16>(X, F, off, xt, dgt, rounds, err, s);
  if (NB == 32) return wcol_t<32>(X, F, off, xt, dgt, rounds, err, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_wquant(int NB, const Fits &F, int off, uint8_t *dg, cudaStream_t s) {
  const int64_t total = (int64_t)NB * F.npad;
  const unsigned grid = (unsigned)((total + 255) / 256);
  if (NB == 16) k_wquant<16><<<grid, 256, 0, s>>>(F, off, dg);
  else if (NB == 32) k_wquant<32><<<grid, 256, 0, s>>>(F, off, dg);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_wcheck(int NB, const Fits &F, int off, cudaStream_t s) {
  if (NB == 16) k_wcheck<16><<<1, 32, 0, s>>>(F, off);
  else if (NB == 32) k_wcheck<32><<<1, 32, 0, s>>>(F, off);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_slot_init(int NB, const Fits &F, int par, const int *mask, cudaStream_t s) {
  if (NB == 16) k_slot_init<16><<<16, 256, 0, s>>>(F, par, mask);
  else if (NB == 32) k_slot_init<32><<<32, 256, 0, s>>>(F, par, mask);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <int NB>
static cudaError_t wxbeta_t(const Dsg &X, const Fits &F, int off, int fuse, const double *beta_in, int *scol,
                            uint8_t *wtile, int *err, int num_sms, cudaStream_t s) {
  static size_t opted = 0;
  static int per_sm = 0;
  const size_t smem = wxbeta_smem(NB);
  if (smem > opted) {
    cudaError_t e = cudaFuncSetAttribute(k_wxbeta<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    opted = smem;
  }
  if (per_sm == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wxbeta<NB>, 128, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);
  }
  const int rows = (int)((X.n + 127) / 128);
  const int split_cap = std::max(1, per_sm * num_sms / rows);
  const int maxkb = (int)((X.P + 127) / 128);
  const int pgrid = std::max(1, std::min(maxkb, num_sms));
  const size_t psmem = (size_t)(F.gridA + 1) * sizeof(int);
  k_wxprep<NB><<<pgrid, 128, psmem, s>>>(X, F, off, beta_in, split_cap, scol, wtile, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)rows, 16);
  k_wxbeta<NB><<<grid, 128, smem, s>>>(X, F, off, fuse, scol, wtile, err);
  return cudaGetLastError();
}

cudaError_t launch_wxbeta(int NB, const Dsg &X, const Fits &F, int off, int fuse, const double *beta_in,
                          int *scol, uint8_t *wtile, int *err, int num_sms, cudaStream_t s) {
  if (NB == 16) return wxbeta_t<16>(X, F, off, fuse, beta_in, scol, wtile, err, num_sms, s);
  if (NB == 32) return wxbeta_t<32>(X, F, off, fuse, beta_in, scol, wtile, err, num_sms, s);
  return cudaErrorInvalidValue;
}

}  // namespace fsqr

namespace fsqr {

// Self-test of the bounded waits (failure detection without a GPU fault):
// one CTA initialises an mbarrier that expects one arrival; with arrive = 0
// nothing ever arrives (the wait must run out after `budget` cycles, record
// its code and return), with arrive = 1 thread 0 arrives first (the wait
// must succeed). No copy, MMA or tensor memory is involved.
__global__ void k_wait_selftest(long long budget, int arrive, int *err, int *ok) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && arrive) mbar_arrive(&bar);
  __syncthreads();
  if (threadIdx.x == 0) ok[0] = mbar_wait_for(&bar, 0u, err, kErrFull, budget) ? 1 : 0;
}

cudaError_t launch_wait_selftest(long long budget, int arrive, int *err, int *ok, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(budget, arrive, err, ok);
  return cudaGetLastError();
}

}  // namespace fsqr
