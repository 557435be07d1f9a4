// Tensor-core column pass of the FS-QRPPA iteration (mixed arithmetic).
//
// s_j = x~_j^T theta^k over the stored genotype columns is computed as an
// exact integer product on the 5th-generation tensor cores:
//   * theta_b is rounded to a 4D-bit fixed-point integer and split into D
//     balanced base-16 digits t in [-8, 8]; every digit is an exact E4M3
//     value. The digits of the NB fits form an N x n matrix (rows b*D + d).
//   * The int8 genotype codes 0/1/2 read as E4M3 bit patterns are the
//     subnormals 0, 2^-9, 2^-8, i.e. exactly g * 2^-9, so the stored
//     matrix is loaded by TMA and multiplied with no conversion pass.
//   * tcgen05.mma kind::f8f6f4 (M = 128 columns, N = digit rows, K = 32
//     samples) accumulates g * t * 2^-9 in FP32 in tensor memory; every
//     partial sum is an integer multiple of 2^-9 below 2^24 * 2^-9, hence
//     exact. The epilogue recombines the digits exactly in int64.
// The FP64 proximal update (eq. beta_update), the stop-test distance and the
// active-column lists follow as in the SIMT column pass.
//
// Roles (192 threads): warp 0 issues TMA loads into a STAGES-deep ring,
// warp 1 issues the MMAs (one elected thread) into a double-buffered TMEM
// accumulator, warps 2-5 (128 threads, one per tile row) run the epilogue.
// CTA c takes the 128-column tiles c, c + grid, c + 2 grid, ...
#include <cuda.h>
#include <math.h>
#include <stdint.h>

#include "fsqr_internal.h"
#include "sm103_ops.cuh"

namespace fsqr {

using namespace sm103;

template <int NB, int D>
struct TcShape {
  static constexpr int NR = NB * D;
  static constexpr int N = NR <= 16 ? 16 : (NR <= 32 ? 32 : 64);
  static constexpr int TMEM_COLS = (2 * N <= 32) ? 32 : ((2 * N <= 64) ? 64 : 128);
  static constexpr int STAGES = 6;
  static constexpr int A_BYTES = 128 * 128;
  static constexpr int B_BYTES = N * 128;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int THREADS = 192;
};

__device__ __forceinline__ double dist_l1_tc(double s, double lam, double b) {
  if (b > 0.0) return fabs(s - lam);
  if (b < 0.0) return fabs(s + lam);
  return fmax(fabs(s) - lam, 0.0);
}

__device__ __forceinline__ int block_of_tc(const int64_t *__restrict__ bp, int G, int64_t j) {
  int lo = 0, hi = G;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(bp + mid) <= j) lo = mid; else hi = mid;
  }
  return lo;
}

template <int NB, int D>
__global__ void __launch_bounds__(192, 1)
    k_col_tc(Dsg X, Fits F, int off, const __grid_constant__ CUtensorMap tmX,
             const __grid_constant__ CUtensorMap tmD, int tiles_per_cta, int *err) {
  using Sh = TcShape<NB, D>;
  constexpr int N = Sh::N;
  constexpr int S = Sh::STAGES;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[S], empty[S], accf[2], acce[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ double sS[kMaxNB], sScale[kMaxNB];
  __shared__ int sIdle[kMaxNB];
  __shared__ double red_rb[128][NB], red_ct[128][NB], red_wm[128][NB];
  __shared__ int scan[Sh::THREADS];

  // 1024-aligned ring of stages, then the active flags of this CTA's columns
  const uint32_t base_u32 = smem_u32(smem_raw);
  uint8_t *ring = smem_raw + (((base_u32 + 1023u) & ~1023u) - base_u32);
  uint8_t *flags = ring + S * Sh::STAGE_BYTES;
  const int T = F.T;  // = 128 * tiles_per_cta

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = *F.it_base + off;
  const double *bcur = F.beta[k & 1];
  double *bnxt = F.beta[(k & 1) ^ 1];
  const int64_t ntiles = (X.p + 127) / 128;
  const int ntl = (int)((blockIdx.x < ntiles) ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0);
  const int nk = (int)((X.n + 127) / 128);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int a = 0; a < 2; ++a) { mbar_init(&accf[a], 1); mbar_init(&acce[a], 128); }
    mbar_init(&drain, 1);
    fence_mbar_init();
  }
  if (threadIdx.x < NB) {
    const int b = threadIdx.x;
    const double *cp = F.c_part[k & 1];
    double Ssum = 0.0;
    for (int c = 0; c < F.gridC; ++c) Ssum += cp[(c * NB + b) * kCPartials + 2];
    sS[b] = Ssum;
    sIdle[b] = (b >= F.nb) || (F.done[b] >= 0);
    sScale[b] = F.scale[b];
  }
  for (int t = threadIdx.x; t < T; t += Sh::THREADS) flags[t] = 0;
  if (warp == 0 && lane == 0) {
    prefetch_tmap(&tmX);
    prefetch_tmap(&tmD);
  }
  if (warp == 1) tmem_alloc(&tmem_base, Sh::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    // ---------------------------------------------------------- TMA producer
    if (lane == 0) {
      int it = 0;
      for (int lt = 0; lt < ntl; ++lt) {
        const int tile = blockIdx.x + lt * gridDim.x;
        for (int kc = 0; kc < nk; ++kc, ++it) {
          const int s = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, err, kErrEmpty)) goto producer_done;
          uint8_t *sa = ring + s * Sh::STAGE_BYTES;
          mbar_arrive_expect_tx(&full[s], Sh::STAGE_BYTES);
          tma_load_2d(sa, &tmX, &full[s], kc * 128, tile * 128);
          tma_load_2d(sa + Sh::A_BYTES, &tmD, &full[s], kc * 128, 0);
        }
      }
    producer_done:;
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_f32acc(0u, 128u, (uint32_t)N);
      int it = 0;
      for (int lt = 0; lt < ntl; ++lt) {
        const int ab = lt & 1;
        const uint32_t aph = (uint32_t)(lt >> 1) & 1u;
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
            mma_f8(dt, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc, (kc | kk) != 0 ? 1u : 0u);
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&accf[ab]);
      }
      // wait for every MMA issued so far before the TMEM is released
      mma_commit(&drain);
      mbar_wait(&drain, 0u, err, kErrFull);
    }
  } else {
    // -------------------------------------------------------------- epilogue
    const int q = warp & 3;           // TMEM lane quarter of this warp
    const int m = q * 32 + lane;      // tile row = column within the tile
    const int et = m;                 // epilogue thread index 0..127
    double rbl[NB], ctl[NB], wml[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) { rbl[b] = 0.0; ctl[b] = 0.0; wml[b] = 0.0; }
    for (int lt = 0; lt < ntl; ++lt) {
      const int ab = lt & 1;
      const uint32_t aph = (uint32_t)(lt >> 1) & 1u;
      if (!mbar_wait(&accf[ab], aph, err, kErrAccFull)) break;
      tc_fence_after();
      uint32_t r[N];
#pragma unroll
      for (int c = 0; c < N / 16; ++c)
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * N + 16 * c), r + 16 * c);
      tmem_wait_ld();
      tc_fence_before();
      mbar_arrive(&acce[ab]);
      const int tile = blockIdx.x + lt * gridDim.x;
      const int64_t sidx = (int64_t)tile * 128 + m;
      if (sidx >= X.p) continue;
      const int64_t j = 1 + X.c + sidx;
      const double aj = __ldg(X.a + j), bj = __ldg(X.b + j);
      const double om = __ldg(F.omega + j);
      const int g = block_of_tc(F.block_ptr, F.G, j);
      const double eta = __ldg(F.eta + g), ie = __ldg(F.inv_eta + g);
      bool act = false;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        // exact recombination of the digit sums: value = 2^9 * accumulator
        long long V = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const float f = __uint_as_float(r[b * D + d]) * 512.0f;
          V = V * 16 + (long long)__float2int_rn(f);
        }
        const double dot = (double)V * (sScale[b] * ldexp(1.0, -4 * D));
        const double s = aj * dot + bj * sS[b];
        const double lamj = F.lam[b] * om;
        const double bo = bcur[j * NB + b];
        if (!sIdle[b]) {
          rbl[b] = fmax(rbl[b], dist_l1_tc(s, lamj, bo));
          const double av = eta * bo + s;
          const double bn = (fmax(av - lamj, 0.0) - fmax(-av - lamj, 0.0)) * ie;
          bnxt[j * NB + b] = bn;
          ctl[b] = fma(bj, bn, ctl[b]);
          act = act || (bn != 0.0);
          wml[b] = fmax(wml[b], fabs(aj * bn));
        }
      }
      if (act) flags[lt * 128 + m] = 1;
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      red_rb[et][b] = rbl[b];
      red_ct[et][b] = ctl[b];
      red_wm[et][b] = wml[b];
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, Sh::TMEM_COLS);
  }
  // per-CTA reductions in a fixed order
  if (threadIdx.x < NB) {
    const int b = threadIdx.x;
    double mx = 0.0, c = 0.0, wm = 0.0;
    for (int t = 0; t < 128; ++t) {
      mx = fmax(mx, red_rb[t][b]);
      c += red_ct[t][b];
      wm = fmax(wm, red_wm[t][b]);
    }
    F.a_rb[blockIdx.x * NB + b] = mx;
    F.a_ct[blockIdx.x * NB + b] = c;
    F.a_wmax[blockIdx.x * NB + b] = wm;
  }
  // ordered compaction of the active flags (local tile order)
  const int per = (T + Sh::THREADS - 1) / Sh::THREADS;
  const int t0 = min(T, (int)threadIdx.x * per), t1 = min(T, t0 + per);
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
  if (threadIdx.x == Sh::THREADS - 1) F.a_cnt[blockIdx.x] = scan[Sh::THREADS - 1];
}

// Dense columns 0..c (intercept and covariates) of the tensor-core column
// pass, in FP64, owning partial slot gridA - 1. One warp per column.
template <int NB>
__global__ void __launch_bounds__(256) k_col_dense(Dsg X, Fits F, int off, int slot) {
  __shared__ double red_rb[8][NB], red_ct[8][NB];
  __shared__ int sflag[64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = *F.it_base + off;
  const double *bcur = F.beta[k & 1];
  double *bnxt = F.beta[(k & 1) ^ 1];
  double S[NB];
  bool idle[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const double *cp = F.c_part[k & 1];
    double Ssum = 0.0;
    for (int c = 0; c < F.gridC; ++c) Ssum += cp[(c * NB + b) * kCPartials + 2];
    S[b] = Ssum;
    idle[b] = (b >= F.nb) || (F.done[b] >= 0);
  }
  for (int t = threadIdx.x; t < 64; t += blockDim.x) sflag[t] = 0;
  double rbl[NB], ctl[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) { rbl[b] = 0.0; ctl[b] = 0.0; }
  __syncthreads();
  for (int64_t j = warp; j <= X.c; j += 8) {
    double dot[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) dot[b] = 0.0;
    if (j >= 1) {
      const double *cv = X.cov + (j - 1) * X.n;
      for (int64_t i = lane; i < X.n; i += 32) {
        const double x = __ldg(cv + i);
#pragma unroll
        for (int b = 0; b < NB; ++b) dot[b] = fma(x, F.theta[i * NB + b], dot[b]);
      }
#pragma unroll
      for (int b = 0; b < NB; ++b)
        for (int o = 16; o; o >>= 1) dot[b] += __shfl_xor_sync(0xffffffffu, dot[b], o);
    }
    if (lane == 0) {
      const double aj = X.a[j], bj = X.b[j];
      const int g = block_of_tc(F.block_ptr, F.G, j);
      const double eta = F.eta[g], ie = F.inv_eta[g];
      bool act = false;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        if (idle[b]) continue;
        const double s = aj * dot[b] + bj * S[b];
        const double lamj = F.lam[b] * F.omega[j];
        const double bo = bcur[j * NB + b];
        if (j >= 1) rbl[b] = fmax(rbl[b], dist_l1_tc(s, lamj, bo));
        const double av = eta * bo + s;
        const double bn = (fmax(av - lamj, 0.0) - fmax(-av - lamj, 0.0)) * ie;
        bnxt[j * NB + b] = bn;
        ctl[b] = fma(bj, bn, ctl[b]);
        act = act || (bn != 0.0 && j >= 1);
      }
      if (act) sflag[j] = 1;
    }
  }
  if (lane == 0)
#pragma unroll
    for (int b = 0; b < NB; ++b) { red_rb[warp][b] = rbl[b]; red_ct[warp][b] = ctl[b]; }
  __syncthreads();
  if (threadIdx.x < NB) {
    const int b = threadIdx.x;
    double mx = 0.0, c = 0.0;
    for (int w = 0; w < 8; ++w) { mx = fmax(mx, red_rb[w][b]); c += red_ct[w][b]; }
    F.a_rb[slot * NB + b] = mx;
    F.a_ct[slot * NB + b] = c;
    F.a_wmax[slot * NB + b] = 0.0;
  }
  if (threadIdx.x == 0) {
    int cnt = 0;
    int *lst = F.a_list + (int64_t)slot * F.T;
    for (int j = 1; j <= X.c; ++j)
      if (sflag[j]) lst[cnt++] = j;
    F.a_cnt[slot] = cnt;
  }
}

// theta^k_b / scale_b rounded to a 4D-bit fixed-point integer, written as D
// balanced base-16 digits encoded as E4M3 bytes, row b*D + d of an N x npad
// byte matrix (rows >= NB*D stay zero).
__constant__ uint8_t kE4M3Int[17] = {0xD0, 0xCE, 0xCC, 0xCA, 0xC8, 0xC4, 0xC0, 0xB8, 0x00,
                                     0x38, 0x40, 0x44, 0x48, 0x4A, 0x4C, 0x4E, 0x50};

template <int NB, int D>
__global__ void __launch_bounds__(256) k_quantize_tc(Fits F, int off, uint8_t *dg) {
  const int k = *F.it_base + off;
  __shared__ double sInv[kMaxNB];
  if (threadIdx.x < NB) {
    const int b = threadIdx.x;
    const double *cp = F.c_part[k & 1];
    double m = 0.0;
    for (int c = 0; c < F.gridC; ++c) m = fmax(m, cp[(c * NB + b) * kCPartials + 3]);
    int E = 0;
    if (m > 0.0) frexp(m, &E);
    const double scale = (m > 0.0) ? ldexp(1.0, E + 1) : 1.0;
    sInv[b] = ldexp(1.0, 4 * D) / scale;
    if (blockIdx.x == 0) F.scale[b] = scale;
  }
  __syncthreads();
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = (int)(g / F.npad);
  const int64_t i = g - (int64_t)b * F.npad;
  if (b >= NB) return;
  long long Xq = __double2ll_rn(F.theta[i * NB + b] * sInv[b]);
  int dig[D];
#pragma unroll
  for (int d = D - 1; d >= 1; --d) {
    const int t = (int)(((Xq + 8) & 15) - 8);
    dig[d] = t;
    Xq = (Xq - t) >> 4;
  }
  dig[0] = (int)Xq;
#pragma unroll
  for (int d = 0; d < D; ++d) dg[(int64_t)(b * D + d) * F.npad + i] = kE4M3Int[dig[d] + 8];
}

// ------------------------------------------------------------------ host

template <int NB, int D>
size_t g_tc_opted = 48 * 1024;

size_t col_tc_smem(int NB, int D, int T) {
  int N = NB * D <= 16 ? 16 : (NB * D <= 32 ? 32 : 64);
  return (size_t)6 * (128 * 128 + N * 128) + 1024 + (size_t)T + 16;
}

template <int NB, int D>
static cudaError_t col_tc_t(const Dsg &X, const Fits &F, int off, const CUtensorMap &tmX,
                            const CUtensorMap &tmD, int grid, int tiles_per_cta, int *err,
                            cudaStream_t s) {
  const size_t smem = col_tc_smem(NB, D, F.T);
  if (smem > g_tc_opted<NB, D>) {
    cudaError_t e = cudaFuncSetAttribute(k_col_tc<NB, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    g_tc_opted<NB, D> = smem;
  }
  k_col_tc<NB, D><<<grid, TcShape<NB, D>::THREADS, smem, s>>>(X, F, off, tmX, tmD, tiles_per_cta, err);
  return cudaGetLastError();
}

cudaError_t launch_col_tc(int NB, int D, const Dsg &X, const Fits &F, int off, const CUtensorMap &tmX,
                          const CUtensorMap &tmD, int grid, int tiles_per_cta, int *err,
                          cudaStream_t s) {
#define FSQR_TC_CASE(nb, d) \
  if (NB == nb && D == d) return col_tc_t<nb, d>(X, F, off, tmX, tmD, grid, tiles_per_cta, err, s);
  FSQR_TC_CASE(1, 7) FSQR_TC_CASE(2, 7) FSQR_TC_CASE(3, 7) FSQR_TC_CASE(4, 7)
  FSQR_TC_CASE(1, 6) FSQR_TC_CASE(2, 6) FSQR_TC_CASE(3, 6) FSQR_TC_CASE(4, 6)
#undef FSQR_TC_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_col_dense(int NB, const Dsg &X, const Fits &F, int off, int slot, cudaStream_t s) {
  switch (NB) {
    case 1: k_col_dense<1><<<1, 256, 0, s>>>(X, F, off, slot); break;
    case 2: k_col_dense<2><<<1, 256, 0, s>>>(X, F, off, slot); break;
    case 3: k_col_dense<3><<<1, 256, 0, s>>>(X, F, off, slot); break;
    case 4: k_col_dense<4><<<1, 256, 0, s>>>(X, F, off, slot); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_quantize_tc(int NB, int D, const Fits &F, int off, uint8_t *dg, cudaStream_t s) {
  const int64_t total = (int64_t)NB * F.npad;
  const unsigned grid = (unsigned)((total + 255) / 256);
#define FSQR_Q_CASE(nb, d) \
  if (NB == nb && D == d) { k_quantize_tc<nb, d><<<grid, 256, 0, s>>>(F, off, dg); return cudaGetLastError(); }
  FSQR_Q_CASE(1, 7) FSQR_Q_CASE(2, 7) FSQR_Q_CASE(3, 7) FSQR_Q_CASE(4, 7)
  FSQR_Q_CASE(1, 6) FSQR_Q_CASE(2, 6) FSQR_Q_CASE(3, 6) FSQR_Q_CASE(4, 6)
#undef FSQR_Q_CASE
  return cudaErrorInvalidValue;
}

int tc_rows(int NB, int D) { return NB * D <= 16 ? 16 : (NB * D <= 32 ? 32 : 64); }

}  // namespace fsqr
