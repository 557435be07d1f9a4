// Tensor-core column pass of the FS-QRPPA iteration (mixed arithmetic).
//
// s_j = x~_j^T theta^k over the stored genotype columns is computed as an
// exact integer product on the 5th-generation tensor cores:
//   * theta_b is rounded to a 4D-bit fixed-point integer and split into D
//     balanced base-16 digits t in [-8, 8]; every digit is an exact E4M3
//     value. The digits of the NB fits form an N x n matrix (rows b*D + d).
//   * The int8 genotype codes 0/1/2 read as E4M3 bit patterns are the
//     subnormals 0, 2^-9, 2^-8, i.e. exactly g * 2^-9, so the codes are
//     multiplied with no conversion. Before the iteration the stored matrix
//     is copied once into tiles of 128 columns x 128 samples laid out as
//     the byte image of the swizzled shared-memory operand (k_tile_x), so
//     every stage is one contiguous 16 KB bulk copy.
//   * tcgen05.mma kind::f8f6f4 (M = 128 columns, N = digit rows, K = 32
//     samples) accumulates g * t * 2^-9 in FP32 in tensor memory; every
//     partial sum is an integer multiple of 2^-9 below 2^24 * 2^-9, hence
//     exact. The epilogue recombines the digits exactly in int64.
// The FP64 proximal update (eq. beta_update), the stop-test distance and the
// active-column lists follow as in the SIMT column pass.
//
// Roles (256 threads): warp 0 issues TMA loads into a STAGES-deep ring,
// warp 1 issues the MMAs (one elected thread) into ACC TMEM accumulators,
// warps 2-5 (128 threads, one per tile row) run the epilogue, warps 6-7
// handle the FP64 dense columns (intercept, covariates) j = blockIdx.x,
// blockIdx.x + grid, ... <= c.
// Schedule: with R = floor(tiles / grid), CTA c takes the 128-column tiles
// c, c + grid, ..., c + (R-1) grid whole. The rem = tiles - R grid tiles
// left over either go whole to CTAs 0..rem-1 (ns = 0), or, when R is small
// and a partial last round would cost a large share of the pass, are cut
// along the samples into ns slices each (ns ~ grid / rem): CTA c < rem * ns
// computes slice c % ns of tail tile c / ns and stores its exact integer
// digit sums; the last slice CTA of a tile to finish adds them up and runs
// that tile's epilogue. List slot c holds CTA c's whole tiles in tile order,
// then its dense columns; slot grid + u holds sliced tail tile u.
#include <cuda.h>
#include <math.h>
#include <stdint.h>

#include "fsqr_device.cuh"
#include "fsqr_internal.h"
#include "sm103_ops.cuh"

namespace fsqr {

using namespace sm103;

// E4M3 encodings of the integers -8..8 (index t + 8).
__constant__ uint8_t kE4M3Int[17] = {0xD0, 0xCE, 0xCC, 0xCA, 0xC8, 0xC4, 0xC0, 0xB8, 0x00,
                                     0x38, 0x40, 0x44, 0x48, 0x4A, 0x4C, 0x4E, 0x50};

template <int NB, int D, int F2 = 0>
struct TcShape {
  static constexpr int NR = NB * D;
  static constexpr int N = NR <= 16 ? 16 : (NR <= 32 ? 32 : 64);
  static constexpr int ACC = 4;  // TMEM accumulator buffers
  static constexpr int TMEM_COLS = (ACC * N <= 32) ? 32 : ((ACC * N <= 64) ? 64 : ((ACC * N <= 128) ? 128 : 256));
  static constexpr int STAGES = 6;
  static constexpr int A_BYTES = 128 * 128;
  static constexpr int B_BYTES = N * 128;
  // 2-bit storage (F2): the stage also holds the 4 KB packed tile that the
  // decode warps expand into the A operand
  static constexpr int RAW_BYTES = F2 ? 128 * 32 : 0;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES + RAW_BYTES;
  static constexpr int THREADS = F2 ? 384 : 256;
};

// Four 2-bit genotype codes (one byte, sample 4q + f in bits 2f) -> four
// bytes holding the codes 0/1/2, which read as E4M3 are exactly g * 2^-9;
// the missing code 3 becomes 0 (mean imputation is applied by the
// correction terms).
__device__ __forceinline__ uint32_t spread_codes(uint32_t b) {
  uint32_t v = (b & 3u) | ((b & 0xCu) << 6) | ((b & 0x30u) << 12) | ((b & 0xC0u) << 18);
  const uint32_t m = v & (v >> 1) & 0x01010101u;
  return v & ~(m * 3u);
}

// As spread_codes for codes already in 0..2 (the sanitised 2-bit tiles): byte
// k of w (codes 4k .. 4k+3) goes to one output word in two shift-and-mask steps.
__device__ __forceinline__ uint32_t spread_clean(uint32_t w, int k) {
  uint32_t x = __byte_perm(w, 0u, 0x4440u | (uint32_t)k);  // byte k, zero-extended
  x = (x | (x << 12)) & 0x000F000Fu;
  return (x | (x << 6)) & 0x03030303u;
}

__device__ __forceinline__ uint4 spread_word_clean(uint32_t w) {
  return make_uint4(spread_clean(w, 0), spread_clean(w, 1), spread_clean(w, 2), spread_clean(w, 3));
}

__device__ __forceinline__ uint4 spread_word(uint32_t w) {
  return make_uint4(spread_codes(w & 0xffu), spread_codes((w >> 8) & 0xffu), spread_codes((w >> 16) & 0xffu),
                    spread_codes(w >> 24));
}

// At most this many sample slices per tail tile.
constexpr int kMaxTailSlices = 16;

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

// Proximal update of stored column j for every fit from V[b], the exact
// integer value of x_j^T theta^_b in units of scale_b * 2^(-4D) (eq.
// beta_update with M_g = eta_g I); accumulates the stop-test distance, the
// constant term and max |a_j beta_j|, and tells whether the column is active.
template <int NB, int D>
__device__ __forceinline__ bool col_update(const Dsg &X, const Fits &F, int64_t j, const long long (&V)[NB],
                                           const double *sS, const double *sScale, const int *sIdle,
                                           const double *bcur, double *bnxt, double (&rbl)[NB],
                                           double (&ctl)[NB], double (&wml)[NB], double aj, double bj,
                                           double om, const double (&bo)[NB], double eta, double ie) {
  // ie is 1/eta_g, or 1/(eta_g + gamma_j) with the elastic-net term
  const double dscale = ldexp(1.0, -4 * D);
  const double gj = F.ridge * om;  // elastic-net quadratic weight (0: weighted l1)
  if (gj != 0.0) ie = 1.0 / (eta + gj);
  bool act = false;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const double dot = (double)V[b] * (sScale[b] * dscale);
    // mean imputation: missing entries read as 0, so their b_j theta_i is taken back out
    const double mc = X.mptr ? miss_dot(X, j - 1 - X.c, F.theta, NB, b) : 0.0;
    const double s = aj * dot + bj * (sS[b] - mc);
    const double lamj = F.lam[b] * om;
    if (!sIdle[b]) {
      rbl[b] = fmax(rbl[b], dist_l1_tc(gj == 0.0 ? s : s - gj * bo[b], lamj, bo[b]));
      const double av = eta * bo[b] + s;
      const double bn = (fmax(av - lamj, 0.0) - fmax(-av - lamj, 0.0)) * ie;
      bnxt[j * NB + b] = bn;
      ctl[b] = fma(bj, bn, ctl[b]);
      act = act || (bn != 0.0);
      wml[b] = fmax(wml[b], fabs(aj * bn));
    }
  }
  return act;
}

// F2 = 1: 2-bit storage. xt then holds tiles of 128 columns x 128 samples
// of packed codes (32 bytes per column, 4 KB per tile, missing codes already
// 0), the producer bulk-copies them into the stage's raw area, and warps
// 8-11 (one thread per tile row) expand them into the E4M3 A operand before
// releasing the stage to the MMA issuer.
template <int NB, int D, int F2>
__global__ void __launch_bounds__(F2 ? 384 : 256, 1)
    k_col_tc(Dsg X, Fits F, int off, const uint8_t *__restrict__ xt, const uint8_t *__restrict__ dgt,
             int rounds, int slices, int32_t *__restrict__ tail_part, unsigned *__restrict__ tail_tick,
             int *err) {
  using Sh = TcShape<NB, D, F2>;
  constexpr int N = Sh::N;
  constexpr int S = Sh::STAGES;
  constexpr int kAcc = Sh::ACC;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[S], empty[S], dec[S], accf[kAcc], acce[kAcc], drain;
  __shared__ uint32_t tmem_base;
  __shared__ double sS[kMaxNB], sScale[kMaxNB];
  __shared__ int sIdle[kMaxNB];
  __shared__ double red[3][256];
  __shared__ int scan[Sh::THREADS];
  __shared__ int s_dense_act[64];
  __shared__ int s_ndense;

  // 1024-aligned ring of stages, then the active flags of this CTA's columns
  const uint32_t base_u32 = smem_u32(smem_raw);
  uint8_t *ring = smem_raw + (((base_u32 + 1023u) & ~1023u) - base_u32);
  uint8_t *flags = ring + S * Sh::STAGE_BYTES;
  const int T = F.T;                       // list stride: 128 * (rounds + 1) + 64
  const int TF = 128 * (rounds + 1);       // flags of the whole-tile columns

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = *F.it_base + off;
  const double *bcur = F.beta[k & 1];
  double *bnxt = F.beta[(k & 1) ^ 1];
  const int64_t ntiles = (X.p + 127) / 128;
  const int ns = slices;
  const int rem = (int)(ntiles - (int64_t)rounds * gridDim.x);
  const bool tail = ns > 0 && rem > 0 && (int)blockIdx.x < rem * ns;
  // whole tiles of this CTA (the leftover one included when not sliced)
  const int R = rounds + ((ns == 0 && (int)blockIdx.x < rem) ? 1 : 0);
  const int tu = tail ? (int)blockIdx.x / ns : 0, tv = tail ? (int)blockIdx.x % ns : 0;
  const int ntl = R + (tail ? 1 : 0);      // local tile lt = R is the tail slice
  const int nk = (int)((X.n + 127) / 128);
  const int tail_k0 = ns ? nk * tv / ns : 0, tail_k1 = ns ? nk * (tv + 1) / ns : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); mbar_init(&dec[s], 128); }
    for (int a = 0; a < kAcc; ++a) { mbar_init(&accf[a], 1); mbar_init(&acce[a], 128); }
    mbar_init(&drain, 1);
    fence_mbar_init();
  }
  if (threadIdx.x < NB) {
    const int b = threadIdx.x;
    sS[b] = F.tot_c[k & 1][b * kCPartials + 2];
    sIdle[b] = (b >= F.nb) || (F.done[b] >= 0);
    sScale[b] = F.scale[b];
  }
  if (threadIdx.x == 0) s_ndense = 0;
  for (int t = threadIdx.x; t < TF; t += Sh::THREADS) flags[t] = 0;
  if (warp == 1) tmem_alloc(&tmem_base, Sh::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  // per-thread partials (max dist, constant term, max |a_j beta_j|)
  double rbl[NB], ctl[NB], wml[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) { rbl[b] = 0.0; ctl[b] = 0.0; wml[b] = 0.0; }

  if (warp == 0) {
    // ---------------------------------------------------------- TMA producer
    if (lane == 0) {
      int it = 0;
      for (int lt = 0; lt < ntl; ++lt) {
        const int tile = lt < R ? (int)blockIdx.x + lt * (int)gridDim.x : rounds * (int)gridDim.x + tu;
        const int k0 = lt < R ? 0 : tail_k0, k1 = lt < R ? nk : tail_k1;
        for (int kc = k0; kc < k1; ++kc, ++it) {
          const int s = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, err, kErrEmpty)) goto producer_done;
          uint8_t *sa = ring + s * Sh::STAGE_BYTES;
          if (F2) {
            mbar_arrive_expect_tx(&full[s], Sh::RAW_BYTES + Sh::B_BYTES);
            bulk_load(sa + Sh::A_BYTES + Sh::B_BYTES, xt + ((int64_t)tile * nk + kc) * Sh::RAW_BYTES,
                      Sh::RAW_BYTES, &full[s]);
          } else {
            mbar_arrive_expect_tx(&full[s], Sh::A_BYTES + Sh::B_BYTES);
            bulk_load(sa, xt + ((int64_t)tile * nk + kc) * Sh::A_BYTES, Sh::A_BYTES, &full[s]);
          }
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
      for (int lt = 0; lt < ntl; ++lt) {
        const int ab = lt % kAcc;
        const uint32_t aph = (uint32_t)(lt / kAcc) & 1u;
        if (!mbar_wait(&acce[ab], aph ^ 1u, err, kErrAccEmpty)) break;
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(ab * N);
        const int k0 = lt < R ? 0 : tail_k0, k1 = lt < R ? nk : tail_k1;
        bool ok = true;
        for (int kc = k0; kc < k1; ++kc, ++it) {
          const int s = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          // F2: the decode warps' arrival implies the bulk copies landed
          if (!mbar_wait(F2 ? &dec[s] : &full[s], ph, err, kErrFull)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(ring + s * Sh::STAGE_BYTES);
          const uint64_t ad = sdesc_k128(sa), bd = sdesc_k128(sa + Sh::A_BYTES);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma_f8(dt, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc, (kc != k0 || kk != 0) ? 1u : 0u);
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&accf[ab]);
      }
      // wait for every MMA issued so far before the TMEM is released
      mma_commit(&drain);
      mbar_wait(&drain, 0u, err, kErrFull);
    }
  } else if (warp >= 8) {
    // ------------------------------------------- 2-bit decode (F2 only)
    // thread m expands row m (tile column m): its 32 packed bytes (128
    // samples) become 8 swizzled 16-byte chunks of the K-major operand
    const int m = threadIdx.x - 256;
    int it = 0;
    for (int lt = 0; lt < ntl; ++lt) {
      const int k0 = lt < R ? 0 : tail_k0, k1 = lt < R ? nk : tail_k1;
      bool ok = true;
      for (int kc = k0; kc < k1; ++kc, ++it) {
        const int s = it % S;
        const uint32_t ph = (uint32_t)(it / S) & 1u;
        if (!mbar_wait(&full[s], ph, err, kErrFull)) { ok = false; break; }
        uint8_t *sa = ring + s * Sh::STAGE_BYTES;
        const uint4 *raw = reinterpret_cast<const uint4 *>(sa + Sh::A_BYTES + Sh::B_BYTES + m * 32);
        const uint4 r0 = raw[0], r1 = raw[1];
        const uint32_t wv[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
#pragma unroll
        for (int c = 0; c < 8; ++c)
          *reinterpret_cast<uint4 *>(sa + m * 128 + ((c ^ (m & 7)) << 4)) = spread_word_clean(wv[c]);
        fence_proxy_async();
        mbar_arrive(&dec[s]);
      }
      if (!ok) break;
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
      // reduce over the 64 dense threads (two warps) through shared memory
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        for (int o = 16; o; o >>= 1) dot[b] += __shfl_xor_sync(0xffffffffu, dot[b], o);
      }
      __shared__ double s_dot[2][NB];
      if (lane == 0)
#pragma unroll
        for (int b = 0; b < NB; ++b) s_dot[warp - 6][b] = dot[b];
      asm volatile("bar.sync 1, 64;" ::: "memory");
      if (dl == 0) {
        const double aj = X.a[j], bj = X.b[j];
        const int g = block_of_tc(F.block_ptr, F.G, j);
        const double gj = F.ridge * F.omega[j];
        const double eta = F.eta[g], ie = gj == 0.0 ? F.inv_eta[g] : 1.0 / (F.eta[g] + gj);
        bool act = false;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          if (sIdle[b]) continue;
          const double s = aj * (s_dot[0][b] + s_dot[1][b]) + bj * sS[b];
          const double lamj = F.lam[b] * F.omega[j];
          const double bo = bcur[j * NB + b];
          if (j >= 1) rbl[b] = fmax(rbl[b], dist_l1_tc(gj == 0.0 ? s : s - gj * bo, lamj, bo));
          const double av = eta * bo + s;
          const double bn = (fmax(av - lamj, 0.0) - fmax(-av - lamj, 0.0)) * ie;
          bnxt[j * NB + b] = bn;
          ctl[b] = fma(bj, bn, ctl[b]);
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
    for (int lt = 0; lt < ntl; ++lt) {
      const int ab = lt % kAcc;
      const uint32_t aph = (uint32_t)(lt / kAcc) & 1u;
      if (lt >= R) {
        // tail slice: store the exact digit sums (accumulator * 2^9) of row m
        if (!mbar_wait(&accf[ab], aph, err, kErrAccFull)) break;
        tc_fence_after();
        uint32_t r[N];
#pragma unroll
        for (int c = 0; c < N / 16; ++c)
          tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * N + 16 * c), r + 16 * c);
        tmem_wait_ld();
        tc_fence_before();
        mbar_arrive(&acce[ab]);
        int32_t *dst = tail_part + (int64_t)(tu * ns + tv) * Sh::NR * 128 + m;
#pragma unroll
        for (int d = 0; d < Sh::NR; ++d) dst[d * 128] = __float2int_rn(__uint_as_float(r[d]) * 512.0f);
        continue;
      }
      // operands of this thread's column, fetched while the MMAs run
      const int tile = blockIdx.x + lt * gridDim.x;
      const int64_t sidx = (int64_t)tile * 128 + m;
      const bool live = sidx < X.p;
      const int64_t j = 1 + X.c + (live ? sidx : 0);
      const double aj = __ldg(X.a + j), bj = __ldg(X.b + j);
      const double om = __ldg(F.omega + j);
      double bo[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) bo[b] = bcur[j * NB + b];
      const int g = block_of_tc(F.block_ptr, F.G, j);
      const double eta = __ldg(F.eta + g), ie = __ldg(F.inv_eta + g);
      if (!mbar_wait(&accf[ab], aph, err, kErrAccFull)) break;
      tc_fence_after();
      uint32_t r[N];
#pragma unroll
      for (int c = 0; c < N / 16; ++c)
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * N + 16 * c), r + 16 * c);
      tmem_wait_ld();
      tc_fence_before();
      mbar_arrive(&acce[ab]);
      if (!live) continue;
      // exact recombination of the digit sums: value = 2^9 * accumulator
      long long V[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        V[b] = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const float f = __uint_as_float(r[b * D + d]) * 512.0f;
          V[b] = V[b] * 16 + (long long)__float2int_rn(f);
        }
      }
      if (col_update<NB, D>(X, F, j, V, sS, sScale, sIdle, bcur, bnxt, rbl, ctl, wml, aj, bj, om, bo, eta, ie))
        flags[lt * 128 + m] = 1;
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, Sh::TMEM_COLS);
  }
  // per-CTA reductions in a fixed order
  for (int b = 0; b < NB; ++b) {
    if (threadIdx.x < 256) {  // the decode warps (F2) hold no partials
      red[0][threadIdx.x] = rbl[b];
      red[1][threadIdx.x] = ctl[b];
      red[2][threadIdx.x] = wml[b];
    }
    __syncthreads();
    const int ops[3] = {0, 1, 0};
    tree_reduce<3>(red, ops, 256);
    if (threadIdx.x == 0) {
      F.a_rb[blockIdx.x * NB + b] = red[0][0];
      F.a_ct[blockIdx.x * NB + b] = red[1][0];
      F.a_wmax[blockIdx.x * NB + b] = red[2][0];
    }
    __syncthreads();
  }
  // ordered compaction of the active flags (local tile order)
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
  if (tail) {
    // the last slice CTA of tail tile tu to finish runs its epilogue into
    // list slot grid + tu (one thread per column)
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(tail_tick + tu, 1u) == (unsigned)(ns - 1)) ? 1 : 0;
    __syncthreads();
    if (s_last) {
      __threadfence();
      const int slot = (int)gridDim.x + tu;
      const int m = threadIdx.x;
      const int64_t sidx = (int64_t)(rounds * (int)gridDim.x + tu) * 128 + m;
      const bool live = m < 128 && sidx < X.p;
      // sums over the slices of the digit sums, 4 columns per int4, every
      // slice's load in flight at once, into the (idle) stage ring
      int32_t *tsum = reinterpret_cast<int32_t *>(ring);
      for (int q = threadIdx.x; q < Sh::NR * 32; q += Sh::THREADS) {
        int4 v4[kMaxTailSlices];
#pragma unroll
        for (int v = 0; v < kMaxTailSlices; ++v)
          if (v < ns)
            v4[v] = __ldcg(reinterpret_cast<const int4 *>(tail_part + (int64_t)(tu * ns + v) * Sh::NR * 128) + q);
        int4 a = make_int4(0, 0, 0, 0);
#pragma unroll
        for (int v = 0; v < kMaxTailSlices; ++v)
          if (v < ns) { a.x += v4[v].x; a.y += v4[v].y; a.z += v4[v].z; a.w += v4[v].w; }
        reinterpret_cast<int4 *>(tsum)[q] = a;
      }
      __syncthreads();
      double rb2[NB], ct2[NB], wm2[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) { rb2[b] = 0.0; ct2[b] = 0.0; wm2[b] = 0.0; }
      bool act = false;
      int64_t j = 0;
      if (live) {
        j = 1 + X.c + sidx;
        long long V[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          V[b] = 0;
#pragma unroll
          for (int d = 0; d < D; ++d) V[b] = V[b] * 16 + (long long)tsum[(b * D + d) * 128 + m];
        }
        const double aj = __ldg(X.a + j), bj = __ldg(X.b + j), om = __ldg(F.omega + j);
        double bo[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) bo[b] = bcur[j * NB + b];
        const int g = block_of_tc(F.block_ptr, F.G, j);
        const double eta = __ldg(F.eta + g), ie = __ldg(F.inv_eta + g);
        act = col_update<NB, D>(X, F, j, V, sS, sScale, sIdle, bcur, bnxt, rb2, ct2, wm2, aj, bj, om, bo, eta,
                                ie);
      }
      for (int b = 0; b < NB; ++b) {
        if (threadIdx.x < 256) {
          red[0][threadIdx.x] = rb2[b];
          red[1][threadIdx.x] = ct2[b];
          red[2][threadIdx.x] = wm2[b];
        }
        __syncthreads();
        const int ops[3] = {0, 1, 0};
        tree_reduce<3>(red, ops, 256);
        if (threadIdx.x == 0) {
          F.a_rb[slot * NB + b] = red[0][0];
          F.a_ct[slot * NB + b] = red[1][0];
          F.a_wmax[slot * NB + b] = red[2][0];
        }
        __syncthreads();
      }
      // ordered compaction of the tile's active columns
      scan[threadIdx.x] = act ? 1 : 0;
      __syncthreads();
      for (int o = 1; o < Sh::THREADS; o <<= 1) {
        int v = (threadIdx.x >= (unsigned)o) ? scan[threadIdx.x - o] : 0;
        __syncthreads();
        scan[threadIdx.x] += v;
        __syncthreads();
      }
      if (act) F.a_list[(int64_t)slot * T + scan[threadIdx.x] - 1] = (int)j;
      if (threadIdx.x == Sh::THREADS - 1) {
        F.a_cnt[slot] = scan[Sh::THREADS - 1];
        tail_tick[tu] = 0u;
      }
    }
  }
  col_finalize<NB>(F);
}

// theta^k_b / scale_b rounded to a 4D-bit fixed-point integer, written as D
// balanced base-16 digits encoded as E4M3 bytes, row b*D + d of an N x npad
// byte matrix (rows >= NB*D stay zero).

template <int NB, int D>
__global__ void __launch_bounds__(256) k_quantize_tc(Fits F, int off, uint8_t *dg) {
  const int k = *F.it_base + off;
  __shared__ double sInv[kMaxNB];
  if (threadIdx.x < NB) {
    const int b = threadIdx.x;
    const double m = F.tot_c[k & 1][b * kCPartials + 3];
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
  long long Xq = fixed_point(F.theta[i * NB + b] * sInv[b]);
  int dig[D];
#pragma unroll
  for (int d = D - 1; d >= 1; --d) {
    const int t = (int)(((Xq + 8) & 15) - 8);
    dig[d] = t;
    Xq = (Xq - t) >> 4;
  }
  dig[0] = (int)Xq;
  // K-chunk kc = i / 128 holds N rows of 128 bytes; row r's 16-byte chunk c
  // sits at chunk position c ^ (r % 8) (the 128-byte swizzle)
  constexpr int N = TcShape<NB, D>::N;
  const int64_t kc = i >> 7;
  const int c = (int)((i & 127) >> 4), bt = (int)(i & 15);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int r = b * D + d;
    dg[kc * (N * 128) + r * 128 + ((c ^ (r & 7)) << 4) + bt] = kE4M3Int[dig[d] + 8];
  }
}

// Copies the stored int8 columns into tiles of 128 columns x 128 samples,
// each the byte image of a 128-byte-swizzled K-major operand: tile (t, kc)
// at xt + (t*nk + kc)*16384, row m = column 128t + m, 16-byte chunk c of the
// row at chunk position c ^ (m % 8); samples >= n and columns >= p are 0.
__global__ void k_tile_x(Dsg X, uint8_t *xt, int64_t nk) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // one 16-byte chunk
  const int64_t ntile = (X.p + 127) / 128;
  if (g >= ntile * nk * 1024) return;
  const int64_t tk = g >> 10;          // tile * nk + kc
  const int w = (int)(g & 1023);       // chunk within the 16 KB tile
  const int m = w >> 3, cp = w & 7;    // row, stored chunk position
  const int c = cp ^ (m & 7);          // logical chunk
  const int64_t t = tk / nk, kc = tk - t * nk;
  const int64_t col = t * 128 + m;
  const int64_t s0 = kc * 128 + c * 16;
  uint4 v = make_uint4(0u, 0u, 0u, 0u);
  if (col < X.p && s0 < X.n) {
    const uint8_t *src = X.geno + col * X.ld + s0;
    if (s0 + 16 <= X.n) {
      v = *reinterpret_cast<const uint4 *>(src);
    } else {
      uint8_t b[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) b[q] = (s0 + q < X.n) ? src[q] : (uint8_t)0;
      v = *reinterpret_cast<const uint4 *>(b);
    }
  }
  *reinterpret_cast<uint4 *>(xt + tk * 16384 + (int64_t)w * 16) = v;
}

// ============================================================ X~ beta (TC)

// Tensor-core X~ beta over the active stored columns (mixed path):
// q_i = sum_{j active} x_ij w_j with w_jb = a_j beta_jb rounded to a
// 4*DWD-bit fixed-point integer (scale 2^(E_b+1) > 2 max|w_b|) and split
// into DWD balanced base-16 digits (E4M3).
//   k_xprep      one thread per active position: its stored column and
//                the digit bytes, written as the byte image of one K-major
//                swizzled operand tile per block of 128 active positions;
//   k_xbeta_tc   CTA (rt, sp): samples [128 rt, +128) (M, the TMEM lanes)
//                over the blocks of split sp. Its threads copy the 128-byte
//                sample runs of a block's active columns with 16-byte
//                asynchronous copies (kXbLag blocks in flight per thread)
//                into a ring of stages as an MN-major operand, a bulk copy
//                brings the block's digit tile, and
//                kind::f8f6f4 MMAs accumulate exact integer sums in FP32 in
//                TMEM. The epilogue writes one exact int64 partial per
//                (split, sample, fit). (TMA tile::gather4 of the runs, 4
//                columns per copy, ran at about 1.5 TB/s here: the copies,
//                not HBM, set the pace.)
// Blocks a thread keeps in flight (asynchronous copies) in the X~ beta pass.
constexpr int kXbLag = 2;

template <int NB, int DWD>
struct XbShape {
  static constexpr int NR = NB * DWD;
  static constexpr int N = ((NR + 15) / 16) * 16;
  static constexpr int A_BYTES = 128 * 128;
  static constexpr int B_BYTES = N * 128;
  static constexpr int BUF = A_BYTES + B_BYTES;
  static constexpr int STAGES = kXbLag + 2;
  static constexpr int TMEM_COLS = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
};

constexpr int kXTMaxSplits = 16;

// The recombined integer sum_j g_ij W_j (|W_j| < 2^43, g <= 2) stays below
// 2^63 and every FP32 digit sum below 2^24 units while fewer than 2^19
// columns are active; beyond that the pass records an error and adds nothing.
constexpr int kMaxActive = 1 << 19;

template <int NB, int DWD>
__global__ void __launch_bounds__(128)
    k_xprep(Dsg X, Fits F, int off, const double *__restrict__ beta_in, int split_cap, int *__restrict__ scol,
            uint8_t *__restrict__ wtile, int *err) {
  using Sh = XbShape<NB, DWD>;
  extern __shared__ int spre[];  // gridA + 1
  __shared__ double sInv[kMaxNB];
  const double *beta = beta_in;
  if (beta == nullptr) {
    const int k = *F.it_base + off;
    beta = F.beta[(k & 1) ^ 1];
  }
  const int gA = F.gridA;
  int A = __ldcg(F.a_pre + gA);
  if (A >= kMaxActive) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(err, 0, 5);
    A = 0;
  }
  const int nkb = (A + 127) / 128;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // splits of the X~ beta pass: enough CTAs for one resident wave
    F.meta_i[0] = max(1, min(kXTMaxSplits, min(nkb, split_cap)));
    F.meta_i[1] = A;
  }
  if (threadIdx.x < NB) {
    const int b = threadIdx.x;
    const double m = F.tot_a[b * 3 + 2];
    int E = 0;
    if (m > 0.0) frexp(m, &E);
    const double scale = (m > 0.0) ? ldexp(1.0, E + 1) : 1.0;
    sInv[b] = ldexp(1.0, 4 * DWD) / scale;
    if (blockIdx.x == 0) {
      F.meta_d[b] = F.tot_a[b * 3 + 1];
      F.meta_d[kMaxNB + b] = scale;
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
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      long long W = (j >= 0) ? fixed_point(aj * beta[(int64_t)j * NB + b] * sInv[b]) : 0;
      int dig[DWD];
#pragma unroll
      for (int d = DWD - 1; d >= 1; --d) {
        const int tt = (int)(((W + 8) & 15) - 8);
        dig[d] = tt;
        W = (W - tt) >> 4;
      }
      dig[0] = (int)W;
#pragma unroll
      for (int d = 0; d < DWD; ++d) {
        const int r = b * DWD + d;
        tile[r * 128 + ((ch ^ (r & 7)) << 4) + bt] = kE4M3Int[dig[d] + 8];
      }
    }
    // digit rows beyond NB*DWD are zero
    for (int r = NB * DWD; r < Sh::N; ++r) tile[r * 128 + ((ch ^ (r & 7)) << 4) + bt] = 0;
  }
}

// CTA (rt, sp). All 128 threads stream the blocks of split sp: each thread
// copies 8 16-byte sample runs of the block's active columns (column k =
// chunk / 8, samples 16 (chunk % 8) .. +15 of the row tile; bytes of samples
// >= n and absent columns zero-filled) into the stage as the 128-byte-
// swizzled MN-major operand, and releases a block to the MMA issuer once its
// own copies of it have landed; thread 0 adds the block's digit tile by a
// bulk copy and issues the MMAs. With fuse = 1 the last split CTA to finish a row tile sums
// the splits' integer partials of its 128 rows and applies the vector update
// (z, r, theta and the stop-test partials, as k_vec), and the last row tile
// to finish writes the totals.
template <int NB, int DWD>
__global__ void __launch_bounds__(128)
    k_xbeta_tc(Dsg X, Fits F, int off, int fuse, const int *__restrict__ scol, const uint8_t *__restrict__ wtile,
               int *err) {
  using Sh = XbShape<NB, DWD>;
  constexpr int N = Sh::N;
  constexpr int ST = Sh::STAGES;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[ST], empty[ST], dbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_last;
  __shared__ double red[kCPartials][256];
  const uint32_t base_u32 = smem_u32(smem_raw);
  uint8_t *ring = smem_raw + (((base_u32 + 1023u) & ~1023u) - base_u32);
  const int tid = threadIdx.x, warp = tid >> 5;
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
    if (warp == 0) tmem_alloc(&tmem_base, Sh::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = idesc_f32acc_amn(0u, 128u, (uint32_t)N);
    // this thread's sample chunk c and the columns k = 16 e + kr (e < 8)
    const int c = tid & 7, kr = tid >> 3;
    const int64_t s0 = i0 + 16 * c;                 // first sample of the chunk
    const uint32_t valid = s0 < F.n ? (uint32_t)(F.n - s0 < 16 ? F.n - s0 : 16) : 0u;
    const int nb = kb1 - kb0;
    int idxA[8], idxB[8];
    auto load_idx = [&](int blk, int (&idx)[8]) {
#pragma unroll
      for (int e = 0; e < 8; ++e) idx[e] = __ldg(scol + (int64_t)blk * 128 + 16 * e + kr);
    };
    bool ok = true;
    // one step: block `it` (column indices in idx) is copied into its stage;
    // block it - kLag, whose copies this thread has waited for, is released
    // to the MMA issuer, which (thread 0) multiplies it.
    auto step = [&](int it, int (&idx)[8]) {
      if (it < nb) {
        const int s = it % ST;
        if (!mbar_wait(&empty[s], ((uint32_t)(it / ST) & 1u) ^ 1u, err, kErrEmpty)) { ok = false; return; }
        uint8_t *stage = ring + s * Sh::BUF;
        if (X.fmt == FSQR_2BIT) {
          // 16 packed samples = 4 bytes per column (in bounds: s0/4 + 4 <= ld):
          // all 8 loads first, then the codes past n cleared and expanded to
          // E4M3 bytes in registers
          uint32_t wv[8];
#pragma unroll
          for (int e = 0; e < 8; ++e)
            wv[e] = (valid > 0 && idx[e] < X.p)
                        ? __ldg(reinterpret_cast<const uint32_t *>(X.geno + (int64_t)idx[e] * X.ld + (s0 >> 2)))
                        : 0u;
          const uint32_t keep = valid >= 16 ? 0xffffffffu : ((1u << (2 * valid)) - 1u);
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int kk = 16 * e + kr;
            *reinterpret_cast<uint4 *>(stage + kk * 128 + ((c ^ (kk & 7)) << 4)) = spread_word(wv[e] & keep);
          }
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int kk = 16 * e + kr;
            uint8_t *dst = stage + kk * 128 + ((c ^ (kk & 7)) << 4);
            if (valid > 0 && idx[e] < X.p)
              cp_async16(dst, X.geno + (int64_t)idx[e] * X.ld + s0, valid);  // bytes past n zero-filled
            else
              *reinterpret_cast<int4 *>(dst) = make_int4(0, 0, 0, 0);
          }
        }
        if (tid == 0) {
          // the digit tile adds transaction bytes to the phase; the 128
          // arrivals come when each thread's copies of the block have landed
          mbar_expect_tx(&full[s], Sh::B_BYTES);
          bulk_load(stage + Sh::A_BYTES, wtile + (int64_t)(kb0 + it) * Sh::B_BYTES, Sh::B_BYTES, &full[s]);
        }
      }
      cp_async_commit();
      const int rt = it - kXbLag;  // block whose copies are now complete
      if (rt >= 0 && rt < nb) {
        cp_async_wait<kXbLag>();
        fence_proxy_async();
        const int s = rt % ST;
        const uint32_t ph = (uint32_t)(rt / ST) & 1u;
        mbar_arrive(&full[s]);  // one arrival per thread and phase (count 128)
        if (tid == 0) {
          if (!mbar_wait(&full[s], ph, err, kErrFull)) { ok = false; return; }
          tc_fence_after();
          const uint32_t sa = smem_u32(ring + s * Sh::BUF);
          const uint64_t ad = sdesc_mn128(sa), bd = sdesc_k128(sa + Sh::A_BYTES);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            mma_f8(tmem, ad + (uint64_t)(q * 256), bd + (uint64_t)(q * 2), idesc, (rt | q) != 0 ? 1u : 0u);
          mma_commit(&empty[s]);
        }
      }
    };
    load_idx(kb0, idxA);
    if (nb > 1) load_idx(kb0 + 1, idxB);
    for (int it = 0; it < nb + kXbLag && ok; it += 2) {
      step(it, idxA);
      if (it + 2 < nb) load_idx(kb0 + it + 2, idxA);
      if (!ok) break;
      step(it + 1, idxB);
      if (it + 3 < nb) load_idx(kb0 + it + 3, idxB);
    }
    cp_async_wait<0>();
    if (tid == 0) mma_commit(&dbar);
    __syncwarp();
    const bool done = mbar_wait(&dbar, 0u, err, kErrAccFull) && ok;
    tc_fence_after();
    // TMEM lane = sample row, columns b*DWD + d
    uint32_t r[N];
#pragma unroll
    for (int cc = 0; cc < N / 16; ++cc)
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(16 * cc), r + 16 * cc);
    tmem_wait_ld();
    if (done)
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        long long v = 0;
#pragma unroll
        for (int d = 0; d < DWD; ++d) {
          const float f = __uint_as_float(r[b * DWD + d]) * 512.0f;
          v = v * 16 + (long long)__float2int_rn(f);
        }
        V[b] = v;
      }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
      tc_fence_after();
      tmem_dealloc(tmem, Sh::TMEM_COLS);
    }
  }

  // operands of the fused vector update
  const int k = fuse ? (*F.it_base + off) : 0;
  bool run[NB];
  double yi = 0.0, zo[NB], th[NB], ro[NB], cv[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) { zo[b] = th[b] = ro[b] = cv[b] = 0.0; run[b] = false; }
  if (fuse) {
#pragma unroll
    for (int b = 0; b < NB; ++b) run[b] = (b < F.nb) && (F.done[b] < 0);
    if (row) {
      yi = __ldg(F.y + i);
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        zo[b] = F.z[i * NB + b];
        th[b] = F.theta[i * NB + b];
        ro[b] = F.r[i * NB + b];
      }
      const double *bt = F.beta[(k & 1) ^ 1];
#pragma unroll 4
      for (int64_t j = 1; j <= X.c; ++j) {
        const double x = __ldg(X.cov + (j - 1) * X.n + i), aj = __ldg(X.a + j);
#pragma unroll
        for (int b = 0; b < NB; ++b) cv[b] = fma(aj * __ldg(bt + j * NB + b), x, cv[b]);
      }
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
      // all split partials are loaded before any is added
      for (int sp0 = 0; sp0 < S; sp0 += 8) {
        long long v[8][NB];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const long long *src = F.xb_ipart + ((int64_t)(sp0 + u) * F.npad + i) * NB;
#pragma unroll
          for (int b = 0; b < NB; ++b) v[u][b] = (sp0 + u < S) ? __ldcg(src + b) : 0;
        }
        if (sp0 == 0)
#pragma unroll
          for (int b = 0; b < NB; ++b) V[b] = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int b = 0; b < NB; ++b) V[b] += v[u][b];
      }
    }
    if (tid == 0) F.xb_tick[blockIdx.x] = 0u;
  }
  double p[NB][kCPartials];
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int q = 0; q < kCPartials; ++q) p[b][q] = 0.0;
  if (row) {
    const double nmu = (double)F.n * F.mu;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      double qc = 0.0;
      if (F.qcorr) {
        qc = F.qcorr[i * NB + b];
        F.qcorr[i * NB + b] = 0.0;
      }
      if (!run[b]) continue;
      const double unit = F.meta_d[kMaxNB + b] * F.xb_unit;
      const double q = F.meta_d[b] + (double)V[b] * unit + cv[b] + qc;
      row_update(F, i * NB + b, F.tau[b], nmu, (double)F.n, q, (double)A * unit, yi, zo[b], th[b], ro[b], p[b]);
    }
  }
  const int par = (k + 1) & 1;
  const int ops[4] = {0, 0, 1, 0};
#pragma unroll
  for (int b = 0; b < NB; ++b) {
#pragma unroll
    for (int q = 0; q < kCPartials; ++q) red[q][tid] = p[b][q];
    __syncthreads();
    tree_reduce<4>(red, ops, 128);
    if (tid == 0 && run[b]) {
      double *cp = F.c_part[par] + (blockIdx.x * NB + b) * kCPartials;
      cp[0] = red[0][0]; cp[1] = red[1][0]; cp[2] = red[2][0]; cp[3] = red[3][0];
    }
    __syncthreads();
  }
  vec_finalize<NB>(F, par, (int)gridDim.x);
}

template <int NB, int DWD>
size_t g_xt_opted = 0;  // the attribute is set on first use (static + dynamic may pass 48 KB)

size_t xbeta_tc_smem(int NB, int DWD) {
  const int N = ((NB * DWD + 15) / 16) * 16;
  return (size_t)(kXbLag + 2) * (128 * 128 + N * 128) + 1024 + 16;
}

template <int NB, int DWD>
static cudaError_t xbeta_tc_t(const Dsg &X, const Fits &F, int off, int fuse, const double *beta_in,
                              int *scol, uint8_t *wtile, int *err, int num_sms, cudaStream_t s) {
  const size_t smem = xbeta_tc_smem(NB, DWD);
  if (smem > g_xt_opted<NB, DWD>) {
    cudaError_t e = cudaFuncSetAttribute(k_xbeta_tc<NB, DWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    g_xt_opted<NB, DWD> = smem;
  }
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_xbeta_tc<NB, DWD>, 128, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);
  }
  const int rows = (int)((X.n + 127) / 128);
  const int split_cap = std::max(1, per_sm * num_sms / rows);
  // the prep grid strides over the blocks of 128 active positions
  const int maxkb = (int)((X.P + 127) / 128);
  const int pgrid = std::max(1, std::min(maxkb, num_sms));
  const size_t psmem = (size_t)(F.gridA + 1) * sizeof(int);
  k_xprep<NB, DWD><<<pgrid, 128, psmem, s>>>(X, F, off, beta_in, split_cap, scol, wtile, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)rows, kXTMaxSplits);
  k_xbeta_tc<NB, DWD><<<grid, 128, smem, s>>>(X, F, off, fuse, scol, wtile, err);
  return cudaGetLastError();
}

// scol: (P + 127)/128*128 ints; wtile: (P + 127)/128 tiles of N*128 bytes.
cudaError_t launch_xbeta_tc(int NB, const Dsg &X, const Fits &F, int off, int fuse, const double *beta_in,
                            int *scol, uint8_t *wtile, int *err, int num_sms, cudaStream_t s) {
  switch (NB) {
    case 1: return xbeta_tc_t<1, 11>(X, F, off, fuse, beta_in, scol, wtile, err, num_sms, s);
    case 2: return xbeta_tc_t<2, 11>(X, F, off, fuse, beta_in, scol, wtile, err, num_sms, s);
    case 3: return xbeta_tc_t<3, 11>(X, F, off, fuse, beta_in, scol, wtile, err, num_sms, s);
    case 4: return xbeta_tc_t<4, 11>(X, F, off, fuse, beta_in, scol, wtile, err, num_sms, s);
    case 8: return xbeta_tc_t<8, 11>(X, F, off, fuse, beta_in, scol, wtile, err, num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

int xbeta_tc_rows(int NB) { return ((NB * 11 + 15) / 16) * 16; }

// ------------------------------------------------------------------ host

template <int NB, int D, int F2>
size_t g_tc_opted = 0;  // the attribute is set on first use

size_t col_tc_smem(int NB, int D, int T, int f2) {
  int N = NB * D <= 16 ? 16 : (NB * D <= 32 ? 32 : 64);
  return (size_t)6 * (128 * 128 + N * 128 + (f2 ? 4096 : 0)) + 1024 + (size_t)T + 16;  // flags use <= T bytes
}

void col_tc_schedule(int64_t p, int64_t n, int num_sms, TcSchedule *out) {
  const int64_t tiles = (p + 127) / 128, nk = (n + 127) / 128;
  TcSchedule &sc = *out;
  sc.grid = std::max(1, num_sms);  // one CTA per SM, even with fewer tiles (they are then sliced)
  sc.rounds = (int)(tiles / sc.grid);
  sc.rem = (int)(tiles - (int64_t)sc.rounds * sc.grid);
  // slicing pays only when a partial last round is a large share of the pass
  // (measured: with 5 whole rounds and 22 leftover tiles it lost 5 %)
  sc.slices = (sc.rem && sc.rounds <= 2)
                  ? (int)std::max<int64_t>(
                        1, std::min<int64_t>(std::min<int64_t>(nk, sc.grid / sc.rem), kMaxTailSlices))
                  : 0;
  sc.list_stride = 128 * (sc.rounds + 1) + 64;
  sc.slots = sc.grid + (sc.slices ? sc.rem : 0);
}

int tc_tail_rows(int NB, int D) { return NB * D; }

template <int NB, int D, int F2>
static cudaError_t col_tc_t(const Dsg &X, const Fits &F, int off, const uint8_t *xt,
                            const uint8_t *dgt, const TcSchedule &sc, int32_t *tail_part,
                            unsigned *tail_tick, int *err, cudaStream_t s) {
  const size_t smem = col_tc_smem(NB, D, F.T, F2);
  if (smem > g_tc_opted<NB, D, F2>) {
    cudaError_t e =
        cudaFuncSetAttribute(k_col_tc<NB, D, F2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    g_tc_opted<NB, D, F2> = smem;
  }
  k_col_tc<NB, D, F2><<<sc.grid, TcShape<NB, D, F2>::THREADS, smem, s>>>(X, F, off, xt, dgt, sc.rounds, sc.slices,
                                                                           tail_part, tail_tick, err);
  return cudaGetLastError();
}

cudaError_t launch_col_tc(int NB, int D, const Dsg &X, const Fits &F, int off, const uint8_t *xt,
                          const uint8_t *dgt, const TcSchedule &sc, int32_t *tail_part,
                          unsigned *tail_tick, int *err, cudaStream_t s) {
  const bool f2 = X.fmt == FSQR_2BIT;
#define FSQR_TC_CASE(nb, d)                                                                   \
  if (NB == nb && D == d)                                                                     \
    return f2 ? col_tc_t<nb, d, 1>(X, F, off, xt, dgt, sc, tail_part, tail_tick, err, s)      \
              : col_tc_t<nb, d, 0>(X, F, off, xt, dgt, sc, tail_part, tail_tick, err, s);
  FSQR_TC_CASE(1, 7) FSQR_TC_CASE(2, 7) FSQR_TC_CASE(3, 7) FSQR_TC_CASE(4, 7) FSQR_TC_CASE(8, 7)
  FSQR_TC_CASE(1, 6) FSQR_TC_CASE(2, 6) FSQR_TC_CASE(3, 6) FSQR_TC_CASE(4, 6) FSQR_TC_CASE(8, 6)
#undef FSQR_TC_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_quantize_tc(int NB, int D, const Fits &F, int off, uint8_t *dg, cudaStream_t s) {
  const int64_t total = (int64_t)NB * F.npad;
  const unsigned grid = (unsigned)((total + 255) / 256);
#define FSQR_Q_CASE(nb, d) \
  if (NB == nb && D == d) { k_quantize_tc<nb, d><<<grid, 256, 0, s>>>(F, off, dg); return cudaGetLastError(); }
  FSQR_Q_CASE(1, 7) FSQR_Q_CASE(2, 7) FSQR_Q_CASE(3, 7) FSQR_Q_CASE(4, 7) FSQR_Q_CASE(8, 7)
  FSQR_Q_CASE(1, 6) FSQR_Q_CASE(2, 6) FSQR_Q_CASE(3, 6) FSQR_Q_CASE(4, 6) FSQR_Q_CASE(8, 6)
#undef FSQR_Q_CASE
  return cudaErrorInvalidValue;
}

int tc_rows(int NB, int D) { return NB * D <= 16 ? 16 : (NB * D <= 32 ? 32 : 64); }

// 2-bit storage: tile (t, kc) at xt + (t*nk + kc)*4096, row m = column
// 128t + m, 32 bytes = its samples 128kc .. 128kc+127 packed 4 per byte as
// stored, with missing codes (3) and samples >= n or columns >= p set to 0.
__global__ void k_tile_x2(Dsg X, uint8_t *xt, int64_t nk) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // one 16-byte half row
  const int64_t ntile = (X.p + 127) / 128;
  if (g >= ntile * nk * 256) return;
  const int64_t tk = g >> 8;
  const int q = (int)(g & 255), m = q >> 1, h = q & 1;
  const int64_t t = tk / nk, kc = tk - t * nk;
  const int64_t col = t * 128 + m;
  const int64_t b0 = kc * 32 + 16 * h;  // first source byte
  uint8_t out[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    uint32_t byte = 0;
    if (col < X.p && b0 + u < X.ld) byte = X.geno[col * X.ld + b0 + u];
    uint32_t o = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int64_t i = 4 * (b0 + u) + f;
      uint32_t code = (byte >> (2 * f)) & 3u;
      if (code == 3u || i >= X.n) code = 0u;
      o |= code << (2 * f);
    }
    out[u] = (uint8_t)o;
  }
  *reinterpret_cast<uint4 *>(xt + tk * 4096 + (int64_t)q * 16) = *reinterpret_cast<const uint4 *>(out);
}

cudaError_t launch_tile_x2(const Dsg &X, uint8_t *xt, int64_t nk, cudaStream_t s) {
  const int64_t halves = (X.p + 127) / 128 * nk * 256;
  if (halves == 0) return cudaSuccess;
  k_tile_x2<<<(unsigned)((halves + 255) / 256), 256, 0, s>>>(X, xt, nk);
  return cudaGetLastError();
}

cudaError_t launch_tile_x(const Dsg &X, uint8_t *xt, int64_t nk, cudaStream_t s) {
  const int64_t chunks = (X.p + 127) / 128 * nk * 1024;
  if (chunks == 0) return cudaSuccess;
  k_tile_x<<<(unsigned)((chunks + 255) / 256), 256, 0, s>>>(X, xt, nk);
  return cudaGetLastError();
}

}  // namespace fsqr
