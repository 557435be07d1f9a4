// Learned warm start: the kernels of a small multilayer perceptron (training
// and inference) and of the start it proposes.
//
// The paper warm-starts each fit of a lambda path from the previous solution
// (Section 7). Here a network f maps per-feature inputs of a new (tau,
// lambda) to a starting coefficient:
//   u_j = (tau, lambda/lambda_max(tau), x~_j^T v / (n lambda_max(tau))),
//   v_i = tau - 1{y_i < y_(ceil(n tau))},
//   h_{l+1} = relu(h_l W_l + b_l) (hidden layers), f = h W_last + b_last;
//   beta_0 = y_(ceil(n tau)), beta_j = sd(y) f(u_j), z = y - X~ beta,
//   theta_i = (tau - 1{z_i < 0}) / n.
// Training minimises sum_r w_r (f(u_r) - t_r)^2 / sum_r w_r by Adam (Kingma
// and Ba, 2015). Parameters are FP32, flat: W_0 (row-major d_0 x d_1), b_0,
// W_1, b_1, ... Every reduction runs in a fixed order (deterministic).
#include <math.h>
#include <stdint.h>

#include "fsqr_internal.h"

namespace fsqr {

// ------------------------------------------------------------------ GEMM

// C[M x N] = epi(op(A)[M x K] op(B)[K x N]) in FP32.
//   op(A)(m, k) = TA ? A[k * lda + m] : A[m * lda + k]
//   op(B)(k, n) = TB ? B[n * ldb + k] : B[k * ldb + n]
// epi: kEpiPlain C = acc; kEpiBiasRelu C = max(acc + bias[n], 0);
//      kEpiBias C = acc + bias[n]; kEpiMask C = acc * (mask[m * ldc + n] > 0).
enum { kEpiPlain = 0, kEpiBiasRelu = 1, kEpiBias = 2, kEpiMask = 3 };

constexpr int kGT = 64;   // output tile
constexpr int kGK = 16;   // k step

template <bool TA, bool TB>
__global__ void __launch_bounds__(256)
    k_gemm(int M, int N, int K, const float *__restrict__ A, int lda, const float *__restrict__ B, int ldb,
           float *__restrict__ C, int ldc, int epi, const float *__restrict__ bias,
           const float *__restrict__ mask) {
  __shared__ float sA[kGK][kGT + 4];
  __shared__ float sB[kGK][kGT + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * kGT, n0 = blockIdx.x * kGT;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  for (int k0 = 0; k0 < K; k0 += kGK) {
    // 64 x 16 elements of each operand, 4 per thread
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = threadIdx.x + e * 256;  // 0..1023
      int mm, kk;
      if (TA) { mm = idx & 63; kk = idx >> 6; } else { kk = idx & 15; mm = idx >> 4; }
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.f;
      if (gm < M && gk < K) v = TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
      sA[kk][mm] = v;
      int nn, kb;
      if (TB) { kb = idx & 15; nn = idx >> 4; } else { nn = idx & 63; kb = idx >> 6; }
      const int gn = n0 + nn, gkb = k0 + kb;
      float w = 0.f;
      if (gn < N && gkb < K) w = TB ? B[(int64_t)gn * ldb + gkb] : B[(int64_t)gkb * ldb + gn];
      sB[kb][nn] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = sA[kk][ty * 4 + q]; b[q] = sB[kk][tx * 4 + q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int m = m0 + ty * 4 + p;
    if (m >= M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int n = n0 + tx * 4 + q;
      if (n >= N) continue;
      float v = acc[p][q];
      if (epi == kEpiBiasRelu) v = fmaxf(v + bias[n], 0.f);
      else if (epi == kEpiBias) v = v + bias[n];
      else if (epi == kEpiMask) v = (mask[(int64_t)m * ldc + n] > 0.f) ? v : 0.f;
      C[(int64_t)m * ldc + n] = v;
    }
  }
}

static cudaError_t gemm(bool ta, bool tb, int M, int N, int K, const float *A, int lda, const float *B, int ldb,
                        float *C, int ldc, int epi, const float *bias, const float *mask, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((N + kGT - 1) / kGT), (unsigned)((M + kGT - 1) / kGT));
  if (!ta && !tb) k_gemm<false, false><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, epi, bias, mask);
  else if (ta && !tb) k_gemm<true, false><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, epi, bias, mask);
  else if (!ta && tb) k_gemm<false, true><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, epi, bias, mask);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// ------------------------------------------------------- small kernels

// out[c] = sum_r G[r * cols + c], one CTA per column, fixed-order tree.
__global__ void __launch_bounds__(256) k_colsum(const float *__restrict__ G, int64_t rows, int cols,
                                                float *__restrict__ out) {
  __shared__ float sh[256];
  const int c = blockIdx.x;
  float a = 0.f;
  for (int64_t r = threadIdx.x; r < rows; r += 256) a += G[r * cols + c];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = sh[0];
}

// One CTA: wsum = sum w, g_r = 2 w_r (f_r - t_r) / wsum, loss = sum w (f-t)^2 / wsum
// (loss and its terms in FP64).
__global__ void __launch_bounds__(1024) k_loss(const float *__restrict__ f, const float *__restrict__ t,
                                               const float *__restrict__ w, int64_t rows, float *__restrict__ g,
                                               double *__restrict__ loss) {
  __shared__ double sh[1024];
  double ws = 0.0;
  for (int64_t r = threadIdx.x; r < rows; r += 1024) ws += (double)w[r];
  sh[threadIdx.x] = ws;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double W = sh[0];
  __syncthreads();
  double l = 0.0;
  for (int64_t r = threadIdx.x; r < rows; r += 1024) {
    const double e = (double)f[r] - (double)t[r];
    l += (double)w[r] * e * e;
    if (g) g[r] = (float)(2.0 * (double)w[r] * e / W);
  }
  sh[threadIdx.x] = l;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = sh[0] / W;
}

// Adam with bias correction; step counts from 1.
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int64_t count, double c1, double c2, float lr, float b1, float b2,
                       float eps) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = (float)((double)mi / c1), vh = (float)((double)vi / c2);
  p[i] -= lr * mh / (sqrtf(vh) + eps);
}

// splitmix64 (Steele, Lea and Flood, 2014): a counter-based 64-bit mixer.
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Uniform batch rows: row r of step `step` draws index mix64(seed, step, r) mod rows.
__global__ void k_sample(const float *__restrict__ x, const float *__restrict__ t, const float *__restrict__ w,
                         int64_t rows, int in, int batch, uint64_t seed, int64_t step, float *__restrict__ xb,
                         float *__restrict__ tb, float *__restrict__ wb) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= batch) return;
  const uint64_t h = mix64(mix64(seed ^ (uint64_t)step * 0xD1B54A32D192ED03ull) + (uint64_t)r);
  const int64_t src = (int64_t)(h % (uint64_t)rows);
  for (int c = 0; c < in; ++c) xb[(int64_t)r * in + c] = x[src * in + c];
  tb[r] = t[src];
  wb[r] = w[src];
}

// He-uniform weights U(-sqrt(6/fan_in), sqrt(6/fan_in)), zero biases.
__global__ void k_mlp_init(float *__restrict__ p, int64_t count, const int *__restrict__ dims, int L,
                           uint64_t seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  int64_t o = 0;
  for (int l = 0; l < L; ++l) {
    const int64_t nw = (int64_t)dims[l] * dims[l + 1];
    if (i < o + nw) {
      const double u = (double)(mix64(seed + (uint64_t)i) >> 11) * 0x1.0p-53;  // [0, 1)
      const double a = sqrt(6.0 / (double)dims[l]);
      p[i] = (float)((2.0 * u - 1.0) * a);
      return;
    }
    o += nw;
    if (i < o + dims[l + 1]) { p[i] = 0.f; return; }
    o += dims[l + 1];
  }
}

// ---------------------------------------------------------- warm start

// u[(j-1)*3 + .] = (tau, frac, s_j / (n lambda_max)) for j = 1..P-1.
__global__ void k_warm_features(const double *__restrict__ s, int64_t P, double n, double tau, double frac,
                                const double *__restrict__ lmax, float *__restrict__ u) {
  const int64_t j = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  const double L = *lmax;
  float *o = u + (j - 1) * 3;
  o[0] = (float)tau;
  o[1] = (float)frac;
  o[2] = (float)(L > 0.0 ? s[j] / (n * L) : 0.0);
}

// beta_0 = q, beta_j = sdy * f_{j-1}.
__global__ void k_warm_beta(const float *__restrict__ f, int64_t P, const double *__restrict__ q, double sdy,
                            double *__restrict__ beta) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  beta[j] = (j == 0) ? *q : sdy * (double)f[j - 1];
}

// z = y - xb, theta_i = (tau - 1{z_i < 0}) / n.
__global__ void k_warm_dual(const double *__restrict__ y, const double *__restrict__ xb, int64_t n, double tau,
                            double *__restrict__ z, double *__restrict__ theta) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double zi = y[i] - xb[i];
  z[i] = zi;
  theta[i] = (tau - (zi < 0.0 ? 1.0 : 0.0)) / (double)n;
}

// ----------------------------------------------------------- launchers

static const int kDims[kMlpLayers + 1] = {kMlpIn, kMlpHidden, kMlpHidden, kMlpHidden, 1};

int64_t mlp_param_count() {
  int64_t c = 0;
  for (int l = 0; l < kMlpLayers; ++l) c += (int64_t)kDims[l] * kDims[l + 1] + kDims[l + 1];
  return c;
}

template <class T>
static void layer_ptrs(T *p, T **W, T **b) {
  int64_t o = 0;
  for (int l = 0; l < kMlpLayers; ++l) {
    W[l] = p + o;
    o += (int64_t)kDims[l] * kDims[l + 1];
    b[l] = p + o;
    o += kDims[l + 1];
  }
}

// Forward pass of `rows` inputs; H[l] (rows x hidden) keep the hidden
// outputs for the backward pass; out (rows).
cudaError_t mlp_forward(const float *params, const float *x, int64_t rows, float *const *H, float *out,
                        cudaStream_t s) {
  const float *W[kMlpLayers], *b[kMlpLayers];
  layer_ptrs(params, W, b);
  const float *in = x;
  for (int l = 0; l < kMlpLayers; ++l) {
    const bool last = l == kMlpLayers - 1;
    float *o = last ? out : H[l];
    cudaError_t e = gemm(false, false, (int)rows, kDims[l + 1], kDims[l], in, kDims[l], W[l], kDims[l + 1], o,
                         kDims[l + 1], last ? kEpiBias : kEpiBiasRelu, b[l], nullptr, s);
    if (e != cudaSuccess) return e;
    in = o;
  }
  return cudaSuccess;
}

// Loss and its gradient over `rows` inputs (forward included). H: hidden
// outputs (kMlpLayers-1 buffers of rows x hidden), G0/G1: rows x hidden
// scratch, f/g: rows.
cudaError_t mlp_grad(const float *params, const float *x, const float *t, const float *w, int64_t rows,
                     float *const *H, float *G0, float *G1, float *f, float *g, float *grad, double *loss,
                     cudaStream_t s) {
  cudaError_t e = mlp_forward(params, x, rows, H, f, s);
  if (e != cudaSuccess) return e;
  k_loss<<<1, 1024, 0, s>>>(f, t, w, rows, g, loss);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const float *W[kMlpLayers], *b[kMlpLayers];
  layer_ptrs(params, W, b);
  float *gW[kMlpLayers], *gb[kMlpLayers];
  layer_ptrs(grad, gW, gb);
  const float *up = g;  // gradient w.r.t. the output of layer l (rows x d_{l+1})
  float *bufs[2] = {G0, G1};
  for (int l = kMlpLayers - 1; l >= 0; --l) {
    const int din = kDims[l], dout = kDims[l + 1];
    const float *hin = l == 0 ? x : H[l - 1];
    // dW_l = h_l^T up, db_l = column sums of up
    if ((e = gemm(true, false, din, dout, (int)rows, hin, din, up, dout, gW[l], dout, kEpiPlain, nullptr, nullptr,
                  s)) != cudaSuccess)
      return e;
    k_colsum<<<dout, 256, 0, s>>>(up, rows, dout, gb[l]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (l == 0) break;
    // gradient w.r.t. h_l: (up W_l^T) masked by relu'(h_l)
    float *dn = bufs[l & 1];
    if ((e = gemm(false, true, (int)rows, din, dout, up, dout, W[l], dout, dn, din, kEpiMask, nullptr, H[l - 1],
                  s)) != cudaSuccess)
      return e;
    up = dn;
  }
  return cudaSuccess;
}

cudaError_t mlp_adam(float *p, const float *g, float *m, float *v, int64_t count, int64_t step, float lr,
                     cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const double c1 = 1.0 - pow(0.9, (double)step), c2 = 1.0 - pow(0.999, (double)step);
  k_adam<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(p, g, m, v, count, c1, c2, lr, b1, b2, eps);
  return cudaGetLastError();
}

cudaError_t mlp_sample(const float *x, const float *t, const float *w, int64_t rows, int batch, uint64_t seed,
                       int64_t step, float *xb, float *tb, float *wb, cudaStream_t s) {
  k_sample<<<(batch + 255) / 256, 256, 0, s>>>(x, t, w, rows, kMlpIn, batch, seed, step, xb, tb, wb);
  return cudaGetLastError();
}

cudaError_t mlp_init(float *p, int *d_dims, uint64_t seed, cudaStream_t s) {
  const int64_t count = mlp_param_count();
  cudaError_t e = cudaMemcpyAsync(d_dims, kDims, sizeof kDims, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  k_mlp_init<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(p, count, d_dims, kMlpLayers, seed);
  return cudaGetLastError();
}

cudaError_t launch_warm_features(const double *s_col, int64_t P, int64_t n, double tau, double frac,
                                 const double *lmax, float *u, cudaStream_t s) {
  if (P <= 1) return cudaSuccess;
  k_warm_features<<<(unsigned)((P - 1 + 255) / 256), 256, 0, s>>>(s_col, P, (double)n, tau, frac, lmax, u);
  return cudaGetLastError();
}

cudaError_t launch_warm_beta(const float *f, int64_t P, const double *q, double sdy, double *beta, cudaStream_t s) {
  k_warm_beta<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(f, P, q, sdy, beta);
  return cudaGetLastError();
}

cudaError_t launch_warm_dual(const double *y, const double *xb, int64_t n, double tau, double *z, double *theta,
                             cudaStream_t s) {
  k_warm_dual<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(y, xb, n, tau, z, theta);
  return cudaGetLastError();
}

}  // namespace fsqr
