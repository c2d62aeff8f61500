// lbm_train.cu -- training kernels of the learned Stefan-Maxwell closure:
// forward and backward passes of the network (two GELU layers of width 128
// and a linear output layer) for a mini-batch, the mean-squared loss over the
// 3M valid outputs, and the Adam update (Kingma & Ba 2015, Algorithm 1).
// FP32 master weights, packed W1 [H][F] | b1 [H] | W2 [H][H] | b2 [H] |
// W3 [O][H] | b3 [O]; the inference path uses a bf16 copy (lbm_mlp.cuh).
#include <cmath>

#include <cuda_runtime.h>

#include "lbm_train.h"

namespace lbm {

namespace {

constexpr int TB = 64;    // output tile edge
constexpr int TK = 16;    // reduction step

// C[i][j] = sum_k A(i,k) B(k,j) (+ bias[j]),  A(i,k) = A[i*sai + k*sak],
// B(k,j) = B[k*sbk + j*sbj],  C row stride ldc.  64 x 64 tiles, 4 x 4 per thread.
__global__ void __launch_bounds__(256) sgemm_kernel(int m, int n, int kdim, const float* __restrict__ A,
                                                    long long sai, long long sak, const float* __restrict__ B,
                                                    long long sbk, long long sbj, float* __restrict__ C,
                                                    long long ldc, const float* __restrict__ bias) {
  __shared__ float As[TK][TB + 1];
  __shared__ float Bs[TK][TB + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * TB, j0 = blockIdx.x * TB;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < kdim; k0 += TK) {
    for (int e = threadIdx.x; e < TB * TK; e += 256) {
      const int r = e / TK, kk = e % TK;
      const int i = i0 + r, k = k0 + kk;
      As[kk][r] = (i < m && k < kdim) ? A[i * sai + k * sak] : 0.0f;
      const int c = e % TB, kb = e / TB;
      const int j = j0 + c, k2 = k0 + kb;
      Bs[kb][c] = (j < n && k2 < kdim) ? B[k2 * sbk + j * sbj] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = As[kk][ty + 16 * q]; b[q] = Bs[kk][tx + 16 * q]; }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[q][r] += a[q] * b[r];
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + ty + 16 * q;
    if (i >= m) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int j = j0 + tx + 16 * r;
      if (j < n) C[i * ldc + j] = acc[q][r] + (bias ? bias[j] : 0.0f);
    }
  }
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_df(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

__global__ void gelu_kernel(const float* __restrict__ h, float* __restrict__ a, long long count) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) a[e] = gelu_f(h[e]);
}
__global__ void gelu_back_kernel(float* __restrict__ d, const float* __restrict__ h, long long count) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) d[e] *= gelu_df(h[e]);
}
// dout = 2 (out - tgt) / (rows * valid) on the valid outputs, 0 elsewhere;
// *loss += sum (out - tgt)^2 / (rows * valid).
__global__ void out_grad_kernel(const float* __restrict__ out, const float* __restrict__ tgt, float* __restrict__ dout,
                                int rows, int O, int valid, double* __restrict__ loss) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double inv = 1.0 / ((double)rows * valid);
  double l = 0.0;
  if (e < (long long)rows * O) {
    const int j = (int)(e % O);
    if (j < valid) {
      const float d = out[e] - tgt[e];
      dout[e] = (float)(2.0 * inv) * d;
      l = (double)d * d * inv;
    } else {
      dout[e] = 0.0f;
    }
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l);
}
// g[j] = sum_i d[i][j] (bias gradients).
__global__ void colsum_kernel(const float* __restrict__ d, int rows, int cols, float* __restrict__ g) {
  __shared__ float sh[256];
  const int j = blockIdx.x;
  float s = 0.0f;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) s += d[(long long)i * cols + j];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) g[j] = sh[0];
}
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long count, float lr, float c1, float c2) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const float gi = g[e];
  const float mi = 0.9f * m[e] + 0.1f * gi;
  const float vi = 0.999f * v[e] + 0.001f * gi * gi;
  m[e] = mi;
  v[e] = vi;
  w[e] -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
}

inline unsigned blocks(long long n, int b) { return (unsigned)((n + b - 1) / b); }

void sgemm(cudaStream_t s, int m, int n, int k, const float* A, long long sai, long long sak, const float* B,
           long long sbk, long long sbj, float* C, long long ldc, const float* bias) {
  dim3 grid(blocks(n, TB), blocks(m, TB));
  sgemm_kernel<<<grid, 256, 0, s>>>(m, n, k, A, sai, sak, B, sbk, sbj, C, ldc, bias);
}

}  // namespace

cudaError_t mlp_train_grad(cudaStream_t s, const MlpShape& sh, const float* w, const float* X, const float* T,
                           int rows, const MlpScratch& z, float* g, double* d_loss) {
  const int H = sh.H, F = sh.F, O = sh.O;
  const float* W1 = w;
  const float* b1 = W1 + (long long)H * F;
  const float* W2 = b1 + H;
  const float* b2 = W2 + (long long)H * H;
  const float* W3 = b2 + H;
  const float* b3 = W3 + (long long)O * H;
  float* gW1 = g;
  float* gb1 = gW1 + (long long)H * F;
  float* gW2 = gb1 + H;
  float* gb2 = gW2 + (long long)H * H;
  float* gW3 = gb2 + H;
  float* gb3 = gW3 + (long long)O * H;
  const long long nh = (long long)rows * H, no = (long long)rows * O;
  // forward
  sgemm(s, rows, H, F, X, F, 1, W1, 1, F, z.h1, H, b1);
  gelu_kernel<<<blocks(nh, 256), 256, 0, s>>>(z.h1, z.a1, nh);
  sgemm(s, rows, H, H, z.a1, H, 1, W2, 1, H, z.h2, H, b2);
  gelu_kernel<<<blocks(nh, 256), 256, 0, s>>>(z.h2, z.a2, nh);
  sgemm(s, rows, O, H, z.a2, H, 1, W3, 1, H, z.out, O, b3);
  // loss and backward
  cudaMemsetAsync(d_loss, 0, sizeof(double), s);
  out_grad_kernel<<<blocks(no, 256), 256, 0, s>>>(z.out, T, z.dout, rows, O, sh.valid, d_loss);
  sgemm(s, O, H, rows, z.dout, 1, O, z.a2, H, 1, gW3, H, nullptr);
  colsum_kernel<<<O, 256, 0, s>>>(z.dout, rows, O, gb3);
  sgemm(s, rows, H, O, z.dout, O, 1, W3, H, 1, z.d2, H, nullptr);
  gelu_back_kernel<<<blocks(nh, 256), 256, 0, s>>>(z.d2, z.h2, nh);
  sgemm(s, H, H, rows, z.d2, 1, H, z.a1, H, 1, gW2, H, nullptr);
  colsum_kernel<<<H, 256, 0, s>>>(z.d2, rows, H, gb2);
  sgemm(s, rows, H, H, z.d2, H, 1, W2, H, 1, z.d1, H, nullptr);
  gelu_back_kernel<<<blocks(nh, 256), 256, 0, s>>>(z.d1, z.h1, nh);
  sgemm(s, H, F, rows, z.d1, 1, H, X, F, 1, gW1, F, nullptr);
  colsum_kernel<<<H, 256, 0, s>>>(z.d1, rows, H, gb1);
  return cudaGetLastError();
}

cudaError_t mlp_train_forward(cudaStream_t s, const MlpShape& sh, const float* w, const float* X, int rows,
                              const MlpScratch& z) {
  const int H = sh.H, F = sh.F, O = sh.O;
  const float* W1 = w;
  const float* b1 = W1 + (long long)H * F;
  const float* W2 = b1 + H;
  const float* b2 = W2 + (long long)H * H;
  const float* W3 = b2 + H;
  const float* b3 = W3 + (long long)O * H;
  const long long nh = (long long)rows * H;
  sgemm(s, rows, H, F, X, F, 1, W1, 1, F, z.h1, H, b1);
  gelu_kernel<<<blocks(nh, 256), 256, 0, s>>>(z.h1, z.a1, nh);
  sgemm(s, rows, H, H, z.a1, H, 1, W2, 1, H, z.h2, H, b2);
  gelu_kernel<<<blocks(nh, 256), 256, 0, s>>>(z.h2, z.a2, nh);
  sgemm(s, rows, O, H, z.a2, H, 1, W3, 1, H, z.out, O, b3);
  return cudaGetLastError();
}

cudaError_t mlp_adam(cudaStream_t s, float* w, const float* g, float* m, float* v, long long count, float lr, int t) {
  const float c1 = 1.0f / (1.0f - (float)std::pow(0.9, t));
  const float c2 = 1.0f / (1.0f - (float)std::pow(0.999, t));
  adam_kernel<<<blocks(count, 256), 256, 0, s>>>(w, g, m, v, count, lr, c1, c2);
  return cudaGetLastError();
}

}  // namespace lbm
