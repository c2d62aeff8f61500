// lbm_noalloc.cu -- conservation sums that allocate nothing.
//
// For callers that cannot call cudaMalloc at the point of use: code running
// under a pool or arena that owns all device memory, plugins handed device
// pointers by a host application that forbids allocation, or real-time loops
// where an allocation (and its implicit synchronisation) is not allowed.
// The reduction's per-block partial sums, which lbm_mix_diagnostics keeps in
// the handle's cudaMalloc'd block, live here in a file-scope __device__ array
// of fixed size that every GPU loading the library holds until exit.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/lbm_mix.h"

void lbm_set_thread_error(const std::string& msg);   // lbm_api.cu

namespace {

constexpr int NA_BLOCK = 256;
constexpr int NA_MAXV = 16;
// 2^18 doubles (2 MiB): per-block partials of up to M + 5 = 13 values, then
// the final sums.  Enough for ~5.1e6 nodes at M = 8 and ~8.4e6 at M = 3.
constexpr long long NA_CAP = 1LL << 18;

static __device__ __align__(256) double g_na_scratch[NA_CAP];

// Device address of g_na_scratch per device, taken once with that device current.
constexpr int NA_MAXDEV = 64;
std::mutex g_na_mu;
double* g_na_ptr[NA_MAXDEV] = {};

__device__ __forceinline__ double na_warp(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// One value set per node: species densities, rho, momentum (3) and rho E of
// natural-layout full populations [M+2][27][N].
__global__ void __launch_bounds__(NA_BLOCK)
na_partials_kernel(const double* __restrict__ pops, int M, long long N, double* __restrict__ partials) {
  __shared__ double red[NA_BLOCK / 32][NA_MAXV];
  const int nv = M + 5;
  double v[NA_MAXV];
  for (int s = 0; s < NA_MAXV; ++s) v[s] = 0.0;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n < N) {
    for (int i = 0; i < 27; ++i) {
      const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
      for (int a = 0; a < M; ++a) v[a] += pops[((long long)a * 27 + i) * N + n];
      const double f = pops[((long long)M * 27 + i) * N + n];
      v[M] += f;
      v[M + 1] += cx * f; v[M + 2] += cy * f; v[M + 3] += cz * f;
      v[M + 4] += pops[((long long)(M + 1) * 27 + i) * N + n];
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int s = 0; s < nv; ++s) {
    const double t = na_warp(v[s]);
    if (lane == 0) red[wid][s] = t;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double t = 0.0;
    for (int w = 0; w < NA_BLOCK / 32; ++w) t += red[w][threadIdx.x];
    partials[(long long)blockIdx.x * nv + threadIdx.x] = t;
  }
}

__global__ void __launch_bounds__(NA_BLOCK)
na_final_kernel(const double* __restrict__ partials, int nblocks, int nv, double* __restrict__ sums) {
  __shared__ double sh[NA_BLOCK];
  for (int s = 0; s < nv; ++s) {
    double t = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += NA_BLOCK) t += partials[(long long)b * nv + s];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int w = NA_BLOCK / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) sums[s] = sh[0];
    __syncthreads();
  }
}

lbm_status na_fail(lbm_status s, const std::string& m) {
  lbm_set_thread_error(m);
  return s;
}

}  // namespace

extern "C" lbm_status lbm_mix_conserved_sums_noalloc(const double* pops, int M, int nx, int ny, int nz,
                                                     double* sums, void* cuda_stream) {
  if (!pops || !sums) return na_fail(LBM_ERR_ARG, "NULL pointer");
  if (M < 1 || M > 8) return na_fail(LBM_ERR_ARG, "M must be in 1..8");
  if (nx < 1 || ny < 1 || nz < 1) return na_fail(LBM_ERR_ARG, "grid dimensions must be >= 1");
  const long long N = (long long)nx * ny * nz;
  const long long nblocks = (N + NA_BLOCK - 1) / NA_BLOCK;
  const int nv = M + 5;
  if (nblocks * nv > NA_CAP)
    return na_fail(LBM_ERR_ARG, "grid too large for the static scratch (2^18 doubles: at most " +
                                    std::to_string((NA_CAP / nv) * NA_BLOCK) + " nodes for M = " +
                                    std::to_string(M) + ")");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(LBM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= NA_MAXDEV) return na_fail(LBM_ERR_UNSUPPORTED, "device index beyond 63");
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_ptr[dev]) {
      // First call on this device: take the device address of the array.
      e = cudaGetSymbolAddress((void**)&g_na_ptr[dev], g_na_scratch);
      if (e != cudaSuccess) {
        g_na_ptr[dev] = nullptr;
        return na_fail(LBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
    }
    scratch = g_na_ptr[dev];
  }
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  // Every block writes its own partials, so nothing in the array needs clearing.
  na_partials_kernel<<<(unsigned)nblocks, NA_BLOCK, 0, stream>>>(pops, M, N, scratch);
  na_final_kernel<<<1, NA_BLOCK, 0, stream>>>(scratch, (int)nblocks, nv, sums);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(LBM_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return LBM_OK;
}
