// lbm_dispatch.h -- launcher table shared by the C-ABI layer and the
// per-species-count instantiation units.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

template <class Real> struct DevParams;
struct CodecParams;

struct LaunchCtx {
  long long N;
  cudaStream_t stream;
  void* pops;
  void* side;
  unsigned* err;
  double* partials;
  const DevParams<double>* p64;
  const DevParams<float>* p32;
  const CodecParams* codec;
  cudaEvent_t* ev;   // 4 events bracketing the step's kernels, or nullptr
};

struct KernelSet {
  cudaError_t (*init)(const LaunchCtx&, const double* X, const double* u, const double* T, const double* P);
  cudaError_t (*step)(const LaunchCtx&, int parity);
  cudaError_t (*moments)(const LaunchCtx&, int parity, double* out);
  cudaError_t (*get_pops)(const LaunchCtx&, int parity, double* out);
  cudaError_t (*set_pops)(const LaunchCtx&, int parity, const double* in);
  cudaError_t (*diag)(const LaunchCtx&, int parity, double* d_sums);
  int launches_per_step;
};

// prec: 0 FP64, 1 FP32, 2 FP16 storage, 3 BF16 storage; nullptr if not built.
const KernelSet* kernel_set_m1(int prec);
const KernelSet* kernel_set_m2(int prec);
const KernelSet* kernel_set_m3(int prec);
const KernelSet* kernel_set_m4(int prec);
const KernelSet* kernel_set_m8(int prec);

}  // namespace lbm
