// lbm_dispatch.h -- launcher table shared by the C-ABI layer and the
// per-species-count instantiation units.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

template <class Real> struct DevParams;

struct LaunchCtx {
  long long N;
  cudaStream_t stream;
  void* pops;
  void* side;
  unsigned* err;
  double* partials;
  const DevParams<double>* p64;
  const DevParams<float>* p32;
  const double* base;   // device table [S][27] of the reference rest equilibria
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

// One launcher table per (species count, precision); see inst_m*_*.cu.
#define LBM_DECLARE_SETS(MM)                           \
  const KernelSet* kernel_set_m##MM##_f64();           \
  const KernelSet* kernel_set_m##MM##_f32();           \
  const KernelSet* kernel_set_m##MM##_f16();           \
  const KernelSet* kernel_set_m##MM##_bf16();
LBM_DECLARE_SETS(1)
LBM_DECLARE_SETS(2)
LBM_DECLARE_SETS(3)
LBM_DECLARE_SETS(4)
LBM_DECLARE_SETS(8)
#undef LBM_DECLARE_SETS

}  // namespace lbm
