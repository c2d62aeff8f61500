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
  int closure;                          // 1: learned closure in the step
  const unsigned char* mlp_img;         // device bf16/FP32 image of the network
  unsigned long long* mlp_stats;        // [accepted, fallback] node counters
  const double* jet;                    // opposed-jets frame: inlet equilibria [(L * 27 + i) * 2 + inlet]
};

// Batched ensemble: many independent domains stepped by single launches.
struct BatchGeom {
  long long N;
  int nx, ny, nz;
  int wall_x;               // always 0: the batch runs periodic domains
};
struct BatchCtx {
  cudaStream_t stream;
  const void* params;       // DevParams<Real>[domains] (device)
  const BatchGeom* geom;    // [domains] (device)
  void* const* pops;        // per-domain population buffers (device array of device pointers)
  void* const* side;        // per-domain scratch buffers
  const int2* tiles_c;      // collide tiles (domain, first node), collide_bs nodes each
  int ntiles_c, grid_c;
  const int2* tiles_l;      // stencil tiles, block_l nodes each
  int ntiles_l, grid_l, block_l;
  unsigned* err;
};

struct KernelSet {
  cudaError_t (*init)(const LaunchCtx&, const double* X, const double* u, const double* T, const double* P);
  cudaError_t (*step)(const LaunchCtx&, int parity);
  cudaError_t (*moments)(const LaunchCtx&, int parity, double* out);
  cudaError_t (*get_pops)(const LaunchCtx&, int parity, double* out);
  cudaError_t (*set_pops)(const LaunchCtx&, int parity, const double* in);
  cudaError_t (*diag)(const LaunchCtx&, int parity, double* d_sums);
  cudaError_t (*samples)(const LaunchCtx&, int parity, float* feat, float* tgt);
  cudaError_t (*mlp_forward)(const LaunchCtx&, const float* feat, float* out, long long n);
  cudaError_t (*mlp_pack)(const LaunchCtx&, const float* w, unsigned char* img);
  cudaError_t (*batch_prepare)();
  cudaError_t (*batch_step)(const BatchCtx&, int parity);
  // The complete equilibria of the two inlet states of the opposed-jets frame:
  // buf = [out: S * 27 * 2][zero: S * 27][X: M * 2][u: 3 * 2][T: 2][P: 2].
  cudaError_t (*jet_table)(const LaunchCtx&, double* buf);
  int launches_per_step;
  int setup_launches;                        // kernels of init_fields / set_populations
  int collide_bs;                            // nodes per collide block
  int mlp_F, mlp_O, mlp_nw, mlp_img_bytes;   // network sizes for this species count
  int mlp_step_ok;                           // the step can run the learned closure
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
LBM_DECLARE_SETS(5)
LBM_DECLARE_SETS(6)
LBM_DECLARE_SETS(7)
LBM_DECLARE_SETS(8)
#undef LBM_DECLARE_SETS

}  // namespace lbm
