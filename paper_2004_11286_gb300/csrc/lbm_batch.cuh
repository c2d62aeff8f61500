// lbm_batch.cuh -- the step of many independent domains (an ensemble of
// uneven grids, each with its own species constants and reference state)
// by one launch per kernel: persistent blocks walk a list of tiles (domain,
// first node), taking the domain's parameters into shared memory whenever
// the domain changes.  Each node's work is exactly the single-domain step's.
#pragma once

#include "lbm_collide.cuh"

namespace lbm {

template <int M, class Real, class Store, int PAR>
__global__ void __launch_bounds__(collide_block<M, Real, 0, Store>(), collide_min_blocks<M, Real, 0, Store>())
collide_batch_kernel(const DevParams<Real>* __restrict__ params, void* const* __restrict__ pops,
                     void* const* __restrict__ side, const int2* __restrict__ tiles, int ntiles,
                     unsigned* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(16) DevParams<Real> sp;
  static_assert(sizeof(DevParams<Real>) % 8 == 0, "8-byte words");
  int cur = -1;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int2 tl = tiles[t];
    if (tl.x != cur) {                       // block-uniform
      __syncthreads();
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(params + tl.x);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&sp);
      for (int k = threadIdx.x; k < (int)(sizeof(DevParams<Real>) / 8); k += blockDim.x) dst[k] = src[k];
      __syncthreads();
      cur = tl.x;
    }
    collide_node<M, Real, Store, PAR, 0>(sp, static_cast<Store*>(pops[cur]), static_cast<Real*>(side[cur]), err,
                                         nullptr, nullptr, (long long)tl.y + threadIdx.x, smem_raw);
  }
}

template <class Real>
__global__ void __launch_bounds__(BLOCK_LIGHT)
grad_GK_batch_kernel(const BatchGeom* __restrict__ geom, void* const* __restrict__ side,
                     const int2* __restrict__ tiles, int ntiles) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int2 tl = tiles[t];
    const BatchGeom g = geom[tl.x];
    grad_GK_node<Real>(g, static_cast<Real*>(side[tl.x]), (long long)tl.y + threadIdx.x);
  }
}

template <class Real>
__global__ void __launch_bounds__(BLOCK_LIGHT)
grad_X_batch_kernel(const BatchGeom* __restrict__ geom, void* const* __restrict__ side,
                    const int2* __restrict__ tiles, int ntiles) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int2 tl = tiles[t];
    const BatchGeom g = geom[tl.x];
    grad_X_node<Real>(g, static_cast<Real*>(side[tl.x]), (long long)tl.y + threadIdx.x);
  }
}

}  // namespace lbm
