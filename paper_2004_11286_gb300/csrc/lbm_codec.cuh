// lbm_codec.cuh -- storage codec of the populations.
//
// FP64 and FP32 storage hold the populations as they are.  The reduced-
// precision storage types hold a shifted, scaled deviation
//     d = s_L (f_i - b_{L,i}),   f_i = b_{L,i} + d / s_L,
// where b_{L,i} is the rest equilibrium of lattice L at a reference state
// (the product weights of that lattice's temperature times its reference
// density) and s_L a per-lattice scale; arithmetic is FP32.  The direction
// index i is always the LOGICAL direction of the population (the AA pattern
// moves values between slots but never changes their direction).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

namespace lbm {

constexpr int MAXS = 10;  // M + 2 <= 10

struct CodecParams {
  float base[MAXS][27];
  float scale[MAXS];
  float inv_scale[MAXS];
};

template <class Store, class Real>
__device__ __forceinline__ Real codec_load(const CodecParams& cp, const Store* __restrict__ p,
                                           long long idx, int L, int i) {
  if constexpr (std::is_same<Store, __half>::value) {
    return (Real)(cp.base[L][i] + __half2float(p[idx]) * cp.inv_scale[L]);
  } else if constexpr (std::is_same<Store, __nv_bfloat16>::value) {
    return (Real)(cp.base[L][i] + __bfloat162float(p[idx]) * cp.inv_scale[L]);
  } else {
    (void)cp; (void)L; (void)i;
    return (Real)p[idx];
  }
}

template <class Store, class Real>
__device__ __forceinline__ void codec_store(const CodecParams& cp, Store* __restrict__ p,
                                            long long idx, int L, int i, Real v) {
  if constexpr (std::is_same<Store, __half>::value) {
    p[idx] = __float2half_rn(((float)v - cp.base[L][i]) * cp.scale[L]);
  } else if constexpr (std::is_same<Store, __nv_bfloat16>::value) {
    p[idx] = __float2bfloat16_rn(((float)v - cp.base[L][i]) * cp.scale[L]);
  } else {
    (void)cp; (void)L; (void)i;
    p[idx] = (Store)v;
  }
}

}  // namespace lbm
