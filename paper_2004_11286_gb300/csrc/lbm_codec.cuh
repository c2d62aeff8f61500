// lbm_codec.cuh -- storage codec of the populations.
//
// Every lattice L is stored as the deviation d = f - b_L,i of its
// populations from the rest equilibrium b of a reference state (the
// host-side table in lbm_api.cu).  FP64 and FP32 storage hold d as it is;
// the reduced-precision types hold s_L d with a per-lattice scale s_L
// (1 / the lattice's reference zeroth moment), and the arithmetic is FP32.
// Deviations are small where the flow is near its reference state, so the
// rounding of storage is relative to them rather than to f.
#pragma once

#include <type_traits>

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

namespace lbm {

template <class Store, class Real, class P>
__device__ __forceinline__ Real codec_decode(const P& p, Store raw, int L) {
  if constexpr (std::is_same<Store, __half>::value) {
    return (Real)(__half2float(raw) * p.inv_scale[L]);
  } else if constexpr (std::is_same<Store, __nv_bfloat16>::value) {
    return (Real)(__bfloat162float(raw) * p.inv_scale[L]);
  } else {
    (void)p; (void)L;
    return (Real)raw;
  }
}

template <class Store, class Real, class P>
__device__ __forceinline__ Real codec_load(const P& p, const Store* __restrict__ ptr, long long idx, int L) {
  return codec_decode<Store, Real>(p, ptr[idx], L);
}

template <class Store, class Real, class P>
__device__ __forceinline__ void codec_store(const P& p, Store* __restrict__ ptr, long long idx, int L, Real d) {
  if constexpr (std::is_same<Store, __half>::value) {
    ptr[idx] = __float2half_rn((float)d * p.scale[L]);
  } else if constexpr (std::is_same<Store, __nv_bfloat16>::value) {
    ptr[idx] = __float2bfloat16_rn((float)d * p.scale[L]);
  } else {
    (void)p; (void)L;
    ptr[idx] = (Store)d;
  }
}

}  // namespace lbm
