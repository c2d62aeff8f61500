// lbm_helpers.cuh -- compile-time direction helpers, product-form and
// energy-ansatz pieces shared by the kernels of the D3Q27 step.
#pragma once

#include <type_traits>
#include <utility>

#include "lbm_device.cuh"
#include "lbm_codec.cuh"
#include "lbm_dispatch.h"

namespace lbm {

constexpr int BLOCK = 128;
constexpr int BLOCK_LIGHT = 256;

__device__ __forceinline__ long long gtid() {
  return (long long)blockIdx.x * blockDim.x + threadIdx.x;
}

// ---------------------------------------------------------------------------
// Energy-lattice ansatz coefficients, Eqs. (gansatz), (grad), (RcorrectionPrime):
// G_i = w_i(theta) [A0 + mt . c_i + sum_ab n_ab c_ia c_ib] + B_i . Z, with
// A0 = M0 - tr(N)/(2 theta), mt = m / theta, n = N/(2 theta^2), N = M - M0 theta I,
// Z_a = (1 - 3 theta)/(2 theta) N_aa.
// ---------------------------------------------------------------------------
template <class Real>
struct GCoef {
  Real A0, nxx, nyy, nzz, nxy, nxz, nyz, Z[3];
  Triplet<Real> w;
};

template <class Real>
__device__ __forceinline__ GCoef<Real> g_coef(Real theta, Real M0, const Real (&Mt)[6]) {
  // Mt = (xx, yy, zz, xy, xz, yz)
  GCoef<Real> c;
  Real Nxx = Mt[0] - M0 * theta, Nyy = Mt[1] - M0 * theta, Nzz = Mt[2] - M0 * theta;
  Real inv_t = Real(1) / theta;
  Real h = Real(0.5) * inv_t * inv_t;
  c.A0 = M0 - Real(0.5) * inv_t * (Nxx + Nyy + Nzz);
  c.nxx = h * Nxx; c.nyy = h * Nyy; c.nzz = h * Nzz;
  c.nxy = Real(2) * h * Mt[3]; c.nxz = Real(2) * h * Mt[4]; c.nyz = Real(2) * h * Mt[5];
  Real zf = (Real(1) - Real(3) * theta) * Real(0.5) * inv_t;
  c.Z[0] = zf * Nxx; c.Z[1] = zf * Nyy; c.Z[2] = zf * Nzz;
  c.w.z = Real(1) - theta; c.w.p = Real(0.5) * theta; c.w.m = c.w.p;   // Eq. (w0)
  return c;
}

// Weight-free bracket of h_i without the first-moment term, and B_i . Z (Eq. Bi).
template <class Real, int I>
__device__ __forceinline__ Real g_even_part(const GCoef<Real>& c) {
  constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
  Real s = c.A0;
  if (cx) s += c.nxx;
  if (cy) s += c.nyy;
  if (cz) s += c.nzz;
  if (cx && cy) s += (cx * cy > 0 ? c.nxy : -c.nxy);
  if (cx && cz) s += (cx * cz > 0 ? c.nxz : -c.nxz);
  if (cy && cz) s += (cy * cz > 0 ? c.nyz : -c.nyz);
  return s;
}
template <class Real, int I>
__device__ __forceinline__ Real g_BZ(const GCoef<Real>& c) {
  constexpr int k2 = c2_of(I);
  if (k2 == 0) return c.Z[0] + c.Z[1] + c.Z[2];
  if (k2 == 1) {
    constexpr int a = cx_of(I) ? 0 : (cy_of(I) ? 1 : 2);
    return Real(-0.5) * c.Z[a];
  }
  return Real(0);
}
template <class Real, int I>
__device__ __forceinline__ Real dotc(const Real (&v)[3]) {
  constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
  Real s = Real(0);
  if (cx) s += (cx > 0 ? v[0] : -v[0]);
  if (cy) s += (cy > 0 ? v[1] : -v[1]);
  if (cz) s += (cz > 0 ? v[2] : -v[2]);
  return s;
}

// Compile-time loop over the 27 velocities.
template <int I, int END, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < END) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, END>(f);
  }
}

// B_i . Z for a vector Z (Eq. Bi): 1 on the rest velocity for every component,
// -1/2 |c_ia| on the six face velocities, 0 elsewhere.
template <class Real, int I>
__device__ __forceinline__ Real BdotZ(const Real (&Z)[3]) {
  constexpr int k2 = c2_of(I);
  if constexpr (k2 == 0) return Z[0] + Z[1] + Z[2];
  else if constexpr (k2 == 1) {
    constexpr int a = cx_of(I) ? 0 : (cy_of(I) ? 1 : 2);
    return Real(-0.5) * Z[a];
  } else {
    return Real(0);
  }
}

// Product of three triplets for velocity I: t_x(c_x) t_y(c_y) t_z(c_z).
template <class Real, int I>
__device__ __forceinline__ Real prod3(const Triplet<Real>& tx, const Triplet<Real>& ty, const Triplet<Real>& tz) {
  return tri(tx, cx_of(I)) * tri(ty, cy_of(I)) * tri(tz, cz_of(I));
}

// Exact telescoped difference a_x a_y a_z - r_x r_y r_z with da = a - r.
template <class Real, int I>
__device__ __forceinline__ Real prod3_diff(const Triplet<Real> (&a)[3], const Triplet<Real> (&r)[3],
                                           const Triplet<Real> (&da)[3]) {
  constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
  return tri(da[0], cx) * tri(a[1], cy) * tri(a[2], cz) + tri(r[0], cx) * tri(da[1], cy) * tri(a[2], cz)
       + tri(r[0], cx) * tri(r[1], cy) * tri(da[2], cz);
}

// Product-form equilibrium relative to the reference rest state (Sec. 2.4):
// for velocity xi and zeta = zr + dz, the triplets a = Psi(xi, zeta),
// r = Psi(0, zr) and their exact difference
//   da = (-xi^2 - dz, (xi + xi^2 + dz)/2, (-xi + xi^2 + dz)/2).
template <class Real>
struct PFDev {
  Triplet<Real> a[3], r[3], da[3];
};
template <class Real>
__device__ __forceinline__ void pf_dev(PFDev<Real>& P, const Real (&xi)[3], Real zr, Real dz) {
  const Real z = zr + dz;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Real x = xi[c], x2 = x * x;
    P.r[c].z = Real(1) - zr; P.r[c].p = Real(0.5) * zr; P.r[c].m = P.r[c].p;
    P.a[c].z = Real(1) - (x2 + z); P.a[c].p = Real(0.5) * (x + x2 + z); P.a[c].m = Real(0.5) * (-x + x2 + z);
    P.da[c].z = -(x2 + dz); P.da[c].p = Real(0.5) * (x + x2 + dz); P.da[c].m = Real(0.5) * (-x + x2 + dz);
  }
}

// 1-D triplets computed on the fly (c is a compile-time constant at every
// call): a = Psi_c(x, z), r = Psi_c(0, zr), da = a - r for z = zr + dz, and
// the velocity difference Psi_c(x) - Psi_c(x + V) with v = V (2x + V).
template <class Real>
__device__ __forceinline__ Real pf_a(int c, Real x, Real x2, Real z) {
  return c == 0 ? Real(1) - (x2 + z) : Real(0.5) * ((c > 0 ? x : -x) + x2 + z);
}
template <class Real>
__device__ __forceinline__ Real pf_r(int c, Real zr) {
  return c == 0 ? Real(1) - zr : Real(0.5) * zr;
}
template <class Real>
__device__ __forceinline__ Real pf_da(int c, Real x, Real x2, Real dz) {
  return c == 0 ? -(x2 + dz) : Real(0.5) * ((c > 0 ? x : -x) + x2 + dz);
}
template <class Real>
__device__ __forceinline__ Real pf_v(int c, Real V, Real v) {
  return c == 0 ? v : Real(-0.5) * (v + (c > 0 ? V : -V));
}
// Psi_I(xi, zr + dz) - Psi_I(0, zr), telescoped over the axes (no cancellation).
template <class Real, int I>
__device__ __forceinline__ Real pf_diff(const Real (&xi)[3], const Real (&x2)[3], Real zr, Real dz) {
  constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
  const Real z = zr + dz;
  return pf_da<Real>(cx, xi[0], x2[0], dz) * pf_a<Real>(cy, xi[1], x2[1], z) * pf_a<Real>(cz, xi[2], x2[2], z)
       + pf_r<Real>(cx, zr) * pf_da<Real>(cy, xi[1], x2[1], dz) * pf_a<Real>(cz, xi[2], x2[2], z)
       + pf_r<Real>(cx, zr) * pf_r<Real>(cy, zr) * pf_da<Real>(cz, xi[2], x2[2], dz);
}
// W_I = Psi_I(0, zr), the reference rest weights.
template <class Real, int I>
__device__ __forceinline__ Real pf_ref(Real zr) {
  return pf_r<Real>(cx_of(I), zr) * pf_r<Real>(cy_of(I), zr) * pf_r<Real>(cz_of(I), zr);
}

// Paired FP32 arithmetic (the f32x2 instructions of sm_100 and later): two
// independent lanes per instruction.
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long ra, rb, rd;
  memcpy(&ra, &a, 8);
  memcpy(&rb, &b, 8);
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
  float2 d;
  memcpy(&d, &rd, 8);
  return d;
}

}  // namespace lbm
