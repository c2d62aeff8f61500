// lbm_eqcodec.cuh -- reduced-precision (FP16 / BF16) storage of the
// populations as shifted deviations from the local equilibrium.
//
// The stored 16-bit value of a population is s_L (f_i - f^eq_i(y)) with y the
// node that wrote it (the sender, x - c_i for the population arriving at x
// in direction i), f^eq_i(y) that node's equilibrium of lattice L in
// direction i (Eqs. 27eq, feq, gieq: the lattice weights at the node's
// velocity and temperature times its density, and the energy lattice's
// equilibrium from its total energy and enthalpy), and s_L a per-lattice
// scale.  After a collision f' - f^eq is the non-equilibrium part, a small
// fraction of f even where the flow moves fast or the composition varies by
// factors, so the 8 (BF16) or 11 (FP16) significant bits are spent on it.
//
// The receiver needs the sender's equilibrium: every collision writes a
// per-node FP32 record of the quantities its equilibria are built from, and
// the receiver rebuilds f^eq_i(y) from the sender's record.  Records are
// node-major, rec_w floats per node (16-byte aligned), in two buffers after
// the side planes: the step of AA parity q reads buffer 1 - q (written by the
// previous step) and writes buffer q.
//
// Record layout (floats), as deviations from the reference rest state where
// the quantity has one (T_r, theta_r, RL of each lattice):
//   [0..3]   u_x, u_y, u_z, dtheta            mixture velocity, theta - theta_r
//   [4..7]   dT, drho, drhoE, Gq              T - T_r, rho - RL_f, rho E - RL_g, Gq = Gc / theta
//   [8]      hq = (H + u^2/2) rho / theta     first-moment factor of g^eq
//   [9..]    drho_1 .. drho_M                 coupled species densities - RL_a (padded to 4)
//   [..+3]   u_sp (weak coupling only)         velocity of the species subsystem
// with Gc = rho (h + theta) / (2 theta), h = H + u^2/2.  The momentum and
// energy shifts are formed as deviations without cancellation (the same
// telescoped forms as the collision's equilibria), so the receiver recovers
// the populations to FP32 rounding of their deviations.
#pragma once

#include "lbm_helpers.cuh"

namespace lbm {

template <class Store, class Real>
constexpr bool kEqCodec = (sizeof(Store) == 2) && sizeof(Real) == 4;

__host__ __device__ constexpr int eq_rec_width(int M, int weak) {
  return 8 + ((1 + M + 3) / 4) * 4 + (weak ? 4 : 0);
}

// Offset (in floats) of the record buffers inside the side/scratch buffer:
// after the NSIDE planes, rounded up to 256 bytes.
__host__ __device__ constexpr long long eq_rec_offset(long long N) {
  return ((long long)NSIDE * N + 63) / 64 * 64;
}

__device__ __forceinline__ float* eq_rec_buf(float* side, long long N, int rw, int buf) {
  return side + eq_rec_offset(N) + (long long)buf * rw * N;
}
__device__ __forceinline__ const float* eq_rec_buf(const float* side, long long N, int rw, int buf) {
  return side + eq_rec_offset(N) + (long long)buf * rw * N;
}

template <int M>
struct EqRec {
  float u[3], dth, dT, drho, drhoE, Gq, hq;
  float ra[M];      // species densities minus RL_a
  float usp[3];
};

template <int M>
__device__ __forceinline__ EqRec<M> load_rec(const float* __restrict__ buf, long long node, int rw, int weak) {
  const float4* q = reinterpret_cast<const float4*>(buf + node * rw);
  EqRec<M> r;
  const float4 a = __ldg(q), b = __ldg(q + 1);
  r.u[0] = a.x; r.u[1] = a.y; r.u[2] = a.z; r.dth = a.w;
  r.dT = b.x; r.drho = b.y; r.drhoE = b.z; r.Gq = b.w;
  constexpr int NT = (1 + M + 3) / 4;
  float t[4 * NT];
#pragma unroll
  for (int k = 0; k < NT; ++k) {
    const float4 c = __ldg(q + 2 + k);
    t[4 * k] = c.x; t[4 * k + 1] = c.y; t[4 * k + 2] = c.z; t[4 * k + 3] = c.w;
  }
  r.hq = t[0];
#pragma unroll
  for (int s = 0; s < M; ++s) r.ra[s] = t[1 + s];
  if (weak) {
    const float4 d = __ldg(q + 2 + NT);
    r.usp[0] = d.x; r.usp[1] = d.y; r.usp[2] = d.z;
  } else {
    r.usp[0] = r.u[0]; r.usp[1] = r.u[1]; r.usp[2] = r.u[2];
  }
  return r;
}

template <int M>
__device__ __forceinline__ void store_rec(float* __restrict__ buf, long long node, int rw, int weak,
                                          const EqRec<M>& r) {
  float4* q = reinterpret_cast<float4*>(buf + node * rw);
  q[0] = make_float4(r.u[0], r.u[1], r.u[2], r.dth);
  q[1] = make_float4(r.dT, r.drho, r.drhoE, r.Gq);
  constexpr int NT = (1 + M + 3) / 4;
  float t[4 * NT];
#pragma unroll
  for (int k = 0; k < 4 * NT; ++k) t[k] = 0.0f;
  t[0] = r.hq;
#pragma unroll
  for (int s = 0; s < M; ++s) t[1 + s] = r.ra[s];
#pragma unroll
  for (int k = 0; k < NT; ++k) q[2 + k] = make_float4(t[4 * k], t[4 * k + 1], t[4 * k + 2], t[4 * k + 3]);
  if (weak) q[2 + NT] = make_float4(r.usp[0], r.usp[1], r.usp[2], 0.0f);
}

// Product form Psi_I(xi, z) = prod_a (b_a + k_a z) with b_0 = 1 - xi^2,
// b_{+-1} = (+-xi + xi^2)/2, k_0 = -1, k_{+-1} = 1/2 (Sec. 2.4), as the
// cubic P0 + P1 z + P2 z^2 + P3 z^3 in z, so the species (one z each) share
// the velocity part.
template <int I>
struct PsiCubic {
  float P0, P1, P2;
  static constexpr float kx = cx_of(I) == 0 ? -1.0f : 0.5f;
  static constexpr float ky = cy_of(I) == 0 ? -1.0f : 0.5f;
  static constexpr float kz = cz_of(I) == 0 ? -1.0f : 0.5f;
  static constexpr float P3 = kx * ky * kz;
  __device__ __forceinline__ PsiCubic(const float (&xi)[3]) {
    auto b = [](int c, float x) { return c == 0 ? 1.0f - x * x : 0.5f * ((c > 0 ? x : -x) + x * x); };
    const float bx = b(cx_of(I), xi[0]), by = b(cy_of(I), xi[1]), bz = b(cz_of(I), xi[2]);
    P0 = bx * by * bz;
    P1 = kx * by * bz + bx * ky * bz + bx * by * kz;
    P2 = kx * ky * bz + kx * by * kz + bx * ky * kz;
  }
  __device__ __forceinline__ float operator()(float z) const { return P0 + z * (P1 + z * (P2 + z * P3)); }
};

// The shifts of direction I of every lattice, as deviations from the
// reference rest state (the arithmetic works on d = f - b_ref):
//   sh_L = f^eq_{L,I}(record) - b_ref_{L,I}.
// Species (Eq. 27eq) as rho_a Psi_I(u_sp, R_a T) - b_ref; momentum (Eq. feq)
// and energy (Eqs. gansatz, gieq) lattices in the telescoped deviation forms
// of the collision (lbm_collide.cuh), which carry no O(f) cancellation.
template <int M, int I>
__device__ __forceinline__ void eq_shift(const DevParams<float>& p, const EqRec<M>& r, float (&sh)[M + 2]) {
  constexpr int k2 = c2_of(I);
  constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
  const float T = p.Tr + r.dT;
  if (p.weak) {
    const PsiCubic<I> ps(r.usp);
#pragma unroll
    for (int a = 0; a < M; ++a) sh[a] = (p.RL[a] + r.ra[a]) * ps(p.R_a[a] * T) - p.bref[a][k2];
  } else {
    const PsiCubic<I> ps(r.u);
#pragma unroll
    for (int a = 0; a < M; ++a) sh[a] = (p.RL[a] + r.ra[a]) * ps(p.R_a[a] * T) - p.bref[a][k2];
  }
  const float rho = p.RL[M] + r.drho;
  const float x2[3] = {r.u[0] * r.u[0], r.u[1] * r.u[1], r.u[2] * r.u[2]};
  // f: rho (Psi_I(u, theta) - W_I(theta_r)) + (rho - RL_f) W_I(theta_r)
  sh[M] = rho * pf_diff<float, I>(r.u, x2, p.thr, r.dth) + r.drho * pf_ref<float, I>(p.thr);
  // g: w_I(theta) [E_I + q^eq . c_I / theta] + B_I . Z relative to its rest value
  const float theta = p.thr + r.dth;
  const float Gc = r.Gq * theta;
  const float usq = x2[0] + x2[1] + x2[2];
  const float dP = r.drho * theta + p.RL[M] * r.dth;
  const float P = rho * theta;
  const float E0 = (p.RL[M + 1] + r.drhoE) - 1.5f * P - Gc * usq;
  const float dE0 = r.drhoE - 1.5f * dP - Gc * usq;
  const float uc = dotc<float, I>(r.u);
  const float ucu = r.Gq * uc * uc;
  const float cc = 0.5f * (float)k2;
  const float Ei = E0 + cc * rho + ucu;
  const float dEi = dE0 + cc * r.drho + ucu;
  const float w0 = 1.0f - theta, w1 = 0.5f * theta;
  const float r0 = 1.0f - p.thr, r1 = 0.5f * p.thr;
  const float d0 = -r.dth, d1 = 0.5f * r.dth;
  const float wx = cx ? w1 : w0, wy = cy ? w1 : w0, wz = cz ? w1 : w0;
  const float rx = cx ? r1 : r0, ry = cy ? r1 : r0, rz = cz ? r1 : r0;
  const float ddx = cx ? d1 : d0, ddy = cy ? d1 : d0, ddz = cz ? d1 : d0;
  const float dwi = ddx * wy * wz + rx * ddy * wz + rx * ry * ddz;
  float bz = 0.0f;
  if constexpr (k2 <= 1) {
    const float z1 = 1.0f - 3.0f * theta;
    const float zb = 0.5f * (z1 * dP - 3.0f * r.dth * p.Pr);
    if constexpr (k2 == 0) {
      bz = 3.0f * zb + z1 * Gc * usq;
    } else {
      constexpr int ax = cx ? 0 : (cy ? 1 : 2);
      bz = -0.5f * (zb + z1 * Gc * x2[ax]);
    }
  }
  sh[M + 1] = dwi * Ei + rx * ry * rz * dEi + bz + wx * wy * wz * r.hq * uc;
}

// The record of a node from its coupled moments, in FP64 (initialisation
// and set_populations): rho_a the coupled species densities, rho, j and rho E
// of the mixture lattices, u_sp the species velocity.
template <int M>
__device__ __forceinline__ EqRec<M> eq_record64(const DevParams<double>& p, const double (&rho_a)[M], double rho,
                                               const double (&j)[3], double rhoE, const double (&u_sp)[3]) {
  double rsp = 0.0;
#pragma unroll
  for (int a = 0; a < M; ++a) rsp += rho_a[a];
  double inv_m = 0.0, Y[M];
#pragma unroll
  for (int a = 0; a < M; ++a) {
    Y[a] = rho_a[a] / rsp;
    inv_m += Y[a] * p.inv_mass[a];
  }
  const double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
  const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const double T = T_from_energy64(p, Y, M, rhoE / rho - 0.5 * usq);   // Eqs. (temperature), (temperature2)
  const double th = p.R_U * inv_m * T;
  double H = 0.0;
#pragma unroll
  for (int a = 0; a < M; ++a) H += Y[a] * H_a64(p, a, T);
  const double hk = H + 0.5 * usq;
  const double Gc = rho * (hk + th) / (2.0 * th);
  EqRec<M> r;
#pragma unroll
  for (int c = 0; c < 3; ++c) { r.u[c] = (float)u[c]; r.usp[c] = (float)u_sp[c]; }
  r.dth = (float)(th - p.thr); r.dT = (float)(T - p.Tr);
  r.drho = (float)(rho - p.RL[M]); r.drhoE = (float)(rhoE - p.RL[M + 1]);
  r.Gq = (float)(Gc / th);
  r.hq = (float)(hk * rho / th);
#pragma unroll
  for (int a = 0; a < M; ++a) r.ra[a] = (float)(rho_a[a] - p.RL[a]);
  return r;
}

}  // namespace lbm
