// lbm_stencil.cuh -- the deferred non-local terms of the step, the two stencil
// passes that build them, and the readers of the state (observables,
// checkpoint copies) that apply them.
//
// The D3Q27 correction A_i . X (Eq. fwithcorrection) and the grad C_p part of
// q^corr (Eq. corrFourier) enter the post-collision populations additively,
// but they need the neighbours' time-t moments, which a node does not have
// when it collides.  Each collision therefore writes its populations without
// them, and the node that receives a population at the next step adds the
// sender's term before using it:
//   f_i += 1/2 c_i . X(x)             (the six face directions)
//   g_i += w_i(theta_x) c_i . K(x),   K = (1/2)(2 - omega_1) P T grad C_p / theta
// with x = y - c_i the sender.  X and K are built between steps by the two
// stencil passes below from side fields each collision writes, so every
// population is exact (synchronous in time t) when it is used.
#pragma once

#include "lbm_helpers.cuh"

namespace lbm {

template <class Real, int I>
__device__ __forceinline__ void incoming_corr(const Real* __restrict__ side, long long N, long long sender,
                                              Real& cf, Real& cg) {
  constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
  const Real th = side[SP_THR * N + sender];
  Real kc = Real(0);
  if constexpr (cx != 0) kc += (cx > 0 ? side[(SP_K + 0) * N + sender] : -side[(SP_K + 0) * N + sender]);
  if constexpr (cy != 0) kc += (cy > 0 ? side[(SP_K + 1) * N + sender] : -side[(SP_K + 1) * N + sender]);
  if constexpr (cz != 0) kc += (cz > 0 ? side[(SP_K + 2) * N + sender] : -side[(SP_K + 2) * N + sender]);
  const Real w0 = Real(1) - th, w1 = Real(0.5) * th;
  const Real w = (cx ? w1 : w0) * (cy ? w1 : w0) * (cz ? w1 : w0);   // Eq. (weights)
  cg = w * kc;
  cf = Real(0);
  if constexpr (c2_of(I) == 1) {
    constexpr int a = cx ? 0 : (cy ? 1 : 2);
    constexpr int sg = cx + cy + cz;
    cf = (sg > 0 ? Real(0.5) : Real(-0.5)) * side[(SP_X + a) * N + sender];
  }
}

// Zeroth/first moments of the (corrected) deviations needed by the
// thermodynamic state (Eqs. densitya, auxua, f0momDensity, f1momMomentum,
// g0momTotalEnergy).
template <int M, class Real, class Store>
__device__ __forceinline__ void load_state_moments(const DevParams<Real>& p, const Store* __restrict__ pops,
                                                   const Real* __restrict__ side, int parity, const Nbr& nb,
                                                   long long n, Real (&rdev)[M], Real (&ja)[M][3],
                                                   Real& rho_dev, Real (&j)[3], Real& rhoE_dev) {
  const long long N = p.N;
#pragma unroll
  for (int a = 0; a < M; ++a) { rdev[a] = Real(0); ja[a][0] = ja[a][1] = ja[a][2] = Real(0); }
  rho_dev = Real(0); j[0] = j[1] = j[2] = Real(0); rhoE_dev = Real(0);
  static_for<0, Q>([&](auto I_) {
    constexpr int i = decltype(I_)::value;
    constexpr int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
    long long node; int slot;
    aa_read_loc(parity, nb, n, i, node, slot);
    Real cf = Real(0), cg = Real(0);
    if constexpr (i != 13) incoming_corr<Real, i>(side, N, nb.idx(-cx, -cy, -cz), cf, cg);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      const Real v = codec_load<Store, Real>(p, pops, (a * Q + slot) * N + node, a);
      rdev[a] += v;
      if (cx) ja[a][0] += cx * v;
      if (cy) ja[a][1] += cy * v;
      if (cz) ja[a][2] += cz * v;
    }
    const Real fv = codec_load<Store, Real>(p, pops, (M * Q + slot) * N + node, M) + cf;
    rho_dev += fv;
    if (cx) j[0] += cx * fv;
    if (cy) j[1] += cy * fv;
    if (cz) j[2] += cz * fv;
    rhoE_dev += codec_load<Store, Real>(p, pops, ((M + 1) * Q + slot) * N + node, M + 1) + cg;
  });
}

// Stencil pass 1 (after a collision): G_alpha = c_omega d_alpha Phi_alpha (the
// inner derivative of Eq. Xalpha) and K_alpha = s d_alpha C_p with s = c2 / theta;
// the sender's theta is copied for the receivers' weights.
template <class Real, class G>
__device__ __forceinline__ void grad_GK_node(const G& p, Real* __restrict__ side, long long n) {
  if (n >= p.N) return;
  const long long N = p.N;
  const Nbr nb = make_nbr(p, n);
  Real d[3] = {Real(0), Real(0), Real(0)}, dc[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
    if (i == 13) continue;
    const long long nn = nb.idx(cx, cy, cz);
    const Real w = iso_w<Real>(i);
    const Real cp = side[SP_CP * N + nn];
    if (cx) { d[0] += (cx * w) * side[(SP_PHI + 0) * N + nn]; dc[0] += (cx * w) * cp; }
    if (cy) { d[1] += (cy * w) * side[(SP_PHI + 1) * N + nn]; dc[1] += (cy * w) * cp; }
    if (cz) { d[2] += (cz * w) * side[(SP_PHI + 2) * N + nn]; dc[2] += (cz * w) * cp; }
  }
  const Real co = Real(3) * side[SP_COM * N + n], sv = Real(3) * side[SP_S * N + n];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    side[(SP_G + c) * N + n] = co * d[c];
    side[(SP_K + c) * N + n] = sv * dc[c];
  }
  side[SP_THR * N + n] = side[SP_TH * N + n];
}

// Stencil pass 2: X_alpha = -d_alpha G_alpha (Eq. Xalpha).
template <class Real, class G>
__device__ __forceinline__ void grad_X_node(const G& p, Real* __restrict__ side, long long n) {
  if (n >= p.N) return;
  const long long N = p.N;
  const Nbr nb = make_nbr(p, n);
  Real d[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
    if (i == 13) continue;
    const long long nn = nb.idx(cx, cy, cz);
    const Real w = iso_w<Real>(i);
    if (cx) d[0] += (cx * w) * side[(SP_G + 0) * N + nn];
    if (cy) d[1] += (cy * w) * side[(SP_G + 1) * N + nn];
    if (cz) d[2] += (cz * w) * side[(SP_G + 2) * N + nn];
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) side[(SP_X + c) * N + n] = Real(-3) * d[c];
}

template <class Real>
__global__ void __launch_bounds__(BLOCK_LIGHT)
grad_GK_kernel(const __grid_constant__ DevParams<Real> p, Real* __restrict__ side) {
  grad_GK_node<Real>(p, side, gtid());
}
template <class Real>
__global__ void __launch_bounds__(BLOCK_LIGHT)
grad_X_kernel(const __grid_constant__ DevParams<Real> p, Real* __restrict__ side) {
  grad_X_node<Real>(p, side, gtid());
}

}  // namespace lbm
