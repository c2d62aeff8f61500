// lbm_kernels.cuh -- CUDA kernels of the multicomponent D3Q27 step and their
// host launchers (templated; instantiated per species count in inst_m*.cu).
//
// One time step is three launches:
//   side_kernel     moments -> Phi_alpha, 1/omega - 1/2, C_p        (per node)
//   grad_kernel     G_alpha = (1/omega - 1/2) d_alpha Phi_alpha     (Eq. Xalpha, inner derivative)
//   collide_kernel  moments, closure, Stefan-Maxwell solve, species/f/g
//                   collisions, X_alpha = -d_alpha G_alpha and grad C_p
//                   from the neighbours' side fields; in-place AA write.
// The side fields are functions of time-t moments only, so every node sees
// synchronous non-local inputs, as the paper's operators require.
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

// ---------------------------------------------------------------------------
// Equilibrium initialisation (Eqs. 27eq, fixed, feq, gieq); natural layout.
// ---------------------------------------------------------------------------
template <int M, class Real, class Store>
__global__ void __launch_bounds__(BLOCK_LIGHT)
init_kernel(const DevParams<Real> p, const CodecParams cp, Store* __restrict__ pops,
            const double* __restrict__ Xin, const double* __restrict__ uin,
            const double* __restrict__ Tin, const double* __restrict__ Pin) {
  const long long n = gtid();
  if (n >= p.N) return;
  const long long N = p.N;
  Real X[M], u[3];
#pragma unroll
  for (int a = 0; a < M; ++a) X[a] = (Real)Xin[a * N + n];
#pragma unroll
  for (int c = 0; c < 3; ++c) u[c] = (Real)uin[c * N + n];
  Real T = (Real)Tin[n], P = (Real)Pin[n];
  Real m = Real(0);
#pragma unroll
  for (int a = 0; a < M; ++a) m += X[a] * p.mass[a];
  Real R = p.R_U / m;
  Real rho = P / (R * T);
  Real Y[M], Cv = Real(0), Cp = Real(0);
#pragma unroll
  for (int a = 0; a < M; ++a) {
    Y[a] = X[a] * p.mass[a] / m;
    Cv += Y[a] * p.Cv_a[a];
    Cp += Y[a] * p.Cp_a[a];
  }
  Real usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  Real rhoE = rho * (Cv * T + Real(0.5) * usq);
#pragma unroll
  for (int a = 0; a < M; ++a) {
    Real ra = Y[a] * rho, ze = p.R_a[a] * T;
    Triplet<Real> tx = psi_triplet(u[0], ze), ty = psi_triplet(u[1], ze), tz = psi_triplet(u[2], ze);
#pragma unroll
    for (int i = 0; i < Q; ++i)
      codec_store<Store, Real>(cp, pops, (a * Q + i) * N + n, a, i,
                               ra * tri(tx, cx_of(i)) * tri(ty, cy_of(i)) * tri(tz, cz_of(i)));
  }
  {
    Real ze = R * T;
    Triplet<Real> tx = psi_triplet(u[0], ze), ty = psi_triplet(u[1], ze), tz = psi_triplet(u[2], ze);
#pragma unroll
    for (int i = 0; i < Q; ++i)
      codec_store<Store, Real>(cp, pops, (M * Q + i) * N + n, M, i,
                               rho * tri(tx, cx_of(i)) * tri(ty, cy_of(i)) * tri(tz, cz_of(i)));
  }
  {
    Real theta = R * T, hk = Cp * T + Real(0.5) * usq;
    Real Mt[6];
    Mt[0] = hk * (P + rho * u[0] * u[0]) + P * u[0] * u[0];
    Mt[1] = hk * (P + rho * u[1] * u[1]) + P * u[1] * u[1];
    Mt[2] = hk * (P + rho * u[2] * u[2]) + P * u[2] * u[2];
    Mt[3] = hk * rho * u[0] * u[1] + P * u[0] * u[1];
    Mt[4] = hk * rho * u[0] * u[2] + P * u[0] * u[2];
    Mt[5] = hk * rho * u[1] * u[2] + P * u[1] * u[2];
    GCoef<Real> gc = g_coef(theta, rhoE, Mt);
    Real mt[3] = {hk * rho * u[0] / theta, hk * rho * u[1] / theta, hk * rho * u[2] / theta};
    static_for<0, Q>([&](auto I_) {
      constexpr int i = decltype(I_)::value;
      Real w = tri(gc.w, cx_of(i)) * tri(gc.w, cy_of(i)) * tri(gc.w, cz_of(i));
      Real v = w * (g_even_part<Real, i>(gc) + dotc<Real, i>(mt)) + g_BZ<Real, i>(gc);
      codec_store<Store, Real>(cp, pops, ((M + 1) * Q + i) * N + n, M + 1, i, v);
    });
  }
}

// ---------------------------------------------------------------------------
// Pass 1: node moments -> side fields Phi_alpha = j_alpha (1 - 3RT) - rho u_alpha^3
// (Eq. Xalpha), c_omega = 1/omega - 1/2 and C_p (its gradient gives
// sum_a H_a grad Y_a = T grad C_p for constant specific heats, Eq. corrFourier).
// Under strong coupling the slaved species' populations are not read.
// ---------------------------------------------------------------------------
template <int M, class Real, class Store>
__global__ void __launch_bounds__(BLOCK_LIGHT)
side_kernel(const DevParams<Real> p, const CodecParams cp, const Store* __restrict__ pops,
            Real* __restrict__ side, int parity) {
  const long long n = gtid();
  if (n >= p.N) return;
  const long long N = p.N;
  const Nbr nb = make_nbr(p, n);
  Real rho_a[M], jsum[3] = {Real(0), Real(0), Real(0)};
  Real rho = Real(0), j[3] = {Real(0), Real(0), Real(0)}, rhoE = Real(0);
#pragma unroll
  for (int a = 0; a < M; ++a) rho_a[a] = Real(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    long long node; int slot;
    aa_read_loc(parity, nb, n, i, node, slot);
    const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      if (!p.weak && a == p.slaved) continue;
      Real v = codec_load<Store, Real>(cp, pops, (a * Q + slot) * N + node, a, i);
      rho_a[a] += v;
      if (p.weak) { jsum[0] += cx * v; jsum[1] += cy * v; jsum[2] += cz * v; }
    }
    Real fv = codec_load<Store, Real>(cp, pops, (M * Q + slot) * N + node, M, i);
    rho += fv; j[0] += cx * fv; j[1] += cy * fv; j[2] += cz * fv;
    rhoE += codec_load<Store, Real>(cp, pops, ((M + 1) * Q + slot) * N + node, M + 1, i);
  }
  Thermo<M, Real> th;
  thermo_state<M, Real>(p, rho_a, jsum, rho, j, rhoE, th);
  Real a3 = Real(1) - Real(3) * th.R * th.T;
#pragma unroll
  for (int c = 0; c < 3; ++c) side[c * N + n] = j[c] * a3 - rho * th.u[c] * th.u[c] * th.u[c];
  side[3 * N + n] = Real(1) / th.omega - Real(0.5);
  side[4 * N + n] = th.Cp;
}

// Pass 2: G_alpha = c_omega d_alpha Phi_alpha (inner derivative of Eq. Xalpha).
template <class Real>
__global__ void __launch_bounds__(BLOCK_LIGHT)
grad_kernel(const DevParams<Real> p, Real* __restrict__ side) {
  const long long n = gtid();
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
    if (cx) d[0] += (cx * w) * side[0 * N + nn];
    if (cy) d[1] += (cy * w) * side[1 * N + nn];
    if (cz) d[2] += (cz * w) * side[2 * N + nn];
  }
  const Real co = side[3 * N + n];
#pragma unroll
  for (int c = 0; c < 3; ++c) side[(5 + c) * N + n] = co * Real(3) * d[c];
}

// ---------------------------------------------------------------------------
// Pass 3: the fused collide + stream of every lattice at one node.
// ---------------------------------------------------------------------------
template <int M, class Real, class Store, int PAR>
__global__ void __launch_bounds__(BLOCK)
collide_kernel(const DevParams<Real> p, const CodecParams cp, Store* __restrict__ pops,
               const Real* __restrict__ side, unsigned* __restrict__ err) {
  const long long n = gtid();
  if (n >= p.N) return;
  const long long N = p.N;
  const Nbr nb = make_nbr(p, n);

  // a1: load (AA addressing of this parity)
  Real k[M][Q], f[Q], g[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    long long node; int slot;
    aa_read_loc(PAR, nb, n, i, node, slot);
#pragma unroll
    for (int a = 0; a < M; ++a) k[a][i] = codec_load<Store, Real>(cp, pops, (a * Q + slot) * N + node, a, i);
    f[i] = codec_load<Store, Real>(cp, pops, (M * Q + slot) * N + node, M, i);
    g[i] = codec_load<Store, Real>(cp, pops, ((M + 1) * Q + slot) * N + node, M + 1, i);
  }

  // a2: moments (Eqs. densitya, auxua, f0momDensity, f1momMomentum, boldP, g0momTotalEnergy, q)
  Real rho_a[M], ja[M][3];
  Real rho = Real(0), j[3] = {Real(0), Real(0), Real(0)}, Pi[6] = {Real(0), Real(0), Real(0), Real(0), Real(0), Real(0)};
  Real rhoE = Real(0), q[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
  for (int a = 0; a < M; ++a) { rho_a[a] = Real(0); ja[a][0] = ja[a][1] = ja[a][2] = Real(0); }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      rho_a[a] += k[a][i];
      if (cx) ja[a][0] += cx * k[a][i];
      if (cy) ja[a][1] += cy * k[a][i];
      if (cz) ja[a][2] += cz * k[a][i];
    }
    rho += f[i];
    if (cx) { j[0] += cx * f[i]; Pi[0] += f[i]; }
    if (cy) { j[1] += cy * f[i]; Pi[1] += f[i]; }
    if (cz) { j[2] += cz * f[i]; Pi[2] += f[i]; }
    if (cx && cy) Pi[3] += (cx * cy) * f[i];
    if (cx && cz) Pi[4] += (cx * cz) * f[i];
    if (cy && cz) Pi[5] += (cy * cz) * f[i];
    rhoE += g[i];
    if (cx) q[0] += cx * g[i];
    if (cy) q[1] += cy * g[i];
    if (cz) q[2] += cz * g[i];
  }

  // a3: coupling + thermodynamics
  Real jsum[3] = {Real(0), Real(0), Real(0)};
  if (p.weak) {
#pragma unroll
    for (int a = 0; a < M; ++a) { jsum[0] += ja[a][0]; jsum[1] += ja[a][1]; jsum[2] += ja[a][2]; }
  }
  Thermo<M, Real> th;
  thermo_state<M, Real>(p, rho_a, jsum, rho, j, rhoE, th);
  if (!p.weak) {
    // Eq. (uMATCH): slaved species momentum = mixture momentum deficit.
    Real o[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
    for (int a = 0; a < M; ++a)
      if (a != p.slaved) { o[0] += ja[a][0]; o[1] += ja[a][1]; o[2] += ja[a][2]; }
#pragma unroll
    for (int a = 0; a < M; ++a)
      if (a == p.slaved) { ja[a][0] = j[0] - o[0]; ja[a][1] = j[1] - o[1]; ja[a][2] = j[2] - o[2]; }
  }
  if (!(rho > Real(0)) || !(th.T > Real(0)) || !(th.rho_sp > Real(0))) atomicOr(err, 1u);
  const Real om = th.omega;
  const Real om1 = omega1_of<M, Real>(p, th);

  // a5: non-local inputs from the neighbours' side fields.
  Real dCp[3] = {Real(0), Real(0), Real(0)}, Xc[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
    if (i == 13) continue;
    const long long nn = nb.idx(cx, cy, cz);
    const Real w = iso_w<Real>(i);
    const Real cpn = side[4 * N + nn];
    if (cx) { dCp[0] += (cx * w) * cpn; Xc[0] += (cx * w) * side[5 * N + nn]; }
    if (cy) { dCp[1] += (cy * w) * cpn; Xc[1] += (cy * w) * side[6 * N + nn]; }
    if (cz) { dCp[2] += (cz * w) * cpn; Xc[2] += (cz * w) * side[7 * N + nn]; }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) { dCp[c] *= Real(3); Xc[c] *= Real(-3); }

  // a4, a6: relaxation times (Eqs. tauab, tau) and the Stefan-Maxwell fluxes.
  Real itab[M][M];
  const Real tm = p.R_U * th.T * th.m;
#pragma unroll
  for (int a = 0; a < M; ++a)
#pragma unroll
    for (int b = 0; b < M; ++b) itab[a][b] = tm * p.Cab[a][b];
  Real J[M][3];
  sm_solve<M, Real>(p, th, itab, ja, J);
  Real V[M][3], beta[M];
#pragma unroll
  for (int a = 0; a < M; ++a) {
    const bool ok = th.rho_a[a] > p.rho_eps * th.rho_sp;
    const Real ir = ok ? Real(1) / th.rho_a[a] : Real(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) V[a][c] = J[a][c] * ir;
    Real it = Real(0);
#pragma unroll
    for (int b = 0; b < M; ++b) it += itab[a][b] * th.Y[b];
    beta[a] = it / (Real(2) + it);                      // dt / (2 tau_a + dt)
  }

  // a7: species collision, Eqs. (SMlbm), (fstar1):
  //   k' = (1 - 2 beta_a) k + 2 beta_a f^eq_a + (beta_a - 1) F_a,
  //   F_ai = sum_b kap_ab [Psi_i(u, R_b T) - Psi_i(u + V_b, R_b T)], kap_ab = Y_a rho_b / tau_ab.
  // The per-axis differences of the triplets are formed exactly:
  //   Psi_0(xi) - Psi_0(xi + V) = V (2 xi + V) = e,  Psi_{+-1}: -e/2 -+ V/2.
  Triplet<Real> te[M][3], td[M][3];
#pragma unroll
  for (int b = 0; b < M; ++b) {
    const Real ze = p.R_a[b] * th.T;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      te[b][c] = psi_triplet(th.u_sp[c], ze);
      const Real v = V[b][c];
      const Real e = v * (Real(2) * th.u_sp[c] + v);
      td[b][c].z = e;
      td[b][c].p = Real(-0.5) * (e + v);
      td[b][c].m = Real(-0.5) * (e - v);
    }
  }
  Real kap[M][M];
#pragma unroll
  for (int a = 0; a < M; ++a)
#pragma unroll
    for (int b = 0; b < M; ++b) kap[a][b] = th.Y[a] * th.rho_a[b] * itab[a][b];

  // a8: momentum lattice, Eqs. (feq), (fwithcorrection), (Ai).
  const Real thetaf = th.R * th.T;
  const Triplet<Real> fx = psi_triplet(th.u[0], thetaf), fy = psi_triplet(th.u[1], thetaf),
                      fz = psi_triplet(th.u[2], thetaf);

  // a9: energy lattice.  Since G is affine in its vector argument,
  //   g' = (1 - omega) g + omega G(q^eq) + w_i c_i . K / theta,
  //   K = (omega - omega_1)(q^b - q^eq) + omega_1 rho sum_a H_a Y_a V_a
  //       + (1/2)(2 - omega_1) P sum_a H_a grad Y_a,
  // which is Eq. (g) with Eqs. (gstareq1mom), (interdiffusion), (corrFourier)
  // written without the 1/(omega - omega_1) factors.
  const Real P = th.P, T = th.T;
  const Real hk = th.Cp * T + Real(0.5) * th.usq;
  const Real* u = th.u;
  Real Peq[6];
  Peq[0] = P + rho * u[0] * u[0]; Peq[1] = P + rho * u[1] * u[1]; Peq[2] = P + rho * u[2] * u[2];
  Peq[3] = rho * u[0] * u[1]; Peq[4] = rho * u[0] * u[2]; Peq[5] = rho * u[1] * u[2];
  Real Mt[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) Mt[s] = hk * Peq[s];
  Mt[0] += P * u[0] * u[0]; Mt[1] += P * u[1] * u[1]; Mt[2] += P * u[2] * u[2];
  Mt[3] += P * u[0] * u[1]; Mt[4] += P * u[0] * u[2]; Mt[5] += P * u[1] * u[2];
  const GCoef<Real> gc = g_coef(thetaf, rhoE, Mt);
  Real dP[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) dP[s] = Pi[s] - Peq[s];
  Real qeq[3] = {hk * j[0], hk * j[1], hk * j[2]};
  Real qb[3];
  qb[0] = q[0] - (u[0] * dP[0] + u[1] * dP[3] + u[2] * dP[4]);
  qb[1] = q[1] - (u[0] * dP[3] + u[1] * dP[1] + u[2] * dP[5]);
  qb[2] = q[2] - (u[0] * dP[4] + u[1] * dP[5] + u[2] * dP[2]);
  Real hyv[3] = {Real(0), Real(0), Real(0)};
  const Real rY = p.weak ? rho / th.rho_sp : Real(1);   // rho Y_a = rY * rho_a
#pragma unroll
  for (int a = 0; a < M; ++a) {
    const Real s = p.Cp_a[a] * th.rho_a[a];
#pragma unroll
    for (int c = 0; c < 3; ++c) hyv[c] += s * V[a][c];
  }
  const Real c1 = om1 * T * rY, c2 = Real(0.5) * (Real(2) - om1) * P * T, dw = om - om1;
  const Real inv_theta = Real(1) / thetaf;
  Real mvec[3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    mvec[c] = (om * qeq[c] + dw * (qb[c] - qeq[c]) + c1 * hyv[c] + c2 * dCp[c]) * inv_theta;

  // a10: collide every direction and store with the AA write addressing.
  // The rest direction (i = 13) is done last: its equilibria and F_a,13 are
  // the conservation remainders (rho_a, rho, rho E minus the other 26),
  // identical to the product forms in exact arithmetic; in finite precision
  // this keeps the per-step zeroth moments free of the systematic bias that
  // sum_i w_i(theta) != 1 would otherwise inject every step.
  const Real one_m_om = Real(1) - om;
  Real s_keq[M], s_F[M], s_feq = Real(0), s_geq = Real(0);
#pragma unroll
  for (int a = 0; a < M; ++a) { s_keq[a] = Real(0); s_F[a] = Real(0); }
  static_for<0, Q>([&](auto I_) {
    constexpr int i = decltype(I_)::value;
    if constexpr (i != 13) {
      constexpr int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
      long long node; int slot;
      aa_write_loc(PAR, nb, n, i, node, slot);
      // species
      Real Dif[M];
#pragma unroll
      for (int b = 0; b < M; ++b) {
        const Real ex = tri(te[b][0], cx), ey = tri(te[b][1], cy), ez = tri(te[b][2], cz);
        const Real dx = tri(td[b][0], cx), dy = tri(td[b][1], cy), dz = tri(td[b][2], cz);
        // a_x a_y a_z - s_x s_y s_z with s = a - d
        const Real sx = ex - dx, sy = ey - dy;
        Dif[b] = dx * ey * ez + sx * dy * ez + sx * sy * dz;
      }
#pragma unroll
      for (int a = 0; a < M; ++a) {
        Real F = Real(0);
#pragma unroll
        for (int b = 0; b < M; ++b) F += kap[a][b] * Dif[b];
        const Real feq = th.rho_a[a] * tri(te[a][0], cx) * tri(te[a][1], cy) * tri(te[a][2], cz);
        s_keq[a] += feq; s_F[a] += F;
        const Real kn = k[a][i] + Real(2) * beta[a] * (feq - k[a][i]) + (beta[a] - Real(1)) * F;
        codec_store<Store, Real>(cp, pops, (a * Q + slot) * N + node, a, i, kn);
      }
      // momentum lattice
      {
        const Real feq = rho * tri(fx, cx) * tri(fy, cy) * tri(fz, cz);
        s_feq += feq;
        Real fn = one_m_om * f[i] + om * feq;
        if constexpr (c2_of(i) == 1) fn += Real(0.5) * dotc<Real, i>(Xc);
        codec_store<Store, Real>(cp, pops, (M * Q + slot) * N + node, M, i, fn);
      }
      // energy lattice
      {
        const Real w = tri(gc.w, cx) * tri(gc.w, cy) * tri(gc.w, cz);
        const Real geq = w * g_even_part<Real, i>(gc) + g_BZ<Real, i>(gc);
        s_geq += geq;
        const Real gn = one_m_om * g[i] + om * geq + w * dotc<Real, i>(mvec);
        codec_store<Store, Real>(cp, pops, ((M + 1) * Q + slot) * N + node, M + 1, i, gn);
      }
    }
  });
  {
    constexpr int i = 13;
    long long node; int slot;
    aa_write_loc(PAR, nb, n, i, node, slot);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      const Real feq = th.rho_a[a] - s_keq[a];
      const Real kn = k[a][i] + Real(2) * beta[a] * (feq - k[a][i]) - (beta[a] - Real(1)) * s_F[a];
      codec_store<Store, Real>(cp, pops, (a * Q + slot) * N + node, a, i, kn);
    }
    codec_store<Store, Real>(cp, pops, (M * Q + slot) * N + node, M, i, one_m_om * f[i] + om * (rho - s_feq));
    codec_store<Store, Real>(cp, pops, ((M + 1) * Q + slot) * N + node, M + 1, i,
                             one_m_om * g[i] + om * (rhoE - s_geq));
  }
}

// ---------------------------------------------------------------------------
// Observables (get_moments): rho, u, T, P, X_a, Y_a, V_a.
// ---------------------------------------------------------------------------
template <int M, class Real, class Store>
__global__ void __launch_bounds__(BLOCK)
moments_kernel(const DevParams<Real> p, const CodecParams cp, const Store* __restrict__ pops,
               int parity, double* __restrict__ out) {
  const long long n = gtid();
  if (n >= p.N) return;
  const long long N = p.N;
  const Nbr nb = make_nbr(p, n);
  Real rho_a[M], ja[M][3], rho = Real(0), j[3] = {Real(0), Real(0), Real(0)}, rhoE = Real(0);
#pragma unroll
  for (int a = 0; a < M; ++a) { rho_a[a] = Real(0); ja[a][0] = ja[a][1] = ja[a][2] = Real(0); }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    long long node; int slot;
    aa_read_loc(parity, nb, n, i, node, slot);
    const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      Real v = codec_load<Store, Real>(cp, pops, (a * Q + slot) * N + node, a, i);
      rho_a[a] += v; ja[a][0] += cx * v; ja[a][1] += cy * v; ja[a][2] += cz * v;
    }
    Real fv = codec_load<Store, Real>(cp, pops, (M * Q + slot) * N + node, M, i);
    rho += fv; j[0] += cx * fv; j[1] += cy * fv; j[2] += cz * fv;
    rhoE += codec_load<Store, Real>(cp, pops, ((M + 1) * Q + slot) * N + node, M + 1, i);
  }
  Real jsum[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
  for (int a = 0; a < M; ++a) { jsum[0] += ja[a][0]; jsum[1] += ja[a][1]; jsum[2] += ja[a][2]; }
  Thermo<M, Real> th;
  thermo_state<M, Real>(p, rho_a, jsum, rho, j, rhoE, th);
  if (!p.weak) {
    Real o[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
    for (int a = 0; a < M; ++a)
      if (a != p.slaved) { o[0] += ja[a][0]; o[1] += ja[a][1]; o[2] += ja[a][2]; }
#pragma unroll
    for (int a = 0; a < M; ++a)
      if (a == p.slaved) { ja[a][0] = j[0] - o[0]; ja[a][1] = j[1] - o[1]; ja[a][2] = j[2] - o[2]; }
  }
  Real itab[M][M];
  const Real tm = p.R_U * th.T * th.m;
#pragma unroll
  for (int a = 0; a < M; ++a)
#pragma unroll
    for (int b = 0; b < M; ++b) itab[a][b] = tm * p.Cab[a][b];
  Real J[M][3];
  sm_solve<M, Real>(p, th, itab, ja, J);
  out[0 * N + n] = (double)rho;
  out[1 * N + n] = (double)th.u[0];
  out[2 * N + n] = (double)th.u[1];
  out[3 * N + n] = (double)th.u[2];
  out[4 * N + n] = (double)th.T;
  out[5 * N + n] = (double)th.P;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    out[(6 + a) * N + n] = (double)(th.m * th.Y[a] * p.inv_mass[a]);
    out[(6 + M + a) * N + n] = (double)th.Y[a];
    const bool ok = th.rho_a[a] > p.rho_eps * th.rho_sp;
    const Real ir = ok ? Real(1) / th.rho_a[a] : Real(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) out[(6 + 2 * M + 3 * a + c) * N + n] = (double)(J[a][c] * ir);
  }
}

// Natural-layout copy of the logical populations (checkpoint interface).
template <int M, class Real, class Store>
__global__ void __launch_bounds__(BLOCK_LIGHT)
get_pops_kernel(const DevParams<Real> p, const CodecParams cp, const Store* __restrict__ pops,
                int parity, double* __restrict__ out) {
  const long long n = gtid();
  if (n >= p.N) return;
  const long long N = p.N;
  const Nbr nb = make_nbr(p, n);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    long long node; int slot;
    aa_read_loc(parity, nb, n, i, node, slot);
    for (int L = 0; L < M + 2; ++L)
      out[(L * Q + i) * N + n] = (double)codec_load<Store, Real>(cp, pops, (L * Q + slot) * N + node, L, i);
  }
}

template <int M, class Real, class Store>
__global__ void __launch_bounds__(BLOCK_LIGHT)
set_pops_kernel(const DevParams<Real> p, const CodecParams cp, Store* __restrict__ pops,
                int parity, const double* __restrict__ in) {
  const long long n = gtid();
  if (n >= p.N) return;
  const long long N = p.N;
  const Nbr nb = make_nbr(p, n);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    long long node; int slot;
    aa_read_loc(parity, nb, n, i, node, slot);
    for (int L = 0; L < M + 2; ++L)
      codec_store<Store, Real>(cp, pops, (L * Q + slot) * N + node, L, i, (Real)in[(L * Q + i) * N + n]);
  }
}

// ---------------------------------------------------------------------------
// a12: FP64 conservation sums.  Pass 1: per-block partials (warp shuffles,
// then shared memory); pass 2: one block sums the partials in a fixed order.
// ---------------------------------------------------------------------------
constexpr int DIAG_BLOCK = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <int M, class Real, class Store>
__global__ void __launch_bounds__(DIAG_BLOCK)
diag_partial_kernel(const DevParams<Real> p, const CodecParams cp, const Store* __restrict__ pops,
                    int parity, double* __restrict__ partials) {
  constexpr int NV = M + 5;
  __shared__ double red[DIAG_BLOCK / 32][NV];
  const long long n = gtid();
  double v[NV];
#pragma unroll
  for (int s = 0; s < NV; ++s) v[s] = 0.0;
  if (n < p.N) {
    const long long N = p.N;
    const Nbr nb = make_nbr(p, n);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      long long node; int slot;
      aa_read_loc(parity, nb, n, i, node, slot);
#pragma unroll
      for (int a = 0; a < M; ++a) v[a] += (double)codec_load<Store, Real>(cp, pops, (a * Q + slot) * N + node, a, i);
      double fv = (double)codec_load<Store, Real>(cp, pops, (M * Q + slot) * N + node, M, i);
      v[M] += fv;
      v[M + 1] += cx_of(i) * fv; v[M + 2] += cy_of(i) * fv; v[M + 3] += cz_of(i) * fv;
      v[M + 4] += (double)codec_load<Store, Real>(cp, pops, ((M + 1) * Q + slot) * N + node, M + 1, i);
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NV; ++s) {
    double t = warp_sum(v[s]);
    if (lane == 0) red[wid][s] = t;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double t = 0.0;
    for (int w = 0; w < DIAG_BLOCK / 32; ++w) t += red[w][threadIdx.x];
    partials[(long long)blockIdx.x * NV + threadIdx.x] = t;
  }
}

static __global__ void __launch_bounds__(DIAG_BLOCK)
diag_final_kernel(const double* __restrict__ partials, int nblocks, int nv, double* __restrict__ sums) {
  __shared__ double sh[DIAG_BLOCK];
  for (int s = 0; s < nv; ++s) {
    double t = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += DIAG_BLOCK) t += partials[(long long)b * nv + s];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int w = DIAG_BLOCK / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) sums[s] = sh[0];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
inline unsigned grid_for(long long N, int block) { return (unsigned)((N + block - 1) / block); }

template <int M, class Real, class Store>
struct Launch {
  static const DevParams<Real>& P(const LaunchCtx& c) {
    if constexpr (sizeof(Real) == 8) return *c.p64; else return *c.p32;
  }
  static cudaError_t init(const LaunchCtx& c, const double* X, const double* u, const double* T,
                          const double* Pr) {
    init_kernel<M, Real, Store><<<grid_for(c.N, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(
        P(c), *c.codec, (Store*)c.pops, X, u, T, Pr);
    return cudaGetLastError();
  }
  static cudaError_t step(const LaunchCtx& c, int parity) {
    Real* side = (Real*)c.side;
    if (c.ev) cudaEventRecord(c.ev[0], c.stream);
    side_kernel<M, Real, Store><<<grid_for(c.N, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(
        P(c), *c.codec, (const Store*)c.pops, side, parity);
    if (c.ev) cudaEventRecord(c.ev[1], c.stream);
    grad_kernel<Real><<<grid_for(c.N, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(P(c), side);
    if (c.ev) cudaEventRecord(c.ev[2], c.stream);
    if (parity == 0)
      collide_kernel<M, Real, Store, 0><<<grid_for(c.N, BLOCK), BLOCK, 0, c.stream>>>(
          P(c), *c.codec, (Store*)c.pops, side, c.err);
    else
      collide_kernel<M, Real, Store, 1><<<grid_for(c.N, BLOCK), BLOCK, 0, c.stream>>>(
          P(c), *c.codec, (Store*)c.pops, side, c.err);
    if (c.ev) cudaEventRecord(c.ev[3], c.stream);
    return cudaGetLastError();
  }
  static cudaError_t moments(const LaunchCtx& c, int parity, double* out) {
    moments_kernel<M, Real, Store><<<grid_for(c.N, BLOCK), BLOCK, 0, c.stream>>>(
        P(c), *c.codec, (const Store*)c.pops, parity, out);
    return cudaGetLastError();
  }
  static cudaError_t get_pops(const LaunchCtx& c, int parity, double* out) {
    get_pops_kernel<M, Real, Store><<<grid_for(c.N, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(
        P(c), *c.codec, (const Store*)c.pops, parity, out);
    return cudaGetLastError();
  }
  static cudaError_t set_pops(const LaunchCtx& c, int parity, const double* in) {
    set_pops_kernel<M, Real, Store><<<grid_for(c.N, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(
        P(c), *c.codec, (Store*)c.pops, parity, in);
    return cudaGetLastError();
  }
  static cudaError_t diag(const LaunchCtx& c, int parity, double* d_sums) {
    const unsigned nb = grid_for(c.N, DIAG_BLOCK);
    diag_partial_kernel<M, Real, Store><<<nb, DIAG_BLOCK, 0, c.stream>>>(
        P(c), *c.codec, (const Store*)c.pops, parity, c.partials);
    diag_final_kernel<<<1, DIAG_BLOCK, 0, c.stream>>>(c.partials, (int)nb, M + 5, d_sums);
    return cudaGetLastError();
  }
  static KernelSet make() {
    KernelSet k;
    k.init = &init; k.step = &step; k.moments = &moments; k.get_pops = &get_pops;
    k.set_pops = &set_pops; k.diag = &diag;
    k.launches_per_step = 3;
    return k;
  }
};

}  // namespace lbm
