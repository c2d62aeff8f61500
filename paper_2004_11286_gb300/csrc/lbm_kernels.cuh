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

// ---------------------------------------------------------------------------
// Equilibrium initialisation (Eqs. 27eq, fixed, feq, gieq), evaluated in FP64
// as full populations and stored as deviations from the base table.
// ---------------------------------------------------------------------------
template <int M, class Store>
__global__ void __launch_bounds__(BLOCK_LIGHT)
init_kernel(const DevParams<double> p, Store* __restrict__ pops, const double* __restrict__ base,
            const double* __restrict__ Xin, const double* __restrict__ uin,
            const double* __restrict__ Tin, const double* __restrict__ Pin) {
  const long long n = gtid();
  if (n >= p.N) return;
  const long long N = p.N;
  double X[M], u[3];
#pragma unroll
  for (int a = 0; a < M; ++a) X[a] = Xin[a * N + n];
#pragma unroll
  for (int c = 0; c < 3; ++c) u[c] = uin[c * N + n];
  const double T = Tin[n], P = Pin[n];
  double m = 0.0;
#pragma unroll
  for (int a = 0; a < M; ++a) m += X[a] * p.mass[a];
  const double R = p.R_U / m;
  const double rho = P / (R * T);
  double Y[M], Cv = 0.0, Cp = 0.0;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    Y[a] = X[a] * p.mass[a] / m;
    Cv += Y[a] * p.Cv_a[a];
    Cp += Y[a] * p.Cp_a[a];
  }
  const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const double rhoE = rho * (Cv * T + 0.5 * usq);
#pragma unroll
  for (int a = 0; a < M; ++a) {
    const double ra = Y[a] * rho, ze = p.R_a[a] * T;
    const Triplet<double> tx = psi_triplet(u[0], ze), ty = psi_triplet(u[1], ze), tz = psi_triplet(u[2], ze);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double v = ra * tri(tx, cx_of(i)) * tri(ty, cy_of(i)) * tri(tz, cz_of(i));
      codec_store<Store, double>(p, pops, (a * Q + i) * N + n, a, v - base[a * Q + i]);
    }
  }
  {
    const double ze = R * T;
    const Triplet<double> tx = psi_triplet(u[0], ze), ty = psi_triplet(u[1], ze), tz = psi_triplet(u[2], ze);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double v = rho * tri(tx, cx_of(i)) * tri(ty, cy_of(i)) * tri(tz, cz_of(i));
      codec_store<Store, double>(p, pops, (M * Q + i) * N + n, M, v - base[M * Q + i]);
    }
  }
  {
    const double theta = R * T, hk = Cp * T + 0.5 * usq;
    double Mt[6];
    Mt[0] = hk * (P + rho * u[0] * u[0]) + P * u[0] * u[0];
    Mt[1] = hk * (P + rho * u[1] * u[1]) + P * u[1] * u[1];
    Mt[2] = hk * (P + rho * u[2] * u[2]) + P * u[2] * u[2];
    Mt[3] = hk * rho * u[0] * u[1] + P * u[0] * u[1];
    Mt[4] = hk * rho * u[0] * u[2] + P * u[0] * u[2];
    Mt[5] = hk * rho * u[1] * u[2] + P * u[1] * u[2];
    const GCoef<double> gc = g_coef(theta, rhoE, Mt);
    const double mt[3] = {hk * rho * u[0] / theta, hk * rho * u[1] / theta, hk * rho * u[2] / theta};
    static_for<0, Q>([&](auto I_) {
      constexpr int i = decltype(I_)::value;
      const double w = tri(gc.w, cx_of(i)) * tri(gc.w, cy_of(i)) * tri(gc.w, cz_of(i));
      const double v = w * (g_even_part<double, i>(gc) + dotc<double, i>(mt)) + g_BZ<double, i>(gc);
      codec_store<Store, double>(p, pops, ((M + 1) * Q + i) * N + n, M + 1, v - base[(M + 1) * Q + i]);
    });
  }
}

// Zeroth/first moments of the stored deviations needed by the thermodynamic
// state (Eqs. densitya, auxua, f0momDensity, f1momMomentum, g0momTotalEnergy).
template <int M, class Real, class Store>
__device__ __forceinline__ void load_state_moments(const DevParams<Real>& p, const Store* __restrict__ pops,
                                                   int parity, const Nbr& nb, long long n, bool skip_slaved,
                                                   Real (&rdev)[M], Real (&ja)[M][3], Real& rho_dev,
                                                   Real (&j)[3], Real& rhoE_dev) {
  const long long N = p.N;
#pragma unroll
  for (int a = 0; a < M; ++a) { rdev[a] = Real(0); ja[a][0] = ja[a][1] = ja[a][2] = Real(0); }
  rho_dev = Real(0); j[0] = j[1] = j[2] = Real(0); rhoE_dev = Real(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    long long node; int slot;
    aa_read_loc(parity, nb, n, i, node, slot);
    const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      if (skip_slaved && a == p.slaved) continue;
      const Real v = codec_load<Store, Real>(p, pops, (a * Q + slot) * N + node, a);
      rdev[a] += v;
      if (cx) ja[a][0] += cx * v;
      if (cy) ja[a][1] += cy * v;
      if (cz) ja[a][2] += cz * v;
    }
    const Real fv = codec_load<Store, Real>(p, pops, (M * Q + slot) * N + node, M);
    rho_dev += fv;
    if (cx) j[0] += cx * fv;
    if (cy) j[1] += cy * fv;
    if (cz) j[2] += cz * fv;
    rhoE_dev += codec_load<Store, Real>(p, pops, ((M + 1) * Q + slot) * N + node, M + 1);
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
side_kernel(const DevParams<Real> p, const Store* __restrict__ pops, Real* __restrict__ side, int parity) {
  const long long n = gtid();
  if (n >= p.N) return;
  const long long N = p.N;
  const Nbr nb = make_nbr(p, n);
  Real rdev[M], ja[M][3], rho_dev, j[3], rhoE_dev;
  load_state_moments<M, Real, Store>(p, pops, parity, nb, n, !p.weak, rdev, ja, rho_dev, j, rhoE_dev);
  Real jsum[3] = {Real(0), Real(0), Real(0)};
  if (p.weak) {
#pragma unroll
    for (int a = 0; a < M; ++a) { jsum[0] += ja[a][0]; jsum[1] += ja[a][1]; jsum[2] += ja[a][2]; }
  }
  Thermo<M, Real> th;
  thermo_state<M, Real>(p, rdev, jsum, rho_dev, j, rhoE_dev, th);
  const Real a3 = Real(1) - Real(3) * th.theta;
#pragma unroll
  for (int c = 0; c < 3; ++c) side[c * N + n] = j[c] * a3 - th.rho * th.u[c] * th.u[c] * th.u[c];
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
// Pass 3: the fused collide + stream of every lattice at one node, written
// for the stored deviations d = f - b of the populations from the reference
// rest equilibria (the update is affine, so d' = f' - b exactly):
//   species (Eq. SMlbm):  d' = d + 2 beta_a (e_a - d) + (beta_a - 1) F_a
//   f (Eq. fwithcorrection): d' = d + omega (e - d) + A_i . X
//   g (Eq. g):            d' = d + omega (e_g - d) + w_i(theta) c_i . K / theta
// with e = f^eq - b formed from deviation quantities (no O(f) cancellation).
// ---------------------------------------------------------------------------
template <int M, class Real, class Store, int PAR>
__global__ void __launch_bounds__(BLOCK)
collide_kernel(const DevParams<Real> p, Store* __restrict__ pops, const Real* __restrict__ side,
               unsigned* __restrict__ err) {
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
    for (int a = 0; a < M; ++a) k[a][i] = codec_load<Store, Real>(p, pops, (a * Q + slot) * N + node, a);
    f[i] = codec_load<Store, Real>(p, pops, (M * Q + slot) * N + node, M);
    g[i] = codec_load<Store, Real>(p, pops, ((M + 1) * Q + slot) * N + node, M + 1);
  }

  // a2: moments of the deviations (the reference tables have zero first and
  // off-diagonal second moments)
  Real rdev[M], ja[M][3];
  Real rho_dev = Real(0), j[3] = {Real(0), Real(0), Real(0)};
  Real S[6] = {Real(0), Real(0), Real(0), Real(0), Real(0), Real(0)};
  Real rhoE_dev = Real(0), q[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
  for (int a = 0; a < M; ++a) { rdev[a] = Real(0); ja[a][0] = ja[a][1] = ja[a][2] = Real(0); }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      rdev[a] += k[a][i];
      if (cx) ja[a][0] += cx * k[a][i];
      if (cy) ja[a][1] += cy * k[a][i];
      if (cz) ja[a][2] += cz * k[a][i];
    }
    rho_dev += f[i];
    if (cx) { j[0] += cx * f[i]; S[0] += f[i]; }
    if (cy) { j[1] += cy * f[i]; S[1] += f[i]; }
    if (cz) { j[2] += cz * f[i]; S[2] += f[i]; }
    if (cx && cy) S[3] += (cx * cy) * f[i];
    if (cx && cz) S[4] += (cx * cz) * f[i];
    if (cy && cz) S[5] += (cy * cz) * f[i];
    rhoE_dev += g[i];
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
  thermo_state<M, Real>(p, rdev, jsum, rho_dev, j, rhoE_dev, th);
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
  const Real rho = th.rho;
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

  // a7: species.  Equilibrium deviation e_ai = rho_a (Psi_i - W_i) + (rho_a - RL_a) W_i
  // with W_i the reference weights; F_ai = sum_b kap_ab [Psi_i(u, R_b T) - Psi_i(u + V_b, R_b T)]
  // (Eq. fstar1), kap_ab = Y_a rho_b / tau_ab, from exact per-axis differences
  //   Psi_0(xi) - Psi_0(xi + V) = V (2 xi + V) = e,  Psi_{+-1}: -e/2 -+ V/2.
  PFDev<Real> sp[M];
  Triplet<Real> td[M][3];
#pragma unroll
  for (int b = 0; b < M; ++b) {
    pf_dev<Real>(sp[b], th.u_sp, p.R_a[b] * p.Tr, p.R_a[b] * th.dT);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
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
  PFDev<Real> fp;
  pf_dev<Real>(fp, th.u, p.thr, th.dtheta);

  // a9: energy lattice.  With N = R^eq - rho E theta I, Eqs. (geq2mom),
  // (eosIdealGas) and Mayer give N = P theta I + rho (h + theta) u u
  // (h = H + u^2/2), so the ansatz of Eqs. (gansatz)-(RcorrectionPrime) reads
  //   G_i(m) = w_i(theta) [E_i + m . c_i / theta] + B_i . Z,
  //   E_i = rho E - 3P/2 + rho |c_i|^2 / 2 + Gc ((u . c_i)^2 / theta - u^2),
  //   Z_a = (1 - 3 theta) P / 2 + (1 - 3 theta) Gc u_a^2,  Gc = rho (h + theta) / (2 theta),
  // whose deviation from the reference rest state is again a small quantity.
  // G is affine in m, so Eq. (g) becomes g' = (1 - omega) g + omega G(q^eq)
  // + w_i c_i . K / theta with K = (omega - omega_1)(q^b - q^eq)
  // + omega_1 rho sum_a H_a Y_a V_a + (1/2)(2 - omega_1) P sum_a H_a grad Y_a
  // (Eqs. gstareq1mom, interdiffusion, corrFourier without their 1/(omega - omega_1)).
  const Real theta = th.theta, thr = p.thr, dth = th.dtheta;
  const Real P = th.P, T = th.T;
  const Real hk = th.Cp * T + Real(0.5) * th.usq;
  const Real inv_theta = Real(1) / theta;
  const Real Gc = rho * (hk + theta) * Real(0.5) * inv_theta;
  const Real* u = th.u;
  Triplet<Real> gw, gwr, gdw;
  gw.z = Real(1) - theta; gw.p = Real(0.5) * theta; gw.m = gw.p;          // Eq. (w0)
  gwr.z = Real(1) - thr; gwr.p = Real(0.5) * thr; gwr.m = gwr.p;
  gdw.z = -dth; gdw.p = Real(0.5) * dth; gdw.m = gdw.p;
  const Real E0 = (p.RL[M + 1] + rhoE_dev) - Real(1.5) * P - Gc * th.usq;
  const Real dE0 = rhoE_dev - Real(1.5) * th.dP - Gc * th.usq;
  Real dZ[3];
  {
    const Real z1 = Real(1) - Real(3) * theta;
    const Real zb = Real(0.5) * (z1 * th.dP - Real(3) * dth * p.Pr);
#pragma unroll
    for (int c = 0; c < 3; ++c) dZ[c] = zb + z1 * Gc * u[c] * u[c];
  }
  Real dP6[6];   // Pi - P^eq from deviations
  dP6[0] = p.cPi + S[0] - th.dP - rho * u[0] * u[0];
  dP6[1] = p.cPi + S[1] - th.dP - rho * u[1] * u[1];
  dP6[2] = p.cPi + S[2] - th.dP - rho * u[2] * u[2];
  dP6[3] = S[3] - rho * u[0] * u[1];
  dP6[4] = S[4] - rho * u[0] * u[2];
  dP6[5] = S[5] - rho * u[1] * u[2];
  Real qeq[3] = {hk * j[0], hk * j[1], hk * j[2]};
  Real qb[3];
  qb[0] = q[0] - (u[0] * dP6[0] + u[1] * dP6[3] + u[2] * dP6[4]);
  qb[1] = q[1] - (u[0] * dP6[3] + u[1] * dP6[1] + u[2] * dP6[5]);
  qb[2] = q[2] - (u[0] * dP6[4] + u[1] * dP6[5] + u[2] * dP6[2]);
  Real hyv[3] = {Real(0), Real(0), Real(0)};
  const Real rY = p.weak ? rho / th.rho_sp : Real(1);   // rho Y_a = rY * rho_a
#pragma unroll
  for (int a = 0; a < M; ++a) {
    const Real s = p.Cp_a[a] * th.rho_a[a];
#pragma unroll
    for (int c = 0; c < 3; ++c) hyv[c] += s * V[a][c];
  }
  const Real c1 = om1 * T * rY, c2 = Real(0.5) * (Real(2) - om1) * P * T, dw = om - om1;
  Real mvec[3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    mvec[c] = (om * qeq[c] + dw * (qb[c] - qeq[c]) + c1 * hyv[c] + c2 * dCp[c]) * inv_theta;

  // a10: collide every direction and store with the AA write addressing.
  // The rest direction (i = 13) is done last: its equilibrium deviations and
  // F_a,13 are the conservation remainders, identical to the product forms in
  // exact arithmetic, so the zeroth moments carry no per-step rounding bias.
  Real s_e[M], s_F[M], s_f = Real(0), s_g = Real(0);
#pragma unroll
  for (int a = 0; a < M; ++a) { s_e[a] = Real(0); s_F[a] = Real(0); }
  static_for<0, Q>([&](auto I_) {
    constexpr int i = decltype(I_)::value;
    if constexpr (i != 13) {
      long long node; int slot;
      aa_write_loc(PAR, nb, n, i, node, slot);
      // species
      Real Dif[M];
#pragma unroll
      for (int b = 0; b < M; ++b) {
        const Real ex = tri(sp[b].a[0], cx_of(i)), ey = tri(sp[b].a[1], cy_of(i)), ez = tri(sp[b].a[2], cz_of(i));
        const Real dx = tri(td[b][0], cx_of(i)), dy = tri(td[b][1], cy_of(i)), dz = tri(td[b][2], cz_of(i));
        const Real sx = ex - dx, sy = ey - dy;
        Dif[b] = dx * ey * ez + sx * dy * ez + sx * sy * dz;
      }
#pragma unroll
      for (int a = 0; a < M; ++a) {
        Real F = Real(0);
#pragma unroll
        for (int b = 0; b < M; ++b) F += kap[a][b] * Dif[b];
        const Real e = th.rho_a[a] * prod3_diff<Real, i>(sp[a].a, sp[a].r, sp[a].da)
                     + th.rho_a_dev[a] * prod3<Real, i>(sp[a].r[0], sp[a].r[1], sp[a].r[2]);
        s_e[a] += e; s_F[a] += F;
        const Real kn = k[a][i] + Real(2) * beta[a] * (e - k[a][i]) + (beta[a] - Real(1)) * F;
        codec_store<Store, Real>(p, pops, (a * Q + slot) * N + node, a, kn);
      }
      // momentum lattice
      {
        const Real e = rho * prod3_diff<Real, i>(fp.a, fp.r, fp.da)
                     + rho_dev * prod3<Real, i>(fp.r[0], fp.r[1], fp.r[2]);
        s_f += e;
        Real fn = f[i] + om * (e - f[i]);
        if constexpr (c2_of(i) == 1) fn += Real(0.5) * dotc<Real, i>(Xc);
        codec_store<Store, Real>(p, pops, (M * Q + slot) * N + node, M, fn);
      }
      // energy lattice
      {
        const Real uc = dotc<Real, i>(th.u);
        const Real cc = Real(0.5) * Real(c2_of(i));
        const Real Ei = E0 + cc * rho + Gc * uc * uc * inv_theta;
        const Real dEi = dE0 + cc * rho_dev + Gc * uc * uc * inv_theta;
        const Real wi = prod3<Real, i>(gw, gw, gw);
        const Real wri = prod3<Real, i>(gwr, gwr, gwr);
        const Real dwi = tri(gdw, cx_of(i)) * tri(gw, cy_of(i)) * tri(gw, cz_of(i))
                       + tri(gwr, cx_of(i)) * tri(gdw, cy_of(i)) * tri(gw, cz_of(i))
                       + tri(gwr, cx_of(i)) * tri(gwr, cy_of(i)) * tri(gdw, cz_of(i));
        const Real e = dwi * Ei + wri * dEi + BdotZ<Real, i>(dZ);
        s_g += e;
        const Real gn = g[i] + om * (e - g[i]) + wi * dotc<Real, i>(mvec);
        codec_store<Store, Real>(p, pops, ((M + 1) * Q + slot) * N + node, M + 1, gn);
      }
    }
  });
  {
    constexpr int i = 13;
    long long node; int slot;
    aa_write_loc(PAR, nb, n, i, node, slot);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      const Real e = th.rho_a_dev[a] - s_e[a];
      const Real kn = k[a][i] + Real(2) * beta[a] * (e - k[a][i]) - (beta[a] - Real(1)) * s_F[a];
      codec_store<Store, Real>(p, pops, (a * Q + slot) * N + node, a, kn);
    }
    codec_store<Store, Real>(p, pops, (M * Q + slot) * N + node, M, f[i] + om * ((rho_dev - s_f) - f[i]));
    codec_store<Store, Real>(p, pops, ((M + 1) * Q + slot) * N + node, M + 1,
                             g[i] + om * ((rhoE_dev - s_g) - g[i]));
  }
}

// ---------------------------------------------------------------------------
// Observables (get_moments): rho, u, T, P, X_a, Y_a, V_a.
// ---------------------------------------------------------------------------
template <int M, class Real, class Store>
__global__ void __launch_bounds__(BLOCK)
moments_kernel(const DevParams<Real> p, const Store* __restrict__ pops, int parity, double* __restrict__ out) {
  const long long n = gtid();
  if (n >= p.N) return;
  const long long N = p.N;
  const Nbr nb = make_nbr(p, n);
  Real rdev[M], ja[M][3], rho_dev, j[3], rhoE_dev;
  load_state_moments<M, Real, Store>(p, pops, parity, nb, n, false, rdev, ja, rho_dev, j, rhoE_dev);
  Real jsum[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
  for (int a = 0; a < M; ++a) { jsum[0] += ja[a][0]; jsum[1] += ja[a][1]; jsum[2] += ja[a][2]; }
  Thermo<M, Real> th;
  thermo_state<M, Real>(p, rdev, jsum, rho_dev, j, rhoE_dev, th);
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
  out[0 * N + n] = (double)th.rho;
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

// Natural-layout full populations (checkpoint interface): f = b + d.
template <int M, class Real, class Store>
__global__ void __launch_bounds__(BLOCK_LIGHT)
get_pops_kernel(const DevParams<Real> p, const Store* __restrict__ pops, const double* __restrict__ base,
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
      out[(L * Q + i) * N + n] = base[L * Q + i] + (double)codec_load<Store, Real>(p, pops, (L * Q + slot) * N + node, L);
  }
}

template <int M, class Real, class Store>
__global__ void __launch_bounds__(BLOCK_LIGHT)
set_pops_kernel(const DevParams<Real> p, Store* __restrict__ pops, const double* __restrict__ base,
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
      codec_store<Store, Real>(p, pops, (L * Q + slot) * N + node, L, (Real)(in[(L * Q + i) * N + n] - base[L * Q + i]));
  }
}

// ---------------------------------------------------------------------------
// a12: FP64 conservation sums of the deviations (the host adds N times the
// reference zeroth moments).  Pass 1: per-block partials (warp shuffles, then
// shared memory); pass 2: one block sums the partials in a fixed order.
// ---------------------------------------------------------------------------
constexpr int DIAG_BLOCK = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <int M, class Real, class Store>
__global__ void __launch_bounds__(DIAG_BLOCK)
diag_partial_kernel(const DevParams<Real> p, const Store* __restrict__ pops, int parity, double* __restrict__ partials) {
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
      for (int a = 0; a < M; ++a) v[a] += (double)codec_load<Store, Real>(p, pops, (a * Q + slot) * N + node, a);
      const double fv = (double)codec_load<Store, Real>(p, pops, (M * Q + slot) * N + node, M);
      v[M] += fv;
      v[M + 1] += cx_of(i) * fv; v[M + 2] += cy_of(i) * fv; v[M + 3] += cz_of(i) * fv;
      v[M + 4] += (double)codec_load<Store, Real>(p, pops, ((M + 1) * Q + slot) * N + node, M + 1);
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NV; ++s) {
    const double t = warp_sum(v[s]);
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
    init_kernel<M, Store><<<grid_for(c.N, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(
        *c.p64, (Store*)c.pops, c.base, X, u, T, Pr);
    return cudaGetLastError();
  }
  static cudaError_t step(const LaunchCtx& c, int parity) {
    Real* side = (Real*)c.side;
    if (c.ev) cudaEventRecord(c.ev[0], c.stream);
    side_kernel<M, Real, Store><<<grid_for(c.N, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(
        P(c), (const Store*)c.pops, side, parity);
    if (c.ev) cudaEventRecord(c.ev[1], c.stream);
    grad_kernel<Real><<<grid_for(c.N, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(P(c), side);
    if (c.ev) cudaEventRecord(c.ev[2], c.stream);
    if (parity == 0)
      collide_kernel<M, Real, Store, 0><<<grid_for(c.N, BLOCK), BLOCK, 0, c.stream>>>(
          P(c), (Store*)c.pops, side, c.err);
    else
      collide_kernel<M, Real, Store, 1><<<grid_for(c.N, BLOCK), BLOCK, 0, c.stream>>>(
          P(c), (Store*)c.pops, side, c.err);
    if (c.ev) cudaEventRecord(c.ev[3], c.stream);
    return cudaGetLastError();
  }
  static cudaError_t moments(const LaunchCtx& c, int parity, double* out) {
    moments_kernel<M, Real, Store><<<grid_for(c.N, BLOCK), BLOCK, 0, c.stream>>>(
        P(c), (const Store*)c.pops, parity, out);
    return cudaGetLastError();
  }
  static cudaError_t get_pops(const LaunchCtx& c, int parity, double* out) {
    get_pops_kernel<M, Real, Store><<<grid_for(c.N, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(
        P(c), (const Store*)c.pops, c.base, parity, out);
    return cudaGetLastError();
  }
  static cudaError_t set_pops(const LaunchCtx& c, int parity, const double* in) {
    set_pops_kernel<M, Real, Store><<<grid_for(c.N, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(
        P(c), (Store*)c.pops, c.base, parity, in);
    return cudaGetLastError();
  }
  static cudaError_t diag(const LaunchCtx& c, int parity, double* d_sums) {
    const unsigned nb = grid_for(c.N, DIAG_BLOCK);
    diag_partial_kernel<M, Real, Store><<<nb, DIAG_BLOCK, 0, c.stream>>>(
        P(c), (const Store*)c.pops, parity, c.partials);
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
