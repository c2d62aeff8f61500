// lbm_device.cuh -- per-node device arithmetic of the multicomponent D3Q27
// lattice Boltzmann step (Sawant, Dorschner & Karlin, arXiv 2004.11286).
//
// Everything here is templated on the species count M (compile-time, so the
// per-node state lives in registers) and on the arithmetic type Real
// (double for the FP64 path, float otherwise).  The storage type of the
// populations is handled by the codec in lbm_codec.cuh.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <type_traits>

namespace lbm {

constexpr int Q = 27;
constexpr int MAXM = 8;
// Scratch planes per node (Real):
//   written by collide:  Phi_x,Phi_y,Phi_z (0-2), c_omega (3), C_p (4), s = c2/theta (5), theta (6)
//   written by grad_GK:  G_x,G_y,G_z (7-9), K_x,K_y,K_z (10-12), theta of the sender (13)
//   written by grad_X:   X_x,X_y,X_z (14-16)
//   with temperature-dependent heats, written by collide: the mixture
//   enthalpy coefficients Phi_2, Phi_3 of H = T (Phi_1 + Phi_2 T + Phi_3 T^2)
//   (Phi_1 in the C_p plane) and T (17-19)
constexpr int NSIDE = 20;
enum SidePlane { SP_PHI = 0, SP_COM = 3, SP_CP = 4, SP_S = 5, SP_TH = 6, SP_G = 7, SP_K = 10, SP_THR = 13, SP_X = 14,
                 SP_HC2 = 17, SP_HC3 = 18, SP_T = 19 };

// Velocity i = (cx+1) + 3(cy+1) + 9(cz+1), Eq. (d3q27vel).
__host__ __device__ constexpr int cx_of(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int cy_of(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int cz_of(int i) { return i / 9 - 1; }
__host__ __device__ constexpr int c2_of(int i) {
  return cx_of(i) * cx_of(i) + cy_of(i) * cy_of(i) + cz_of(i) * cz_of(i);
}
__host__ __device__ constexpr int opp_of(int i) { return 26 - i; }
__host__ __device__ constexpr int c_of(int i, int a) {
  return a == 0 ? cx_of(i) : (a == 1 ? cy_of(i) : cz_of(i));
}

// Isotropic D3Q27 gradient weights (second-order isotropic operator of Sec. 4.1):
// d_a phi(x) = 3 sum_i w_i c_ia phi(x + c_i).
template <class Real>
__host__ __device__ constexpr Real iso_w(int i) {
  return c2_of(i) == 0 ? Real(8) / Real(27)
       : c2_of(i) == 1 ? Real(2) / Real(27)
       : c2_of(i) == 2 ? Real(1) / Real(54) : Real(1) / Real(216);
}

// Constants derived on the host from the problem statement.
template <class Real>
struct DevParams {
  long long N;
  int nx, ny, nz;
  int M;
  int slaved;            // strong coupling: slaved species index
  int weak;              // 1 = weak coupling (Sec. 3.5.1)
  int wall_x;            // 1 = bounce-back walls at x = -1/2 and x = nx - 1/2 (closed tube)
  int omega_is_fixed, omega1_is_fixed;
  Real omega_fixed, omega1_fixed;
  Real R_U;
  Real rho_eps;          // V_a = 0 where rho_a <= rho_eps * rho
  Real cond_bound;       // FP64 re-solve threshold for the SM system (FP32 paths)
  Real closure_bound;    // learned closure: largest accepted residual of the J-form system
  Real mass[MAXM];
  Real inv_mass[MAXM];
  Real R_a[MAXM];
  Real Cv_a[MAXM];
  Real Cp_a[MAXM];
  Real mu[MAXM];
  Real lam[MAXM];
  Real inv_lam[MAXM];
  Real phi[MAXM][MAXM];  // Wilke factors, Eq. (wilkePhi)
  Real Cab[MAXM][MAXM];  // 1 / (D_ab m_a m_b): 1/tau_ab = R_U T m Cab (Eq. tauab)
  double Cab64[MAXM][MAXM];
  // Reference rest state.  Populations are stored as deviations d = f - b
  // from each lattice's rest equilibrium b at this state; RL[L] = sum_i b_Li.
  Real RL[MAXM + 2];
  double RL64[MAXM + 2]; // the same in FP64 (the FP64 re-solve of the SM system)
  Real Yr[MAXM];         // reference mass fractions, RL[a] / sum_a RL[a]
  Real Tr, Rr, thr, Pr;  // reference T, mixture R, theta = R T, P = RL[f] theta
  Real Cvr;              // reference mixture C_v
  Real cE;               // RL[g] - RL[f] Cvr Tr       (rounding-level constant)
  Real cPi;              // sum_i b_fi c_ix^2 - RL[f] thr (rounding-level constant)
  Real cS;               // RL[f] - sum_a RL[a]
  Real Rsp;              // sum_a RL[a]
  Real scale[MAXM + 2], inv_scale[MAXM + 2];   // storage scale of reduced-precision modes
  // Reduced-precision storage (lbm_eqcodec.cuh): the reference rest
  // equilibria b_L,i by lattice and |c_i|^2, and the width in floats of the
  // per-node equilibrium record (0 in the FP64 and FP32 modes).
  Real bref[MAXM + 2][4];
  int rec_w;
  // Temperature-dependent heats (Sec. 3.1), tvar = 1: per mass and per species
  // C_{a,v}(T) = sum_k cvp[a][k] T^k (k < nterm), U_a(T) = T sum_k Uc[a][k] T^k
  // with Uc = cvp / (k + 1), H_a(T) = T sum_k Hc[a][k] T^k (Hc = Uc, plus R_a
  // at k = 0); Uar[a] = U_a(T_r), Ur the reference mixture's U(T_r).
  int tvar, nterm;
  Real cvp[MAXM][3], Uc[MAXM][3], Hc[MAXM][3], Uar[MAXM];
  Real Ur;
  int frame;             // 1 = opposed-jets frame (lbm_frame.cuh): nozzle rows [jet_y0, jet_y1)
  int jet_y0, jet_y1;
};

// Byte offsets k * N * sizeof(stored type) of the population planes
// k = L * 27 + i (a kernel parameter: addresses then add a constant-bank
// operand to the node's own address instead of multiplying by N).
struct PlaneOffsets {
  long long off[(MAXM + 2) * 27];
};

// ---------------------------------------------------------------------------
// Product form, Sec. 2.4: triplets Psi_0, Psi_{+1}, Psi_{-1}.
// ---------------------------------------------------------------------------
template <class Real>
struct Triplet { Real m, z, p; };   // values for c = -1, 0, +1

template <class Real>
__device__ __forceinline__ Triplet<Real> psi_triplet(Real xi, Real zeta) {
  Real s = xi * xi + zeta;
  Triplet<Real> t;
  t.z = Real(1) - s;
  t.p = Real(0.5) * (s + xi);
  t.m = Real(0.5) * (s - xi);
  return t;
}

template <class Real>
__device__ __forceinline__ Real tri(const Triplet<Real>& t, int c) {
  return c < 0 ? t.m : (c == 0 ? t.z : t.p);
}

// ---------------------------------------------------------------------------
// Grid addressing.
// ---------------------------------------------------------------------------
struct Nbr {
  unsigned xs[3], ys[3], zs[3];  // wrapped coordinates for offsets -1, 0, +1 (y, z pre-scaled); N < 2^31
  unsigned wall;                 // bit 0: a wall lies at -x of this node, bit 1: at +x
  __device__ __forceinline__ long long idx(int dx, int dy, int dz) const {
    return (long long)(zs[dz + 1] + ys[dy + 1] + xs[dx + 1]);
  }
};

// Neighbour table of node n on the grid of p (any type with nx, ny, nz,
// wall_x): periodic, except that with walls normal to x the neighbour
// beyond a wall is the node itself (its mirror image across the wall).
template <class P>
__device__ __forceinline__ Nbr make_nbr(const P& p, long long n_) {
  Nbr b;
  const unsigned n = (unsigned)n_;
  const unsigned nx = (unsigned)p.nx, ny = (unsigned)p.ny, nz = (unsigned)p.nz;
  const unsigned x = n % nx;
  const unsigned t = n / nx;
  const unsigned y = t % ny;
  const unsigned z = t / ny;
  const unsigned pl = nx * ny;
  const bool w = p.wall_x != 0;
  b.xs[0] = x == 0 ? (w ? x : nx - 1) : x - 1;  b.xs[1] = x;  b.xs[2] = x == nx - 1 ? (w ? x : 0) : x + 1;
  b.wall = w ? ((x == 0 ? 1u : 0u) | (x == nx - 1 ? 2u : 0u)) : 0u;
  b.ys[0] = (y == 0 ? ny - 1 : y - 1) * nx;  b.ys[1] = y * nx;  b.ys[2] = (y == ny - 1 ? 0 : y + 1) * nx;
  b.zs[0] = (z == 0 ? nz - 1 : z - 1) * pl;  b.zs[1] = z * pl;
  b.zs[2] = (z == nz - 1 ? 0 : z + 1) * pl;
  return b;
}

// A copy of a node index that the compiler cannot identify with the
// original (see opaque below): at even parity every store address of a
// phase is the node's own, and would otherwise be kept live from the loads.
__device__ __forceinline__ long long opaque_idx(long long a) {
  long long b;
  asm volatile("mov.b64 %0, %1;" : "=l"(b) : "l"(a));
  return b;
}

// A copy of the neighbour table that the compiler cannot identify with the
// original, so addresses recomputed from it are not merged with (and kept
// live from) those of an earlier phase of the same kernel.
__device__ __forceinline__ Nbr opaque(const Nbr& a) {
  Nbr b;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    asm volatile("mov.u32 %0, %1;" : "=r"(b.xs[k]) : "r"(a.xs[k]));
    asm volatile("mov.u32 %0, %1;" : "=r"(b.ys[k]) : "r"(a.ys[k]));
    asm volatile("mov.u32 %0, %1;" : "=r"(b.zs[k]) : "r"(a.zs[k]));
  }
  b.wall = a.wall;
  return b;
}

// Halfway bounce-back at the walls normal to x: direction i arrives from
// beyond a wall (its sender x - c_i is outside), or would leave through one.
__device__ __forceinline__ bool arrives_from_wall(const Nbr& nb, int i) {
  const int cx = cx_of(i);
  return (cx > 0 && (nb.wall & 1u)) || (cx < 0 && (nb.wall & 2u));
}
__device__ __forceinline__ bool leaves_to_wall(const Nbr& nb, int i) {
  const int cx = cx_of(i);
  return (cx > 0 && (nb.wall & 2u)) || (cx < 0 && (nb.wall & 1u));
}

// AA pattern.  parity 0 (even time level): logical population i of node x
// lives in slot i of x; the collision writes its result for direction i to
// slot opp(i) of x.  parity 1: logical population i of x lives in slot
// opp(i) of x - c_i; the collision writes direction i to slot i of x + c_i.
// Each node reads and writes the same set of addresses in a step.
// Walls (WALL, halfway bounce-back) change only the odd level: a population
// arriving from beyond a wall is the node's own opposite one, which its
// previous odd-level collision left in slot i of the node itself; one that
// would leave is kept at the node, in slot opp(i), for its next even level.
template <bool WALL>
__device__ __forceinline__ void aa_read_loc(int parity, const Nbr& nb, long long n, int i,
                                            long long& node, int& slot) {
  if (parity == 0) { node = n; slot = i; }
  else if (WALL && arrives_from_wall(nb, i)) { node = n; slot = i; }
  else { node = nb.idx(-cx_of(i), -cy_of(i), -cz_of(i)); slot = opp_of(i); }
}
template <bool WALL>
__device__ __forceinline__ void aa_write_loc(int parity, const Nbr& nb, long long n, int i,
                                             long long& node, int& slot) {
  if (parity == 0 || (WALL && leaves_to_wall(nb, i))) { node = n; slot = opp_of(i); }
  else { node = nb.idx(cx_of(i), cy_of(i), cz_of(i)); slot = i; }
}

// ---------------------------------------------------------------------------
// Per-node thermodynamic state (Secs. 2.1, 3.1, 3.3, 3.5), carried as full
// values plus their deviations from the reference rest state, so that every
// equilibrium can be formed as a small deviation without cancellation.
// ---------------------------------------------------------------------------
template <int M, class Real>
struct Thermo {
  Real rho_a[M], rho_a_dev[M];   // coupled species densities and deviations from RL[a]
  Real Y[M];
  Real rho_sp;                   // density seen by the species (rho under strong coupling)
  Real rho, rho_dev;             // mixture density (momentum lattice), deviation from RL[f]
  Real m, R, Cv, Cp, usq;
  Real T, dT, theta, dtheta, P, dP;
  Real u[3];                     // mixture velocity (momentum lattice)
  Real u_sp[3];                  // velocity seen by the species
  Real omega;
};

// rdev: species zeroth-moment deviations (the slaved entry is ignored under
// strong coupling); ja_sum: sum of species momenta (weak coupling only);
// rho_dev, j, rhoE_dev: momentum/energy lattice moments as deviations.
template <int M, class Real>
__device__ __forceinline__ void thermo_state(const DevParams<Real>& p, const Real (&rdev)[M],
                                             const Real (&ja_sum)[3], Real rho_dev, const Real (&j)[3],
                                             Real rhoE_dev, Thermo<M, Real>& th) {
  th.rho_dev = rho_dev;
  th.rho = p.RL[M] + rho_dev;
  const Real rho = th.rho;
  const Real inv_rho = Real(1) / rho;
  th.u[0] = j[0] * inv_rho; th.u[1] = j[1] * inv_rho; th.u[2] = j[2] * inv_rho;
  Real sp_dev;   // rho_sp - Rsp
  if (!p.weak) {
    // Eqs. (rhoMATCH), (uMATCH): the slaved species takes the deficit.
    Real others = Real(0);
#pragma unroll
    for (int a = 0; a < M; ++a) if (a != p.slaved) others += rdev[a];
#pragma unroll
    for (int a = 0; a < M; ++a) {
      th.rho_a_dev[a] = (a == p.slaved) ? p.cS + rho_dev - others : rdev[a];
      th.rho_a[a] = p.RL[a] + th.rho_a_dev[a];
    }
    th.rho_sp = rho;
    sp_dev = p.cS + rho_dev;
    th.u_sp[0] = th.u[0]; th.u_sp[1] = th.u[1]; th.u_sp[2] = th.u[2];
  } else {
    sp_dev = Real(0);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      th.rho_a_dev[a] = rdev[a];
      th.rho_a[a] = p.RL[a] + rdev[a];
      sp_dev += rdev[a];
    }
    th.rho_sp = p.Rsp + sp_dev;
    const Real is = Real(1) / th.rho_sp;
    th.u_sp[0] = ja_sum[0] * is; th.u_sp[1] = ja_sum[1] * is; th.u_sp[2] = ja_sum[2] * is;
  }
  const Real inv_sp = Real(1) / th.rho_sp;
  Real inv_m = Real(0), d_inv_m = Real(0), Cv = Real(0), dCv = Real(0), Cp = Real(0);
#pragma unroll
  for (int a = 0; a < M; ++a) {
    th.Y[a] = th.rho_a[a] * inv_sp;                               // Eq. (mixtureDensity)
    const Real dY = (th.rho_a_dev[a] - p.Yr[a] * sp_dev) * inv_sp; // Y_a - Yr_a
    inv_m += th.Y[a] * p.inv_mass[a];                             // Eq. (meanMolecularWeight)
    d_inv_m += dY * p.inv_mass[a];
    Cv += th.Y[a] * p.Cv_a[a];                                    // Eq. (Cvmix)
    dCv += dY * p.Cv_a[a];
    Cp += th.Y[a] * p.Cp_a[a];
  }
  th.m = Real(1) / inv_m;
  th.R = p.R_U * inv_m;                                           // Eq. (defineSpecificGasContant)
  const Real dR = p.R_U * d_inv_m;
  th.Cv = Cv; th.Cp = Cp;
  th.usq = th.u[0] * th.u[0] + th.u[1] * th.u[1] + th.u[2] * th.u[2];
  if (!p.tvar) {
    // Eq. (temperature2) with T0 = 0, rho E = rho (C_v T + u^2/2), written for
    // T - Tr:  rho C_v (T - Tr) = rho E - rho u^2/2 - rho C_v Tr.
    th.dT = (p.cE + rhoE_dev - Real(0.5) * rho * th.usq - rho_dev * p.Cvr * p.Tr - rho * dCv * p.Tr)
          / (rho * Cv);
  } else {
    // Eq. (temperature) with T0 = 0: rho U(T) = rho E - rho u^2/2, U = sum_a Y_a U_a,
    // written for dT = T - Tr as  rho [U(T) - U(Tr)] = rhs  with
    //   rhs = rho E - rho U(Tr) - rho u^2/2
    //       = cE + (rho E - RL_g) - (rho - RL_f) U_r - rho sum_a (Y_a - Yr_a) U_a(Tr) - rho u^2/2
    // and U(T) - U(Tr) = dT sum_k u_k (T^k + T^(k-1) Tr + ... + Tr^k) (no
    // cancellation), solved by Newton's method (U' = C_v > 0).
    Real um[3] = {Real(0), Real(0), Real(0)}, cm[3] = {Real(0), Real(0), Real(0)}, sdU = Real(0);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      const Real dY = (th.rho_a_dev[a] - p.Yr[a] * sp_dev) * inv_sp;
      sdU += dY * p.Uar[a];
#pragma unroll
      for (int k = 0; k < 3; ++k) { um[k] += th.Y[a] * p.Uc[a][k]; cm[k] += th.Y[a] * p.cvp[a][k]; }
    }
    const Real rhs = p.cE + rhoE_dev - rho_dev * p.Ur - rho * sdU - Real(0.5) * rho * th.usq;
    const Real Tr = p.Tr;
    Real dT = rhs / (rho * (cm[0] + Tr * (cm[1] + Tr * cm[2])));
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const Real T = Tr + dT;
      const Real G = um[0] + um[1] * (T + Tr) + um[2] * (T * T + T * Tr + Tr * Tr);
      const Real cvT = cm[0] + T * (cm[1] + T * cm[2]);
      dT -= (rho * dT * G - rhs) / (rho * cvT);
    }
    th.dT = dT;
    const Real T = Tr + dT;
    th.Cv = cm[0] + T * (cm[1] + T * cm[2]);
    th.Cp = th.Cv + th.R;
  }
  th.T = p.Tr + th.dT;
  th.theta = th.R * th.T;
  th.dtheta = dR * th.T + p.Rr * th.dT;
  th.P = rho * th.theta;                                          // Eq. (eosIdealGas)
  th.dP = rho_dev * th.theta + p.RL[M] * th.dtheta;
  if (p.omega_is_fixed) {
    th.omega = p.omega_fixed;
  } else {
    // Wilke, Eqs. (viscosityMixture), (wilkePhi); X_a = m Y_a / m_a.
    Real X[M];
#pragma unroll
    for (int a = 0; a < M; ++a) X[a] = th.m * th.Y[a] * p.inv_mass[a];
    Real mu = Real(0);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      Real den = Real(0);
#pragma unroll
      for (int b = 0; b < M; ++b) den += p.phi[a][b] * X[b];
      mu += p.mu[a] * X[a] / den;
    }
    th.omega = Real(2) * th.P / (th.P + Real(2) * mu);            // Eq. (omega)
  }
}

// FP64 forms for initialisation, records and the host: per-mass heat, internal
// energy and enthalpy of species a at T (Eqs. specUa, specHa, T0 = 0), and the
// T that solves sum_a Y_a U_a(T) = e (Eq. temperature) by Newton's method.
__host__ __device__ inline double cv_a64(const DevParams<double>& p, int a, double T) {
  return p.tvar ? p.cvp[a][0] + T * (p.cvp[a][1] + T * p.cvp[a][2]) : p.Cv_a[a];
}
__host__ __device__ inline double U_a64(const DevParams<double>& p, int a, double T) {
  return p.tvar ? T * (p.Uc[a][0] + T * (p.Uc[a][1] + T * p.Uc[a][2])) : p.Cv_a[a] * T;
}
__host__ __device__ inline double H_a64(const DevParams<double>& p, int a, double T) {
  return U_a64(p, a, T) + p.R_a[a] * T;
}
__host__ __device__ inline double T_from_energy64(const DevParams<double>& p, const double* Y, int M, double e) {
  double cv0 = 0.0;
  for (int a = 0; a < M; ++a) cv0 += Y[a] * cv_a64(p, a, 0.0);
  double T = e / cv0;
  if (!p.tvar) return T;
  for (int it = 0; it < 60; ++it) {
    double U = 0.0, cv = 0.0;
    for (int a = 0; a < M; ++a) { U += Y[a] * U_a64(p, a, T); cv += Y[a] * cv_a64(p, a, T); }
    const double dT = (U - e) / cv;
    T -= dT;
    if (fabs(dT) <= 1e-15 * fabs(T)) break;
  }
  return T;
}

// Species enthalpy H_a(T) (Eq. specHa, T0 = 0): C_{a,p} T with constant
// heats, T (Hc_0 + Hc_1 T + Hc_2 T^2) with temperature-dependent ones.
template <class Real>
__device__ __forceinline__ Real enthalpy_a(const DevParams<Real>& p, int a, Real T) {
  if (!p.tvar) return p.Cp_a[a] * T;
  return T * (p.Hc[a][0] + T * (p.Hc[a][1] + T * p.Hc[a][2]));
}
// Mixture enthalpy H = sum_a Y_a H_a (Eq. specH).
template <int M, class Real>
__device__ __forceinline__ Real enthalpy(const DevParams<Real>& p, const Thermo<M, Real>& th) {
  if (!p.tvar) return th.Cp * th.T;
  Real h = Real(0);
#pragma unroll
  for (int a = 0; a < M; ++a) h += th.Y[a] * enthalpy_a(p, a, th.T);
  return h;
}

template <int M, class Real>
__device__ __forceinline__ Real omega1_of(const DevParams<Real>& p, const Thermo<M, Real>& th) {
  if (p.omega1_is_fixed) return p.omega1_fixed;
  // Mathur, Eq. (conductivityMixture); Eq. (omega1).
  Real s1 = Real(0), s2 = Real(0);
#pragma unroll
  for (int a = 0; a < M; ++a) {
    Real X = th.m * th.Y[a] * p.inv_mass[a];
    s1 += X * p.lam[a];
    s2 += X * p.inv_lam[a];
  }
  Real lam = Real(0.5) * (s1 + Real(1) / s2);
  Real pc = th.P * th.Cp;
  return Real(2) * pc / (pc + Real(2) * lam);
}

// ---------------------------------------------------------------------------
// Stefan-Maxwell diffusion fluxes J_a = rho_a V_a from Eq. (transform12),
// written for J (well posed when rho_a -> 0):
//   J_a + 1/2 sum_{b != a} (1/tau_ab) (Y_b J_a - Y_a J_b) = j_a - rho_a u.
// The matrix is I plus a singular column-diagonally-dominant M-matrix
// (columns sum to one), so elimination without pivoting is stable; its
// 1-norm condition number is bounded by 1 + max_b sum_{a != b} Y_a/tau_ab.
// ---------------------------------------------------------------------------
template <int M, class T>
__device__ __forceinline__ void sm_eliminate(T (&A)[M][M], T (&r)[M][3], T (&J)[M][3]) {
#pragma unroll
  for (int k = 0; k < M; ++k) {
    T inv = T(1) / A[k][k];
#pragma unroll
    for (int i = k + 1; i < M; ++i) {
      T l = A[i][k] * inv;
#pragma unroll
      for (int jj = k + 1; jj < M; ++jj) A[i][jj] -= l * A[k][jj];
#pragma unroll
      for (int c = 0; c < 3; ++c) r[i][c] -= l * r[k][c];
    }
  }
#pragma unroll
  for (int k = M - 1; k >= 0; --k) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T s = r[k][c];
#pragma unroll
      for (int jj = k + 1; jj < M; ++jj) s -= A[k][jj] * J[jj][c];
      J[k][c] = s / A[k][k];
    }
  }
}

// FP64 species moments for the FP64 re-solve: densities, momenta, the
// velocity the species see and their total density (Eqs. rhoMATCH, uMATCH
// under strong coupling; Eqs. rhoSPEC, uSPEC under weak coupling).
template <int M>
struct SpMoments64 {
  double rho_a[M], ja[M][3], u[3], rho_sp;
};
// Default source of the FP64 re-solve's inputs: the arithmetic-type moments.
struct FromThermo {};

// The exact solve.  In the FP32 paths a system whose condition bound
// exceeds p.cond_bound is solved in FP64 instead.  Its solution splits into
// the components the system damps (by 1/tau) and the one it passes
// unchanged: A Y = Y, so r + s Y gives J + s Y, and the component of r along
// sum_a r_a = j - rho u (under either coupling) is zero in exact arithmetic.
// Formed in FP32 that component is rounding noise of the size of eps |j|, a
// common shift of every species velocity that swamps diffusion velocities of
// order r tau.  So the FP64 system takes
//   * `mom` (an SpMoments64 filler): moments summed in FP64 from the stored
//     populations, where sum_a r_a vanishes to FP64 rounding (the readers);
//   * FromThermo: the FP32 moments with that component removed,
//     r_a -= Y_a sum_b r_b (the collide: there the shift is harmless, the force
//     of Eq. fstar1 multiplies it by 1/tau_ab and the update by beta_a - 1,
//     about -2 tau_a, and re-reading the stage in FP64 costs 2 % of the step).
template <int M, class Real, class Mom = FromThermo>
__device__ __forceinline__ void sm_solve(const DevParams<Real>& p, const Thermo<M, Real>& th,
                                         const Real (&itab)[M][M], const Real (&ja)[M][3],
                                         Real (&J)[M][3], const Mom& mom = Mom{}) {
  Real A[M][M], r[M][3];
  Real cond = Real(0);
#pragma unroll
  for (int a = 0; a < M; ++a) {
    Real diag = Real(1);
#pragma unroll
    for (int b = 0; b < M; ++b) {
      if (b != a) {
        diag += Real(0.5) * itab[a][b] * th.Y[b];
        A[a][b] = Real(-0.5) * itab[a][b] * th.Y[a];
      }
    }
    A[a][a] = diag;
#pragma unroll
    for (int c = 0; c < 3; ++c) r[a][c] = ja[a][c] - th.rho_a[a] * th.u_sp[c];
    cond = fmax(cond, Real(2) * (diag - Real(1)));
  }
  if constexpr (sizeof(Real) == 4) {
    if (cond + Real(1) > p.cond_bound) {
      // Ill-conditioned system in the FP32 paths: re-solve in FP64.
      double A64[M][M], r64[M][3], J64[M][3], Y64[M];
      double tm;
      if constexpr (std::is_same<Mom, FromThermo>::value) {
        tm = (double)p.R_U * (double)th.T * (double)th.m;
#pragma unroll
        for (int a = 0; a < M; ++a) {
          Y64[a] = (double)th.Y[a];
#pragma unroll
          for (int c = 0; c < 3; ++c) r64[a][c] = (double)ja[a][c] - (double)th.rho_a[a] * (double)th.u_sp[c];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          double sr = 0.0;
#pragma unroll
          for (int a = 0; a < M; ++a) sr += r64[a][c];
#pragma unroll
          for (int a = 0; a < M; ++a) r64[a][c] -= Y64[a] * sr;
        }
      } else {
        SpMoments64<M> m;
        mom(m);
        double inv_m = 0.0;
#pragma unroll
        for (int a = 0; a < M; ++a) {
          Y64[a] = m.rho_a[a] / m.rho_sp;
          inv_m += Y64[a] / (double)p.mass[a];
#pragma unroll
          for (int c = 0; c < 3; ++c) r64[a][c] = m.ja[a][c] - m.rho_a[a] * m.u[c];
        }
        tm = (double)p.R_U * (double)th.T / inv_m;
      }
#pragma unroll
      for (int a = 0; a < M; ++a) {
        double diag = 1.0;
#pragma unroll
        for (int b = 0; b < M; ++b) {
          if (b != a) {
            const double it = tm * p.Cab64[a][b];
            diag += 0.5 * it * Y64[b];
            A64[a][b] = -0.5 * it * Y64[a];
          }
        }
        A64[a][a] = diag;
      }
      sm_eliminate<M, double>(A64, r64, J64);
#pragma unroll
      for (int a = 0; a < M; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) J[a][c] = (Real)J64[a][c];
      return;
    }
  }
  sm_eliminate<M, Real>(A, r, J);
}

}  // namespace lbm
