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
#include "lbm_eqcodec.cuh"

namespace lbm {

// Four consecutive values (16-byte aligned for FP32, 32-byte for FP64).
template <class Real>
__device__ __forceinline__ void load4(const Real* __restrict__ f, Real* v) {
  if constexpr (sizeof(Real) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(f);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(f);
    const double2 b = *reinterpret_cast<const double2*>(f + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
}
template <class Real>
__device__ __forceinline__ void store4(Real* __restrict__ f, const Real* v) {
  if constexpr (sizeof(Real) == 4) {
    *reinterpret_cast<float4*>(f) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    *reinterpret_cast<double2*>(f) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(f + 2) = make_double2(v[2], v[3]);
  }
}

// Read-only gathers of the deferred terms through the non-coherent data path
// (LBM_SIDE_LDG = 1; the collide never writes the planes it gathers from).
#ifndef LBM_SIDE_LDG
#define LBM_SIDE_LDG 1
#endif
template <class Real>
__device__ __forceinline__ Real side_ld(const Real* p) {
#if LBM_SIDE_LDG
  return __ldg(p);
#else
  return *p;
#endif
}

// The deferred terms of the population that `sender` sent in direction I,
// for a sender whose theta is th.
template <class Real, int I>
__device__ __forceinline__ void incoming_corr_th(const Real* __restrict__ side, long long N, long long sender,
                                                 Real th, Real& cf, Real& cg) {
  constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
  Real kc = Real(0);
  if constexpr (cx != 0) kc += (cx > 0 ? side_ld(side + (SP_K + 0) * N + sender) : -side_ld(side + (SP_K + 0) * N + sender));
  if constexpr (cy != 0) kc += (cy > 0 ? side_ld(side + (SP_K + 1) * N + sender) : -side_ld(side + (SP_K + 1) * N + sender));
  if constexpr (cz != 0) kc += (cz > 0 ? side_ld(side + (SP_K + 2) * N + sender) : -side_ld(side + (SP_K + 2) * N + sender));
  const Real w0 = Real(1) - th, w1 = Real(0.5) * th;
  const Real w = (cx ? w1 : w0) * (cy ? w1 : w0) * (cz ? w1 : w0);   // Eq. (weights)
  cg = w * kc;
  cf = Real(0);
  if constexpr (c2_of(I) == 1) {
    constexpr int a = cx ? 0 : (cy ? 1 : 2);
    constexpr int sg = cx + cy + cz;
    cf = (sg > 0 ? Real(0.5) : Real(-0.5)) * side_ld(side + (SP_X + a) * N + sender);
  }
}
template <class Real, int I>
__device__ __forceinline__ void incoming_corr(const Real* __restrict__ side, long long N, long long sender,
                                              Real& cf, Real& cg) {
  incoming_corr_th<Real, I>(side, N, sender, side_ld(side + SP_THR * N + sender), cf, cg);
}

// Reduced-precision storage: the record of the node that sent the population
// arriving at n in direction I, the equilibrium shifts of every lattice for
// that population (lbm_eqcodec.cuh) and its deferred terms.  The sender is
// n - c_I; with walls, a population arriving from beyond a wall is n's own
// population of direction opp(I) reflected, so it was stored with n's shift
// for opp(I) and carries n's terms for I negated.
template <int M, int I, bool WALL>
__device__ __forceinline__ void eq_incoming(const DevParams<float>& p, const float* __restrict__ side,
                                            const Nbr& nb, long long n, int parity, float& cf, float& cg,
                                            float (&sh)[M + 2]) {
  const long long N = p.N;
  const float* rin = eq_rec_buf(side, N, p.rec_w, 1 - parity);
  bool refl = false;
  long long snd = n;
  if constexpr (I != 13) {
    if (WALL && arrives_from_wall(nb, I)) refl = true;
    else snd = nb.idx(-cx_of(I), -cy_of(I), -cz_of(I));
  }
  const EqRec<M> r = load_rec<M>(rin, snd, p.rec_w, p.weak);
  if (WALL && refl) eq_shift<M, opp_of(I)>(p, r, sh);
  else eq_shift<M, I>(p, r, sh);
  cf = 0.0f; cg = 0.0f;
  if constexpr (I != 13) {
    incoming_corr_th<float, I>(side, N, snd, p.thr + r.dth, cf, cg);
    if (WALL && refl) { cf = -cf; cg = -cg; }
  }
}

// The deferred terms of the population arriving in direction I at node n.
// With walls (WALL), one arriving from beyond a wall is the node's own
// population of direction opp(I) reflected, so its terms are the node's own
// for opp(I): those of I at the node, negated (w_opp(I) = w_I, c_opp(I) = -c_I).
template <class Real, int I, bool WALL>
__device__ __forceinline__ void deferred_terms(const Real* __restrict__ side, long long N, const Nbr& nb,
                                               long long n, Real& cf, Real& cg) {
  if constexpr (WALL) {
    if (arrives_from_wall(nb, I)) {
      incoming_corr<Real, I>(side, N, n, cf, cg);
      cf = -cf;
      cg = -cg;
      return;
    }
  }
  incoming_corr<Real, I>(side, N, nb.idx(-cx_of(I), -cy_of(I), -cz_of(I)), cf, cg);
}

// The decoding terms of the population arriving at n in direction I for the
// readers of the state: the deferred non-local terms cf (f) and cg (g), and
// with 16-bit storage the equilibrium shifts sh of every lattice (zero
// otherwise); walls are handled whether or not the grid has them.
template <int M, class Real, class Store, int I>
__device__ __forceinline__ void incoming_terms(const DevParams<Real>& p, const Real* __restrict__ side,
                                               const Nbr& nb, long long n, int parity, Real& cf, Real& cg,
                                               Real (&sh)[M + 2]) {
  cf = Real(0); cg = Real(0);
  if constexpr (kEqCodec<Store, Real>) {
    eq_incoming<M, I, true>(p, side, nb, n, parity, cf, cg, sh);
  } else {
#pragma unroll
    for (int L = 0; L < M + 2; ++L) sh[L] = Real(0);
    if constexpr (I != 13) deferred_terms<Real, I, true>(side, p.N, nb, n, cf, cg);
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
    aa_read_loc<true>(parity, nb, n, i, node, slot);
    Real cf, cg, sh[M + 2];
    incoming_terms<M, Real, Store, i>(p, side, nb, n, parity, cf, cg, sh);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      const Real v = codec_load<Store, Real>(p, pops, (a * Q + slot) * N + node, a) + sh[a];
      rdev[a] += v;
      if (cx) ja[a][0] += cx * v;
      if (cy) ja[a][1] += cy * v;
      if (cz) ja[a][2] += cz * v;
    }
    const Real fv = codec_load<Store, Real>(p, pops, (M * Q + slot) * N + node, M) + cf + sh[M];
    rho_dev += fv;
    if (cx) j[0] += cx * fv;
    if (cy) j[1] += cy * fv;
    if (cz) j[2] += cz * fv;
    rhoE_dev += codec_load<Store, Real>(p, pops, ((M + 1) * Q + slot) * N + node, M + 1) + cg + sh[M + 1];
  });
}

// Stencil pass 1 (after a collision): G_alpha = c_omega d_alpha Phi_alpha (the
// inner derivative of Eq. Xalpha) and K_alpha = s d_alpha C_p with s = c2 / theta;
// the sender's theta is copied for the receivers' weights.
// With temperature-dependent heats (tvar) the enthalpy field differentiated
// is H-like: Phi_1 + T_n Phi_2 + T_n^2 Phi_3 of the neighbours with this
// node's T_n, so that K = s sum_k T^(k-1) grad Phi_k = (s / T) sum_a H_a grad Y_a.
template <class Real, class G>
__device__ __forceinline__ void grad_GK_node(const G& p, Real* __restrict__ side, long long n, bool tvar = false) {
  if (n >= p.N) return;
  const long long N = p.N;
  const Nbr nb = make_nbr(p, n);
  Real d[3] = {Real(0), Real(0), Real(0)}, dc[3] = {Real(0), Real(0), Real(0)};
  const Real Tn = tvar ? side[SP_T * N + n] : Real(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
    if (i == 13) continue;
    const long long nn = nb.idx(cx, cy, cz);
    const Real w = iso_w<Real>(i);
    Real cp = side[SP_CP * N + nn];
    if (tvar) cp += Tn * (side[SP_HC2 * N + nn] + Tn * side[SP_HC3 * N + nn]);
    // beyond a wall the mirror image of Phi_x is odd, the other fields even
    const bool mirror = (cx < 0 && (nb.wall & 1u)) || (cx > 0 && (nb.wall & 2u));
    if (cx) {
      const Real phx = side[(SP_PHI + 0) * N + nn];
      d[0] += (cx * w) * (mirror ? -phx : phx);
      dc[0] += (cx * w) * cp;
    }
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

// ---------------------------------------------------------------------------
// Row-blocked stencil passes (grids with nx a multiple of ROWV): one thread
// computes ROWV consecutive nodes of a row.  The D3Q27 weights factor per
// axis, w_i = w(c_ix) w(c_iy) w(c_iz) with w(0) = 2/3, w(+-1) = 1/6, so the
// isotropic gradient separates over the nine neighbour rows (c_y, c_z):
//   d_x phi = (1/72) sum_{cy,cz} W(cy) W(cz) [phi(x+1) - phi(x-1)]
//   d_y phi = (1/72) sum_{cz} W(cz) [s(+1, cz) - s(-1, cz)]
//   d_z phi = (1/72) sum_{cy} W(cy) [s(cy, +1) - s(cy, -1)]
// with W(0) = 4, W(+-1) = 1 and s = phi(x-1) + 4 phi(x) + phi(x+1) on the
// row.  Each row is read once as ROWV + 2 values (x0-1 .. x0+ROWV) shared by
// the thread's nodes: the middle ones as 16-byte vector loads, the two ends
// as scalar loads or (SHFL) from the neighbouring lanes, which hold them as
// their own middle values, except at warp and row edges.  Every lane of a
// warp takes part in the shuffles; lanes past the grid compute on the last
// nodes and store nothing.
// ---------------------------------------------------------------------------
#ifndef LBM_STENCIL_ROW
#define LBM_STENCIL_ROW 4
#endif
constexpr int ROWV = LBM_STENCIL_ROW;
static_assert(ROWV == 4 || ROWV == 8, "row blocking of 4 or 8 nodes");

// Row coordinates of the nodes n0 .. n0+ROWV-1 (x0 = n0 mod nx, a multiple of ROWV).
struct RowV {
  unsigned x0, xm, xp;       // first x, its left neighbour, the right neighbour of the last node (periodic)
  unsigned ys[3], zs[3];     // wrapped row offsets for c_y, c_z = -1, 0, +1
  bool from_left, from_right;   // the end values are held by lane - 1 / lane + 1 (same row)
  bool wlo, whi;                // walls: the left / right end value is a mirror image
  __device__ __forceinline__ unsigned row(int cy, int cz) const { return zs[cz + 1] + ys[cy + 1]; }
};
template <class P>
__device__ __forceinline__ RowV make_row(const P& p, unsigned n0) {
  RowV r;
  const unsigned nx = (unsigned)p.nx, ny = (unsigned)p.ny, nz = (unsigned)p.nz;
  r.x0 = n0 % nx;
  const unsigned t = n0 / nx, y = t % ny, z = t / ny, pl = nx * ny;
  const bool w = p.wall_x != 0;
  r.wlo = w && r.x0 == 0;
  r.whi = w && r.x0 + ROWV == nx;
  r.xm = r.x0 == 0 ? (w ? 0 : nx - 1) : r.x0 - 1;
  r.xp = r.x0 + ROWV == nx ? (w ? nx - 1 : 0) : r.x0 + ROWV;
  const unsigned lane = threadIdx.x & 31u;
  r.from_left = lane > 0 && r.x0 != 0;
  r.from_right = lane < 31 && r.x0 + ROWV != nx;
  r.ys[0] = (y == 0 ? ny - 1 : y - 1) * nx;  r.ys[1] = y * nx;  r.ys[2] = (y == ny - 1 ? 0 : y + 1) * nx;
  r.zs[0] = (z == 0 ? nz - 1 : z - 1) * pl;  r.zs[1] = z * pl;  r.zs[2] = (z == nz - 1 ? 0 : z + 1) * pl;
  return r;
}
// ODD: the field is odd under the mirror at a wall (Phi_x).
template <class Real, bool SHFL, bool ODD = false>
__device__ __forceinline__ void load_row(const Real* __restrict__ f, const RowV& r, unsigned rb, Real (&v)[ROWV + 2]) {
  if constexpr (SHFL) {
#pragma unroll
    for (int q = 0; q < ROWV; q += 4) load4<Real>(f + rb + r.x0 + q, v + 1 + q);
    const Real left = __shfl_up_sync(0xffffffffu, v[ROWV], 1);
    const Real right = __shfl_down_sync(0xffffffffu, v[1], 1);
    v[0] = r.from_left ? left : f[rb + r.xm];
    v[ROWV + 1] = r.from_right ? right : f[rb + r.xp];
  } else {
    v[0] = f[rb + r.xm];
#pragma unroll
    for (int q = 0; q < ROWV; q += 4) load4<Real>(f + rb + r.x0 + q, v + 1 + q);
    v[ROWV + 1] = f[rb + r.xp];
  }
  if constexpr (ODD) {
    if (r.wlo) v[0] = -v[0];
    if (r.whi) v[ROWV + 1] = -v[ROWV + 1];
  }
}
// End values by shuffle in the second pass only: in the first (four fields
// per row) the shuffles raised it from 64 to 80 registers and it ran slower,
// also when held to 64 (measured on GB300, 128^3 acoustic pulse).  Without
// shuffles the end loads go first: issued after the vector load the pass
// took 58 registers and ran 9 % slower.
#ifndef LBM_GK_SHFL
#define LBM_GK_SHFL 0
#endif
#ifndef LBM_X_SHFL
#define LBM_X_SHFL 1
#endif
// Adds row (cy, cz) of a field to the a-derivative accumulators d[ROWV] (a = 0, 1, 2).
template <class Real, int A>
__device__ __forceinline__ void row_derivative(const Real (&v)[ROWV + 2], int cy, int cz, Real (&d)[ROWV]) {
  const Real Wy = cy ? Real(1) : Real(4), Wz = cz ? Real(1) : Real(4);
#pragma unroll
  for (int j = 0; j < ROWV; ++j) {
    if constexpr (A == 0) d[j] += (Wy * Wz) * (v[j + 2] - v[j]);
    else {
      const Real s = v[j] + Real(4) * v[j + 1] + v[j + 2];
      if constexpr (A == 1) d[j] += (cy * Wz) * s;
      else d[j] += (cz * Wy) * s;
    }
  }
}

// Pass 1 on ROWV nodes: G_a = c_omega d_a Phi_a, K = s grad C_p, theta copied.
template <class Real>
__device__ __forceinline__ void grad_GK_row(const DevParams<Real>& p, Real* __restrict__ side, unsigned n0,
                                            bool store) {
  const long long N = p.N;
  const RowV r = make_row(p, n0);
  Real dp[3][ROWV], dc[3][ROWV];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < ROWV; ++j) dp[a][j] = dc[a][j] = Real(0);
#pragma unroll
  for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
    for (int cy = -1; cy <= 1; ++cy) {
      const unsigned rb = r.row(cy, cz);
      Real v[ROWV + 2];
      load_row<Real, LBM_GK_SHFL, true>(side + (SP_PHI + 0) * N, r, rb, v);
      row_derivative<Real, 0>(v, cy, cz, dp[0]);
      if (cy) { load_row<Real, LBM_GK_SHFL>(side + (SP_PHI + 1) * N, r, rb, v); row_derivative<Real, 1>(v, cy, cz, dp[1]); }
      if (cz) { load_row<Real, LBM_GK_SHFL>(side + (SP_PHI + 2) * N, r, rb, v); row_derivative<Real, 2>(v, cy, cz, dp[2]); }
      load_row<Real, LBM_GK_SHFL>(side + SP_CP * N, r, rb, v);
      row_derivative<Real, 0>(v, cy, cz, dc[0]);
      if (cy) row_derivative<Real, 1>(v, cy, cz, dc[1]);
      if (cz) row_derivative<Real, 2>(v, cy, cz, dc[2]);
    }
  if (!store) return;
  const unsigned own = r.row(0, 0) + r.x0;
  const Real k72 = Real(1) / Real(72);
#pragma unroll
  for (int q = 0; q < ROWV; q += 4) {
    Real co[4], sv[4], th[4];
    load4<Real>(side + SP_COM * N + own + q, co);
    load4<Real>(side + SP_S * N + own + q, sv);
    load4<Real>(side + SP_TH * N + own + q, th);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Real g[4], k[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) { g[j] = co[j] * (dp[a][q + j] * k72); k[j] = sv[j] * (dc[a][q + j] * k72); }
      store4<Real>(side + (SP_G + a) * N + own + q, g);
      store4<Real>(side + (SP_K + a) * N + own + q, k);
    }
    store4<Real>(side + SP_THR * N + own + q, th);
  }
}

// Pass 2 on ROWV nodes: X_a = -d_a G_a.
template <class Real>
__device__ __forceinline__ void grad_X_row(const DevParams<Real>& p, Real* __restrict__ side, unsigned n0,
                                           bool store) {
  const long long N = p.N;
  const RowV r = make_row(p, n0);
  Real d[3][ROWV];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < ROWV; ++j) d[a][j] = Real(0);
#pragma unroll
  for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
    for (int cy = -1; cy <= 1; ++cy) {
      const unsigned rb = r.row(cy, cz);
      Real v[ROWV + 2];
      load_row<Real, LBM_X_SHFL>(side + (SP_G + 0) * N, r, rb, v);
      row_derivative<Real, 0>(v, cy, cz, d[0]);
      if (cy) { load_row<Real, LBM_X_SHFL>(side + (SP_G + 1) * N, r, rb, v); row_derivative<Real, 1>(v, cy, cz, d[1]); }
      if (cz) { load_row<Real, LBM_X_SHFL>(side + (SP_G + 2) * N, r, rb, v); row_derivative<Real, 2>(v, cy, cz, d[2]); }
    }
  if (!store) return;
  const unsigned own = r.row(0, 0) + r.x0;
  const Real k72 = Real(-1) / Real(72);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int q = 0; q < ROWV; q += 4) {
      Real x[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = d[a][q + j] * k72;
      store4<Real>(side + (SP_X + a) * N + own + q, x);
    }
}

// LBM_GK_MINB > 0 sets a minimum of resident blocks per SM (FP32); by
// default the compiler chooses (64 registers, four blocks of 256).
#ifndef LBM_GK_MINB
#define LBM_GK_MINB 0
#endif
template <class Real>
__global__ void
#if LBM_GK_MINB > 0
__launch_bounds__(BLOCK_LIGHT, sizeof(Real) == 4 ? LBM_GK_MINB : 1)
#else
__launch_bounds__(BLOCK_LIGHT)
#endif
grad_GK_row_kernel(const __grid_constant__ DevParams<Real> p, Real* __restrict__ side) {
  const long long t = gtid();
  const bool in = ROWV * t < p.N;
  grad_GK_row<Real>(p, side, (unsigned)(in ? ROWV * t : p.N - ROWV), in);
}
template <class Real>
__global__ void __launch_bounds__(BLOCK_LIGHT)
grad_X_row_kernel(const __grid_constant__ DevParams<Real> p, Real* __restrict__ side) {
  const long long t = gtid();
  const bool in = ROWV * t < p.N;
  grad_X_row<Real>(p, side, (unsigned)(in ? ROWV * t : p.N - ROWV), in);
}

template <class Real>
__global__ void __launch_bounds__(BLOCK_LIGHT)
grad_GK_kernel(const __grid_constant__ DevParams<Real> p, Real* __restrict__ side) {
  grad_GK_node<Real>(p, side, gtid(), p.tvar != 0);
}
template <class Real>
__global__ void __launch_bounds__(BLOCK_LIGHT)
grad_X_kernel(const __grid_constant__ DevParams<Real> p, Real* __restrict__ side) {
  grad_X_node<Real>(p, side, gtid());
}

}  // namespace lbm
