// lbm_collide.cuh -- the fused collide + stream of every lattice at one node.
//
// Written for the stored deviations d = f - b of the populations from the
// reference rest equilibria (the update is affine, so d' = f' - b exactly):
//   species (Eq. SMlbm):     d' = d + 2 beta_a (e_a - d) + (beta_a - 1) F_a
//   f (Eq. fwithcorrection): d' = d + omega (e - d)         [+ A_i . X, deferred]
//   g (Eq. g):               d' = d + omega (e_g - d) + w_i(theta) c_i . K / theta
// with every equilibrium deviation e = f^eq - b formed from deviation
// quantities (no O(f) cancellation).  The node also writes its side fields
// for the stencil passes of lbm_stencil.cuh.
#pragma once

#include "lbm_stencil.cuh"
#include "lbm_mlp.cuh"

namespace lbm {

// Threads per block: the deviations of all S lattices are staged in shared
// memory (S * 27 values per thread), kept near 110 KB per block.  With the
// learned closure (CL = 1) a block is one 128-node tile of the network.
#ifndef LBM_COLLIDE_BS
#define LBM_COLLIDE_BS 128
#endif
// The stage holds every population in the arithmetic type, decoded and with
// its deferred terms added.
template <class Real, class Store>
using StageSp = Real;
template <int M, class Real, class Store>
constexpr long long stage_per_node() {
  return (long long)M * 27 * sizeof(StageSp<Real, Store>) + 2LL * 27 * sizeof(Real);
}
// Tiles of the network per block: two (256 nodes, 8 warps) where the stage of
// 256 nodes, the weight image and two activation tiles fit in shared memory.
template <int M, class Real, class Store = Real>
constexpr int kMlpTiles =
    stage_per_node<M, Real, Store>() * 2 * MLP_TILE + mlp_smem<M, 2>() <= 227LL * 1024 ? 2 : 1;
template <int M, class Real, int CL = 0, class Store = Real>
constexpr int collide_block() {
  constexpr long long per = stage_per_node<M, Real, Store>();
  if constexpr (CL) return MLP_TILE * kMlpTiles<M, Real, Store>;
  return per * LBM_COLLIDE_BS <= 113 * 1024 ? LBM_COLLIDE_BS
       : (per * 64 <= 113 * 1024 ? 64 : 32);
}

// Store addresses recomputed in each store phase from an opaque copy of the
// node index (1), or left to the compiler, which at even parity (every
// address the node's own) keeps load addresses live for the stores (0).
#ifndef LBM_OPAQUE_STORE
#define LBM_OPAQUE_STORE 2
#endif
template <int M, class Store>
constexpr bool kOpaqueStore = LBM_OPAQUE_STORE == 2 ? (M >= 3 || sizeof(Store) == 2) : LBM_OPAQUE_STORE != 0;

// Minimum resident blocks per SM asked of the register allocator, capped by
// what the shared-memory tile allows (LBM_COLLIDE_MINB overrides).  Measured
// on GB300 with 128-node blocks:
//   M <= 2, FP32 storage: 3 (168 registers; 256^3 shear layer 4321 MLUPS
//     against 3443 at 4, where the odd-parity kernel spills);
//   M <= 2, 16-bit storage: 4 (128 registers; 2411 against 2158 at 3);
//   M = 3: 3 (128^3 mixture FP32 2987 against 2961 at 2, BF16 1451 against 977);
//   M >= 4: 2 (255 registers; the stage allows no more from M = 5 on).
template <int M, class Real, int CL = 0, class Store = Real>
constexpr int collide_min_blocks() {
  if constexpr (CL) return 1;
#ifdef LBM_COLLIDE_MINB
  constexpr int want = LBM_COLLIDE_MINB;
#else
  constexpr int want = M <= 2 ? (sizeof(Store) == 2 ? 4 : 3) : (M == 3 ? 3 : 2);
#endif
  constexpr long long bytes = stage_per_node<M, Real, Store>() * collide_block<M, Real, 0, Store>();
  constexpr long long nb = (227LL * 1024) / bytes;
  constexpr int fit = nb >= 8 ? 8 : (nb < 1 ? 1 : (int)nb);
  return want < fit ? want : fit;
}

// Bulk (TMA engine) row loads of the populations where the grid allows them,
// from LBM_COLLIDE_BULK_MIN_M species: measured on GB300 (128^3 random
// mixtures) M = 3 FP32 2585 against 2301 MLUPS for register loads, M = 8
// 635 against 576, but M = 2 3464 against 3566 (the 128^3 acoustic pulse).
#ifndef LBM_COLLIDE_BULK
#define LBM_COLLIDE_BULK 1
#endif
#ifndef LBM_COLLIDE_BULK_MIN_M
#define LBM_COLLIDE_BULK_MIN_M 3
#endif

// Population addresses as the node's own plus a per-plane byte offset from
// the kernel parameters (1), or from the plane index times the grid size (0).
// Measured on GB300: 256^3 shear layer FP32 4652 against 4430 MLUPS, 128^3
// ternary mixture 3211 against 3048 (the same offsets for the gathers of the
// side planes measured no faster: 4553).
#ifndef LBM_PLANE_OFFSETS
#define LBM_PLANE_OFFSETS 1
#endif

// Species counts from which the species update loops over the velocities at
// run time rather than unrolled (see the species phase of collide_node).
#ifndef LBM_SPECIES_LOOP_MIN_M
#define LBM_SPECIES_LOOP_MIN_M 4
#endif
// Unrolled species update with per-axis factor tables (1) or the factors
// recomputed at every velocity (0).
#ifndef LBM_SPECIES_AXIS_TABLES
#define LBM_SPECIES_AXIS_TABLES 1
#endif
// FP32: the load phase's moment sums as pairs of lanes (species 2k, 2k + 1;
// f, g) of the paired FP32 instructions (1), or one sum at a time (0).
// Auto (2): where measured faster, M >= 3 or 16-bit storage (the FP32 M = 2
// kernel spills with them: 256^3 shear layer 3909 against 4455 MLUPS).
#ifndef LBM_PAIRED_MOMENTS
#define LBM_PAIRED_MOMENTS 2
#endif
// FP32, M = 2 or 3: species 0 and 1 updated as one pair of lanes of the
// paired FP32 instructions (1), or one species at a time (0).
#ifndef LBM_SPECIES_PAIRS
#define LBM_SPECIES_PAIRS 1
#endif

template <int M, class Real, int CL = 0, class Store = Real>
constexpr size_t collide_stage_bytes() {
  return (size_t)(stage_per_node<M, Real, Store>() * collide_block<M, Real, CL, Store>() + 15) / 16 * 16;
}
// Bulk row loads (LD = 1) add one halo value per staged plane and an mbarrier.
template <int M, class Real>
constexpr size_t collide_halo_bytes() {
  return ((size_t)(M + 2) * Q * sizeof(Real) + 7) / 8 * 8;
}
template <int M, class Real, int CL = 0, int LD = 0, class Store = Real>
constexpr size_t collide_smem() {
  if constexpr (CL) return collide_stage_bytes<M, Real, CL, Store>() + mlp_smem<M, kMlpTiles<M, Real, Store>>();
  if constexpr (LD) return collide_stage_bytes<M, Real, CL, Store>() + collide_halo_bytes<M, Real>() + 8;
  return collide_stage_bytes<M, Real, CL, Store>();
}
// The network closure exists for the FP32-arithmetic paths with M >= 2.
template <int M, class Real>
constexpr bool kMlpOk = (M >= 2) && sizeof(Real) == 4;

// Bulk row loads of the row segment [x0, x0 + BS) whose first node is n0:
// every lattice plane of every velocity as one aligned copy of BS values of
// its source row (the segment's own row at even parity, the row y - c_y,
// z - c_z at odd parity) into buf[plane][BS], completing on mbar (armed by
// the caller); at odd parity on segmented rows the value each x-shifted
// velocity needs from outside the segment goes to halo[plane].  Planes are
// shared out over lanes lane, lane + nlanes, ...
template <int M, class Real, class Store, int PAR, int BS>
__device__ __forceinline__ void issue_row_loads(const DevParams<Real>& p, const Store* __restrict__ pops, Real* buf,
                                                Real* halo, uint32_t mbar, long long n0, int lane, int nlanes) {
  const long long N = p.N;
  const long long rowi = n0 / p.nx;
  const int x0 = (int)(n0 - rowi * p.nx);
  const int yr = (int)(rowi % p.ny), zr0 = (int)(rowi / p.ny);
  const bool whole_row = p.nx == BS;
  for (int k = lane; k < (M + 2) * Q; k += nlanes) {
    const int L = k / Q, i = k % Q;
    const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
    int ys = yr, zs = zr0, slot = i;
    if (PAR) {
      ys = yr - cy; ys = ys < 0 ? ys + p.ny : (ys >= p.ny ? ys - p.ny : ys);
      zs = zr0 - cz; zs = zs < 0 ? zs + p.nz : (zs >= p.nz ? zs - p.nz : zs);
      slot = Q - 1 - i;
    }
    const Store* src = pops + ((long long)(L * Q + slot) * N + ((long long)zs * p.ny + ys) * p.nx);
    bulk_g2s(buf + (size_t)k * BS, src + x0, (uint32_t)(BS * sizeof(Real)), mbar);
    if (PAR && cx != 0 && !whole_row) {
      int xh = cx > 0 ? x0 - 1 : x0 + BS;
      xh = xh < 0 ? xh + p.nx : (xh >= p.nx ? xh - p.nx : xh);
      halo[k] = (Real)src[xh];
    }
  }
}

// One node's collide + stream (thread threadIdx.x of the block; the block's
// shared memory holds the stage and, with CL = 1, the network's tile).
// WALL: bounce-back walls normal to x (register-load path only).
// POFF: the byte offsets of the population planes come from poff (the
// kernel's parameter block), else they are computed from the grid size.
// FRAME: the outermost x and y layers are the opposed-jets frame, whose nodes
// take no collision (lbm_frame.cuh).
template <int M, class Real, class Store, int PAR, int CL, int LD = 0, bool WALL = false, bool POFF = false,
          bool FRAME = false>
__device__ __forceinline__ void collide_node(const DevParams<Real>& p, Store* __restrict__ pops,
                                             Real* __restrict__ side, unsigned* __restrict__ err,
                                             const unsigned char* __restrict__ mlp_img,
                                             unsigned long long* __restrict__ mlp_stats, long long n_raw,
                                             unsigned char* smem_raw, const long long* poff = nullptr) {
  constexpr int BS = collide_block<M, Real, CL, Store>();
  using SpT = StageSp<Real, Store>;
  // 16-bit storage: shifted deviations from the senders' equilibria (lbm_eqcodec.cuh)
  constexpr bool EQ = kEqCodec<Store, Real>;
  static_assert(!LD || std::is_same<Store, Real>::value, "bulk loads stage the stored type");
  static_assert(!(LD && WALL), "walls use the register-load path");
  // Stage, thread-private columns: species [M*27][BS] (SpT), then f, g [2*27][BS] (Real).
  SpT* const sps = reinterpret_cast<SpT*>(smem_raw);
  Real* const sfg = reinterpret_cast<Real*>(smem_raw + (size_t)M * Q * BS * sizeof(SpT));
  Real* const sm = reinterpret_cast<Real*>(smem_raw);   // the whole stage when SpT == Real
  const long long N = p.N;
  const int tid = threadIdx.x;
  // With the network every thread of the block takes part in its tile; the
  // threads past the grid compute on a copy of the last node and store nothing.
  const bool active = n_raw < N;
  if constexpr (!CL) {
    if (!active) return;
  }
  const long long n = active ? n_raw : N - 1;
  if constexpr (FRAME && !CL) {
    const long long x = n % p.nx, y = (n / p.nx) % p.ny;
    if (x == 0 || x == p.nx - 1 || y == 0 || y == p.ny - 1) return;
  }
  MlpBlock<M, kMlpTiles<M, Real, Store>> mlp{smem_raw + collide_stage_bytes<M, Real, CL, Store>(), 0u, 0u};
  if constexpr (CL) mlp.begin_setup(mlp_img);
  const Nbr nb = make_nbr(p, n);
  // Population k = L * 27 + slot of node `node`.
  auto pop_at = [&](long long k, long long node) -> Store* {
    if constexpr (POFF) return reinterpret_cast<Store*>(reinterpret_cast<char*>(pops + node) + poff[k]);
    else return pops + (k * N + node);
  };

  // a1 + a2: load (AA addressing), add the deferred terms of the previous
  // step, accumulate the moments of the deviations (the reference tables have
  // zero first and off-diagonal second moments) and stage the values.
  Real rdev[M], ja[M][3];
  Real rho_dev = Real(0), j[3] = {Real(0), Real(0), Real(0)};
  Real S[6] = {Real(0), Real(0), Real(0), Real(0), Real(0), Real(0)};
  Real rhoE_dev = Real(0), q[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
  for (int a = 0; a < M; ++a) { rdev[a] = Real(0); ja[a][0] = ja[a][1] = ja[a][2] = Real(0); }
  // The staged value of lattice L, velocity i (cx its x component) for this
  // thread.  With bulk row loads at odd parity a velocity's source row sits
  // in the stage shifted by cx; the value that falls outside the segment is
  // the plane's halo value (or wraps, when the segment is the whole row).
  Real* const halo = sfg + 2 * Q * BS;
  const bool whole_row = p.nx == BS;
  // momentum/energy planes (L = M, M + 1), and species planes when SpT == Real
  auto plane = [&](int L, int i) -> Real* {
    return L >= M ? sfg + ((L - M) * Q + i) * BS : reinterpret_cast<Real*>(sps) + (L * Q + i) * BS;
  };
  auto cell = [&](int L, int i, int cx) -> Real& {
    Real* const pl = plane(L, i);
    if constexpr (LD && PAR) {
      const int li = tid - cx;
      if (li < 0 || li >= BS) return whole_row ? pl[li < 0 ? BS - 1 : 0] : halo[L * Q + i];
      return pl[li];
    } else {
      (void)cx;
      return pl[tid];
    }
  };
  auto species_val = [&](int a, int i, int cx) -> Real { return cell(a, i, cx); };
  // FP32: species 2k and 2k + 1, and the f and g lattices, accumulate as
  // the two lanes of paired FP32 instructions.
  constexpr bool PA = std::is_same<Real, float>::value &&
                      (LBM_PAIRED_MOMENTS == 2 ? (M >= 3 || sizeof(Store) == 2) : LBM_PAIRED_MOMENTS != 0);
  constexpr int MP = PA ? M / 2 : 0;
  float2 pr[MP > 0 ? MP : 1][4];         // (rho, j_x, j_y, j_z) of species 2k | 2k + 1
  float2 pfg[4];                         // (rho, j) of f | (rho E, q) of g
  if constexpr (PA) {
#pragma unroll
    for (int k = 0; k < MP; ++k)
#pragma unroll
      for (int c = 0; c < 4; ++c) pr[k][c] = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 4; ++c) pfg[c] = make_float2(0.f, 0.f);
  }
  auto acc2 = [](float2& a, float2 v, int c) {
    if (c > 0) a = add2(a, v);
    else if (c < 0) a = sub2(a, v);
  };
  auto accumulate = [&](auto I_, const Real* v, Real fv, Real gv) {
    constexpr int i = decltype(I_)::value;
    constexpr int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
    if constexpr (PA) {
#pragma unroll
      for (int k = 0; k < MP; ++k) {
        const float2 vv = make_float2(v[2 * k], v[2 * k + 1]);
        pr[k][0] = add2(pr[k][0], vv);
        acc2(pr[k][1], vv, cx); acc2(pr[k][2], vv, cy); acc2(pr[k][3], vv, cz);
      }
      if constexpr (M % 2) {
        rdev[M - 1] += v[M - 1];
        if (cx) ja[M - 1][0] += cx * v[M - 1];
        if (cy) ja[M - 1][1] += cy * v[M - 1];
        if (cz) ja[M - 1][2] += cz * v[M - 1];
      }
      const float2 fg = make_float2(fv, gv);
      pfg[0] = add2(pfg[0], fg);
      acc2(pfg[1], fg, cx); acc2(pfg[2], fg, cy); acc2(pfg[3], fg, cz);
    } else {
#pragma unroll
      for (int a = 0; a < M; ++a) {
        rdev[a] += v[a];
        if (cx) ja[a][0] += cx * v[a];
        if (cy) ja[a][1] += cy * v[a];
        if (cz) ja[a][2] += cz * v[a];
      }
      rho_dev += fv;
      if (cx) j[0] += cx * fv;
      if (cy) j[1] += cy * fv;
      if (cz) j[2] += cz * fv;
      rhoE_dev += gv;
      if (cx) q[0] += cx * gv;
      if (cy) q[1] += cy * gv;
      if (cz) q[2] += cz * gv;
    }
    if (cx) S[0] += fv;
    if (cy) S[1] += fv;
    if (cz) S[2] += fv;
    if (cx && cy) S[3] += (cx * cy) * fv;
    if (cx && cz) S[4] += (cx * cz) * fv;
    if (cy && cz) S[5] += (cy * cz) * fv;
  };
  if constexpr (LD) {
    // The block is the row segment [x0, x0 + BS) of one grid row.  Every
    // lattice plane of every velocity arrives as one aligned bulk copy of the
    // BS values of its source row (the node's own row at even parity, the
    // row y - c_y, z - c_z at odd parity); the senders' deferred terms are
    // gathered while the copies are in flight.
    const uint32_t mbar = smem_u32(reinterpret_cast<unsigned char*>(halo) + collide_halo_bytes<M, Real>());
    if (tid == 0) {
      mbar_init(mbar, 1);
      mbar_expect_tx(mbar, (uint32_t)((M + 2) * Q * BS * sizeof(Real)));
    }
    __syncthreads();
    issue_row_loads<M, Real, Store, PAR, BS>(p, pops, sm, halo, mbar, n_raw - tid, tid, BS);
    Real cfv[Q], cgv[Q];
    static_for<0, Q>([&](auto I_) {
      constexpr int i = decltype(I_)::value;
      cfv[i] = Real(0); cgv[i] = Real(0);
      if constexpr (i != 13)
        incoming_corr<Real, i>(side, N, nb.idx(-cx_of(i), -cy_of(i), -cz_of(i)), cfv[i], cgv[i]);
    });
    if (!mbar_wait(mbar, 0u)) atomicOr(err, 4u);
    __syncthreads();                                   // halo values
    static_for<0, Q>([&](auto I_) {
      constexpr int i = decltype(I_)::value;
      constexpr int cx = cx_of(i);
      Real v[M];
#pragma unroll
      for (int a = 0; a < M; ++a) v[a] = species_val(a, i, cx);
      Real& fc = cell(M, i, cx);
      Real& gc = cell(M + 1, i, cx);
      Real fv = fc, gv = gc;
      if constexpr (c2_of(i) == 1) { fv += cfv[i]; fc = fv; }
      if constexpr (i != 13) { gv += cgv[i]; gc = gv; }
      accumulate(I_, v, fv, gv);
    });
  } else {
    static_for<0, Q>([&](auto I_) {
      constexpr int i = decltype(I_)::value;
      long long node; int slot;
      aa_read_loc<WALL>(PAR, nb, n, i, node, slot);
      Real cf = Real(0), cg = Real(0);
      Real v[M + 2];   // species, then the shifts of f and g (zero without the shifted codec)
      if constexpr (EQ) eq_incoming<M, i, WALL>(p, side, nb, n, PAR, cf, cg, v);
      else if constexpr (i != 13) deferred_terms<Real, i, WALL>(side, N, nb, n, cf, cg);
#pragma unroll
      for (int a = 0; a < M; ++a) {
        const Real d = codec_load<Store, Real>(p, pop_at(a * Q + slot, node), 0, a);
        if constexpr (EQ) v[a] += d; else v[a] = d;
        sps[(a * Q + i) * BS + tid] = v[a];
      }
      Real fv = codec_load<Store, Real>(p, pop_at(M * Q + slot, node), 0, M) + cf;
      Real gv = codec_load<Store, Real>(p, pop_at((M + 1) * Q + slot, node), 0, M + 1) + cg;
      if constexpr (EQ) { fv += v[M]; gv += v[M + 1]; }
      sfg[i * BS + tid] = fv;
      sfg[(Q + i) * BS + tid] = gv;
      accumulate(I_, v, fv, gv);
    });
  }

  if constexpr (PA) {
#pragma unroll
    for (int k = 0; k < MP; ++k) {
      rdev[2 * k] = pr[k][0].x; rdev[2 * k + 1] = pr[k][0].y;
#pragma unroll
      for (int c = 0; c < 3; ++c) { ja[2 * k][c] = pr[k][c + 1].x; ja[2 * k + 1][c] = pr[k][c + 1].y; }
    }
    rho_dev = pfg[0].x; rhoE_dev = pfg[0].y;
#pragma unroll
    for (int c = 0; c < 3; ++c) { j[c] = pfg[c + 1].x; q[c] = pfg[c + 1].y; }
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
  if (active && (!(rho > Real(0)) || !(th.T > Real(0)) || !(th.rho_sp > Real(0)))) atomicOr(err, 1u);
  const Real om = th.omega;
  const Real om1 = omega1_of<M, Real>(p, th);
  const Real P = th.P, T = th.T;

  // a5: this node's side fields: Phi_alpha = j_alpha (1 - 3RT) - rho u_alpha^3 and
  // c_omega = 1/omega - 1/2 (Eq. Xalpha); C_p and s = (1/2)(2 - omega_1) P T / theta
  // (sum_a H_a grad Y_a = T grad C_p for constant specific heats, Eq. corrFourier).
  if (active) {
    const Real a3 = Real(1) - Real(3) * th.theta;
#pragma unroll
    for (int c = 0; c < 3; ++c) side[(SP_PHI + c) * N + n] = j[c] * a3 - rho * th.u[c] * th.u[c] * th.u[c];
    side[SP_COM * N + n] = Real(1) / om - Real(0.5);
    if (!p.tvar) {
      side[SP_CP * N + n] = th.Cp;
    } else {
      // sum_a H_a grad Y_a = sum_k T^k grad Phi_k with H = T (Phi_1 + Phi_2 T + Phi_3 T^2)
      Real h1 = Real(0), h2 = Real(0), h3 = Real(0);
#pragma unroll
      for (int a = 0; a < M; ++a) { h1 += th.Y[a] * p.Hc[a][0]; h2 += th.Y[a] * p.Hc[a][1]; h3 += th.Y[a] * p.Hc[a][2]; }
      side[SP_CP * N + n] = h1;
      side[SP_HC2 * N + n] = h2;
      side[SP_HC3 * N + n] = h3;
      side[SP_T * N + n] = T;
    }
    side[SP_S * N + n] = Real(0.5) * (Real(2) - om1) * P * T / th.theta;
    side[SP_TH * N + n] = th.theta;
  }

  // a4, a6: relaxation times (Eqs. tauab, tau) and the Stefan-Maxwell fluxes.
  Real itab[M][M];
  const Real tm = p.R_U * th.T * th.m;
#pragma unroll
  for (int a = 0; a < M; ++a)
#pragma unroll
    for (int b = 0; b < M; ++b) itab[a][b] = tm * p.Cab[a][b];
  Real J[M][3];
  if constexpr (CL) {
    // a6': the network proposes the normalised fluxes; it is accepted where
    // the residual of the J-form system stays within the bound, else the
    // exact solve runs (Eq. transform12).
    Real r[M][3], sr = Real(0);
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        r[a][c] = ja[a][c] - th.rho_a[a] * th.u_sp[c];
        sr = fmax(sr, fabs(r[a][c]));
      }
    const Real inv_s = sr > Real(0) ? Real(1) / sr : Real(0);
    {
      float f[MlpDims<M>::F];
      sm_feature_values<M, Real>(p, th, itab, r, inv_s, f);
#pragma unroll
      for (int k0 = 0; k0 < MlpDims<M>::F; k0 += 8) store_row8(mlp.act(), mlp.row(), k0, MlpDims<M>::F, f + k0);
    }
    mlp.finish_setup();
    float out[MlpDims<M>::O];
    const bool ran = mlp.forward(out, err);
    // J~ = J0 + correction, J0 = (r / s) / A_aa the one-sweep Jacobi estimate
    Real rn[M][3], Jn[M][3], diag[M];
    sm_diagonal<M, Real>(th, itab, diag);
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        rn[a][c] = r[a][c] * inv_s;
        Jn[a][c] = rn[a][c] / diag[a] + (Real)out[3 * a + c];
      }
    const Real res = sm_residual<M, Real>(th, itab, diag, rn, Jn);
    const bool accept = ran && (sr == Real(0) || res <= p.closure_bound);
    if (accept) {
#pragma unroll
      for (int a = 0; a < M; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) J[a][c] = sr * Jn[a][c];
    } else {
      sm_solve<M, Real>(p, th, itab, ja, J);
    }
    const unsigned acc = __ballot_sync(0xffffffffu, active && accept);
    const unsigned act = __ballot_sync(0xffffffffu, active);
    if ((tid & 31) == 0 && act) {
      atomicAdd(&mlp_stats[0], (unsigned long long)__popc(acc));
      atomicAdd(&mlp_stats[1], (unsigned long long)__popc(act & ~acc));
    }
  } else {
    sm_solve<M, Real>(p, th, itab, ja, J);
  }
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

  // The stores run in three phases (f, g, species).  Each starts from an
  // opaque copy of the neighbour table so that the 26 neighbour addresses are
  // recomputed there rather than held live since the load phase.  The rest
  // direction (i = 13) of every lattice goes last: its equilibrium deviation
  // (and F_a,13) is the conservation remainder, identical to the product form
  // in exact arithmetic, so the zeroth moments carry no per-step rounding bias.

  // a8: momentum lattice, Eqs. (feq), (fwithcorrection), (Ai):
  //   e_i = rho (Psi_i(u, theta) - W_i) + (rho - RL_f) W_i,  W_i = Psi_i(0, theta_r).
  {
    Real s_f = Real(0);
    const Real x2[3] = {th.u[0] * th.u[0], th.u[1] * th.u[1], th.u[2] * th.u[2]};
    const Nbr nbw = opaque(nb);
    const long long nw = kOpaqueStore<M, Store> ? opaque_idx(n) : n;
    static_for<0, Q>([&](auto I_) {
      constexpr int i = decltype(I_)::value;
      if constexpr (i != 13) {
        long long node; int slot;
        aa_write_loc<WALL>(PAR, nbw, nw, i, node, slot);
        const Real e = rho * pf_diff<Real, i>(th.u, x2, p.thr, th.dtheta) + rho_dev * pf_ref<Real, i>(p.thr);
        s_f += e;
        const Real fv = cell(M, i, cx_of(i));
        const Real out = fv + om * (e - fv);
        if (active) codec_store<Store, Real>(p, pop_at(M * Q + slot, node), 0, M, EQ ? out - e : out);
      }
    });
    long long node; int slot;
    aa_write_loc<WALL>(PAR, nbw, nw, 13, node, slot);
    const Real fv = cell(M, 13, 0);
    const Real e13 = rho_dev - s_f;
    const Real out = fv + om * (e13 - fv);
    if (active) codec_store<Store, Real>(p, pop_at(M * Q + slot, node), 0, M, EQ ? out - e13 : out);
  }

  // a9: energy lattice.  With N = R^eq - rho E theta I, Eqs. (geq2mom),
  // (eosIdealGas) and Mayer give N = P theta I + rho (h + theta) u u
  // (h = H + u^2/2), so the ansatz of Eqs. (gansatz)-(RcorrectionPrime) reads
  //   G_i(m) = w_i(theta) [E_i + m . c_i / theta] + B_i . Z,
  //   E_i = rho E - 3P/2 + rho |c_i|^2 / 2 + Gc ((u . c_i)^2 / theta - u^2),
  //   Z_a = (1 - 3 theta) P / 2 + (1 - 3 theta) Gc u_a^2,  Gc = rho (h + theta) / (2 theta),
  // whose deviation from the reference rest state is again small.  G is
  // affine in m, so Eq. (g) becomes g' = (1 - omega) g + omega G(q^eq)
  // + w_i c_i . K / theta with K = (omega - omega_1)(q^b - q^eq)
  // + omega_1 rho sum_a H_a Y_a V_a + (1/2)(2 - omega_1) P sum_a H_a grad Y_a
  // (Eqs. gstareq1mom, interdiffusion, corrFourier without their
  // 1/(omega - omega_1)); the last, non-local term is deferred.
  {
    const Real theta = th.theta, thr = p.thr, dth = th.dtheta;
    const Real hk = enthalpy<M, Real>(p, th) + Real(0.5) * th.usq;     // h = H + u^2/2
    const Real inv_theta = Real(1) / theta;
    const Real Gc = rho * (hk + theta) * Real(0.5) * inv_theta;
    const Real* u = th.u;
    const Real E0 = (p.RL[M + 1] + rhoE_dev) - Real(1.5) * P - Gc * th.usq;
    const Real dE0 = rhoE_dev - Real(1.5) * th.dP - Gc * th.usq;
    Real dZ[3];
    {
      const Real z1 = Real(1) - Real(3) * theta;
      const Real zb = Real(0.5) * (z1 * th.dP - Real(3) * dth * p.Pr);
#pragma unroll
      for (int c = 0; c < 3; ++c) dZ[c] = zb + z1 * Gc * u[c] * u[c];
    }
    Real mvec[3], qt[3];
    {
      Real dP6[6];   // Pi - P^eq from deviations
      dP6[0] = p.cPi + S[0] - th.dP - rho * u[0] * u[0];
      dP6[1] = p.cPi + S[1] - th.dP - rho * u[1] * u[1];
      dP6[2] = p.cPi + S[2] - th.dP - rho * u[2] * u[2];
      dP6[3] = S[3] - rho * u[0] * u[1];
      dP6[4] = S[4] - rho * u[0] * u[2];
      dP6[5] = S[5] - rho * u[1] * u[2];
      const Real qeq[3] = {hk * j[0], hk * j[1], hk * j[2]};
      qt[0] = qeq[0] * inv_theta; qt[1] = qeq[1] * inv_theta; qt[2] = qeq[2] * inv_theta;
      Real qb[3];
      qb[0] = q[0] - (u[0] * dP6[0] + u[1] * dP6[3] + u[2] * dP6[4]);
      qb[1] = q[1] - (u[0] * dP6[3] + u[1] * dP6[1] + u[2] * dP6[5]);
      qb[2] = q[2] - (u[0] * dP6[4] + u[1] * dP6[5] + u[2] * dP6[2]);
      Real hyv[3] = {Real(0), Real(0), Real(0)};
      const Real rY = p.weak ? rho / th.rho_sp : Real(1);   // rho Y_a = rY * rho_a
      if (!p.tvar) {
#pragma unroll
        for (int a = 0; a < M; ++a) {
          const Real sv = p.Cp_a[a] * th.rho_a[a];          // H_a / T
#pragma unroll
          for (int c = 0; c < 3; ++c) hyv[c] += sv * V[a][c];
        }
      } else {
#pragma unroll
        for (int a = 0; a < M; ++a) {
          const Real sv = enthalpy_a(p, a, T) * th.rho_a[a] / T;
#pragma unroll
          for (int c = 0; c < 3; ++c) hyv[c] += sv * V[a][c];
        }
      }
      const Real c1 = om1 * T * rY, dw = om - om1;
#pragma unroll
      for (int c = 0; c < 3; ++c) mvec[c] = (om * qeq[c] + dw * (qb[c] - qeq[c]) + c1 * hyv[c]) * inv_theta;
    }
    if constexpr (EQ) {
      // this node's equilibrium record, for the receivers of its populations
      if (active) {
        EqRec<M> r;
#pragma unroll
        for (int c = 0; c < 3; ++c) { r.u[c] = u[c]; r.usp[c] = th.u_sp[c]; }
        r.dth = dth; r.dT = th.dT; r.drho = rho_dev; r.drhoE = rhoE_dev;
        r.Gq = Gc * inv_theta; r.hq = hk * rho * inv_theta;
#pragma unroll
        for (int a = 0; a < M; ++a) r.ra[a] = th.rho_a_dev[a];
        store_rec<M>(eq_rec_buf(side, N, p.rec_w, PAR), n, p.rec_w, p.weak, r);
      }
    }
    const Real w0 = Real(1) - theta, w1 = Real(0.5) * theta;          // Eq. (w0)
    const Real r0 = Real(1) - thr, r1 = Real(0.5) * thr;
    const Real d0 = -dth, d1 = Real(0.5) * dth;
    Real s_g = Real(0);
    const Nbr nbw = opaque(nb);
    const long long nw = kOpaqueStore<M, Store> ? opaque_idx(n) : n;
    // The equilibrium deviation depends on c_i only through |c_ia| and
    // (u . c_i)^2, so it is the same for i and opp(i): one evaluation per
    // pair of opposite velocities; the flux term w_i c_i . m changes sign.
    static_for<0, 13>([&](auto I_) {
      constexpr int i = decltype(I_)::value, o = Q - 1 - i;
      constexpr int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
      long long node_i, node_o; int slot_i, slot_o;
      aa_write_loc<WALL>(PAR, nbw, nw, i, node_i, slot_i);
      aa_write_loc<WALL>(PAR, nbw, nw, o, node_o, slot_o);
      const Real uc = dotc<Real, i>(th.u);
      const Real cc = Real(0.5) * Real(c2_of(i));
      const Real ucu = Gc * uc * uc * inv_theta;
      const Real Ei = E0 + cc * rho + ucu;
      const Real dEi = dE0 + cc * rho_dev + ucu;
      const Real wx = cx ? w1 : w0, wy = cy ? w1 : w0, wz = cz ? w1 : w0;
      const Real rx = cx ? r1 : r0, ry = cy ? r1 : r0, rz = cz ? r1 : r0;
      const Real dx = cx ? d1 : d0, dy = cy ? d1 : d0, dz = cz ? d1 : d0;
      const Real wi = wx * wy * wz;
      const Real dwi = dx * wy * wz + rx * dy * wz + rx * ry * dz;
      const Real e = dwi * Ei + rx * ry * rz * dEi + BdotZ<Real, i>(dZ);
      s_g += e + e;
      const Real fl = wi * dotc<Real, i>(mvec);
      const Real gvi = cell(M + 1, i, cx), gvo = cell(M + 1, o, -cx);
      const Real out_i = gvi + om * (e - gvi) + fl;
      const Real out_o = gvo + om * (e - gvo) - fl;
      if (active) {
        const Real sq = EQ ? wi * dotc<Real, i>(qt) : Real(0);
        codec_store<Store, Real>(p, pop_at((M + 1) * Q + slot_i, node_i), 0, M + 1, EQ ? out_i - (e + sq) : out_i);
        codec_store<Store, Real>(p, pop_at((M + 1) * Q + slot_o, node_o), 0, M + 1, EQ ? out_o - (e - sq) : out_o);
      }
    });
    long long node; int slot;
    aa_write_loc<WALL>(PAR, nbw, nw, 13, node, slot);
    const Real gv = cell(M + 1, 13, 0);
    const Real e13 = rhoE_dev - s_g;
    const Real out = gv + om * (e13 - gv);
    if (active) codec_store<Store, Real>(p, pop_at((M + 1) * Q + slot, node), 0, M + 1, EQ ? out - e13 : out);
  }

  // a7: species, Eqs. (SMlbm), (fstar1).  Equilibrium deviation
  //   e_ai = rho_a (Psi_i(u, R_a T) - W_ai) + (rho_a - RL_a) W_ai,
  // F_ai = sum_b kap_ab [Psi_i(u, R_b T) - Psi_i(u + V_b, R_b T)], kap_ab = Y_a rho_b / tau_ab,
  // the bracket from exact per-axis differences
  //   Psi_0(xi) - Psi_0(xi + V) = V (2 xi + V) = v,  Psi_{+-1}: -v/2 -+ V/2.
  {
    const Real x2[3] = {th.u_sp[0] * th.u_sp[0], th.u_sp[1] * th.u_sp[1], th.u_sp[2] * th.u_sp[2]};
    Real zr[M], dz[M], ev[M][3];
#pragma unroll
    for (int b = 0; b < M; ++b) {
      zr[b] = p.R_a[b] * p.Tr;
      dz[b] = p.R_a[b] * th.dT;
#pragma unroll
      for (int c = 0; c < 3; ++c) ev[b][c] = V[b][c] * (Real(2) * th.u_sp[c] + V[b][c]);
    }
    // F_ai = Y_a sum_b (1/tau_ab) rho_b Dif_bi with 1/tau_ab = R_U T m C_ab:
    // the constants C_ab stay in the parameter block, no M x M array is live.
    Real tY[M];
    {
      const Real tm = p.R_U * th.T * th.m;
#pragma unroll
      for (int a = 0; a < M; ++a) tY[a] = tm * th.Y[a];
    }
    Real s_e[M], s_F[M];
#pragma unroll
    for (int a = 0; a < M; ++a) { s_e[a] = Real(0); s_F[a] = Real(0); }
    const Nbr nbw = opaque(nb);
    const long long nw = kOpaqueStore<M, Store> ? opaque_idx(n) : n;
    // One velocity of the species update.  With many species the velocity
    // loop runs at run time: unrolled, the compiler keeps every species' axis
    // factors of all 26 velocities live at once and spills.
    auto species_velocity = [&](int i, int cx, int cy, int cz, long long node, int slot) {
      Real Dif[M];
#pragma unroll
      for (int b = 0; b < M; ++b) {
        // a = Psi(u), s = Psi(u + V) per axis; Dif = a_x a_y a_z - s_x s_y s_z
        const Real z = zr[b] + dz[b];
        const Real ax = pf_a<Real>(cx, th.u_sp[0], x2[0], z);
        const Real ay = pf_a<Real>(cy, th.u_sp[1], x2[1], z);
        const Real az = pf_a<Real>(cz, th.u_sp[2], x2[2], z);
        const Real tx = pf_v<Real>(cx, V[b][0], ev[b][0]);
        const Real ty = pf_v<Real>(cy, V[b][1], ev[b][1]);
        const Real tz = pf_v<Real>(cz, V[b][2], ev[b][2]);
        const Real sx = ax - tx, sy = ay - ty;
        Dif[b] = th.rho_a[b] * (tx * ay * az + sx * ty * az + sx * sy * tz);
      }
#pragma unroll
      for (int a = 0; a < M; ++a) {
        Real F = Real(0);
#pragma unroll
        for (int b = 0; b < M; ++b) F += p.Cab[a][b] * Dif[b];
        F *= tY[a];
        // Psi_i(u, zr + dz) - Psi_i(0, zr), telescoped over the axes
        const Real zz = zr[a] + dz[a];
        const Real rx = pf_r<Real>(cx, zr[a]), ry = pf_r<Real>(cy, zr[a]);
        const Real d = pf_da<Real>(cx, th.u_sp[0], x2[0], dz[a]) * pf_a<Real>(cy, th.u_sp[1], x2[1], zz)
                           * pf_a<Real>(cz, th.u_sp[2], x2[2], zz)
                     + rx * pf_da<Real>(cy, th.u_sp[1], x2[1], dz[a]) * pf_a<Real>(cz, th.u_sp[2], x2[2], zz)
                     + rx * ry * pf_da<Real>(cz, th.u_sp[2], x2[2], dz[a]);
        const Real e = th.rho_a[a] * d + th.rho_a_dev[a] * (rx * ry * pf_r<Real>(cz, zr[a]));
        s_e[a] += e; s_F[a] += F;
        const Real kv = species_val(a, i, cx);
        const Real out = kv + Real(2) * beta[a] * (e - kv) + (beta[a] - Real(1)) * F;
        if (active) codec_store<Store, Real>(p, pop_at(a * Q + slot, node), 0, a, EQ ? out - e : out);
      }
    };
    if constexpr (M >= LBM_SPECIES_LOOP_MIN_M) {
#pragma unroll 1
      for (int i = 0; i < Q; ++i) {
        if (i == 13) continue;
        const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
        long long node; int slot;
        if (PAR == 0 || (WALL && leaves_to_wall(nbw, i))) {
          node = nw; slot = Q - 1 - i;
        } else {
          const unsigned xs = cx < 0 ? nbw.xs[0] : (cx > 0 ? nbw.xs[2] : nbw.xs[1]);
          const unsigned ys = cy < 0 ? nbw.ys[0] : (cy > 0 ? nbw.ys[2] : nbw.ys[1]);
          const unsigned zs = cz < 0 ? nbw.zs[0] : (cz > 0 ? nbw.zs[2] : nbw.zs[1]);
          node = (long long)(zs + ys + xs); slot = i;
        }
        species_velocity(i, cx, cy, cz, node, slot);
      }
    } else if constexpr (LBM_SPECIES_PAIRS && std::is_same<Real, float>::value && M >= 2 && M <= 3) {
      // Per-axis factor tables as below; species 0 and 1 run as the two lanes
      // of paired FP32 instructions (for a pair, the lanes are species 0, 1 of
      // the same velocity), species 2 (M = 3) alone.
      //   A = Psi_c(u, z)   T = Psi_c(u) - Psi_c(u + V)   D = A - Psi_c(0, zr)   R = Psi_c(0, zr)
      float2 A2[3][3], T2[3][3], D2[3][3], R2[2];
      float A[3][3], Tt[3][3], Da[3][3], Rr[2];    // species 2 (M = 3)
      {
        const Real z0 = zr[0] + dz[0], z1 = zr[1] + dz[1];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
#pragma unroll
          for (int c = -1; c <= 1; ++c) {
            A2[ax][c + 1] = make_float2(pf_a<Real>(c, th.u_sp[ax], x2[ax], z0), pf_a<Real>(c, th.u_sp[ax], x2[ax], z1));
            T2[ax][c + 1] = make_float2(pf_v<Real>(c, V[0][ax], ev[0][ax]), pf_v<Real>(c, V[1][ax], ev[1][ax]));
            D2[ax][c + 1] = make_float2(pf_da<Real>(c, th.u_sp[ax], x2[ax], dz[0]),
                                        pf_da<Real>(c, th.u_sp[ax], x2[ax], dz[1]));
          }
        R2[0] = make_float2(pf_r<Real>(0, zr[0]), pf_r<Real>(0, zr[1]));
        R2[1] = make_float2(pf_r<Real>(1, zr[0]), pf_r<Real>(1, zr[1]));
        if constexpr (M == 3) {
          const Real z2 = zr[2] + dz[2];
#pragma unroll
          for (int ax = 0; ax < 3; ++ax)
#pragma unroll
            for (int c = -1; c <= 1; ++c) {
              A[ax][c + 1] = pf_a<Real>(c, th.u_sp[ax], x2[ax], z2);
              Tt[ax][c + 1] = pf_v<Real>(c, V[2][ax], ev[2][ax]);
              Da[ax][c + 1] = pf_da<Real>(c, th.u_sp[ax], x2[ax], dz[2]);
            }
          Rr[0] = pf_r<Real>(0, zr[2]);
          Rr[1] = pf_r<Real>(1, zr[2]);
        }
      }
      // F_a = sum_b K_ab Dif_b with K_ab = tY_a C_ab = Y_a / tau_ab
      float K[M][M];
#pragma unroll
      for (int a = 0; a < M; ++a)
#pragma unroll
        for (int b = 0; b < M; ++b) K[a][b] = tY[a] * p.Cab[a][b];
      const float2 rho2 = make_float2(th.rho_a[0], th.rho_a[1]);
      const float2 rd2 = make_float2(th.rho_a_dev[0], th.rho_a_dev[1]);
      const float2 bb2 = make_float2(Real(2) * beta[0], Real(2) * beta[1]);
      const float2 bm2 = make_float2(beta[0] - Real(1), beta[1] - Real(1));
      float2 se2 = make_float2(0.f, 0.f), sF2 = make_float2(0.f, 0.f);
      static_for<0, Q>([&](auto I_) {
        constexpr int i = decltype(I_)::value;
        if constexpr (i != 13) {
          constexpr int cx = cx_of(i) + 1, cy = cy_of(i) + 1, cz = cz_of(i) + 1;
          constexpr int kx = cx == 1 ? 0 : 1, ky = cy == 1 ? 0 : 1, kz = cz == 1 ? 0 : 1;
          long long node; int slot;
          aa_write_loc<WALL>(PAR, nbw, nw, i, node, slot);
          const float2 ayz = mul2(A2[1][cy], A2[2][cz]);
          const float2 sx = sub2(A2[0][cx], T2[0][cx]), sy = sub2(A2[1][cy], T2[1][cy]);
          const float2 in = fma2(sy, T2[2][cz], mul2(T2[1][cy], A2[2][cz]));
          const float2 dif = mul2(rho2, fma2(T2[0][cx], ayz, mul2(sx, in)));
          float dif_2 = 0.f, ayz_2 = 0.f;
          if constexpr (M == 3) {
            ayz_2 = A[1][cy] * A[2][cz];
            const float tsx = A[0][cx] - Tt[0][cx], tsy = A[1][cy] - Tt[1][cy];
            dif_2 = th.rho_a[2] * (Tt[0][cx] * ayz_2 + tsx * (Tt[1][cy] * A[2][cz] + tsy * Tt[2][cz]));
          }
          float F0 = K[0][0] * dif.x + K[0][1] * dif.y, F1 = K[1][0] * dif.x + K[1][1] * dif.y;
          if constexpr (M == 3) { F0 += K[0][2] * dif_2; F1 += K[1][2] * dif_2; }
          const float2 F = make_float2(F0, F1);
          const float2 rx = R2[kx], ry = R2[ky], rz = R2[kz];
          const float2 t1 = fma2(ry, D2[2][cz], mul2(D2[1][cy], A2[2][cz]));
          const float2 d = fma2(D2[0][cx], ayz, mul2(rx, t1));
          const float2 e = fma2(rho2, d, mul2(rd2, mul2(mul2(rx, ry), rz)));
          se2 = add2(se2, e);
          sF2 = add2(sF2, F);
          const float2 kv = make_float2(species_val(0, i, cx - 1), species_val(1, i, cx - 1));
          const float2 out = fma2(bm2, F, fma2(bb2, sub2(e, kv), kv));
          const float2 st = EQ ? sub2(out, e) : out;
          if (active) {
            codec_store<Store, Real>(p, pop_at(0 * Q + slot, node), 0, 0, st.x);
            codec_store<Store, Real>(p, pop_at(1 * Q + slot, node), 0, 1, st.y);
          }
          if constexpr (M == 3) {
            const float F2 = K[2][0] * dif.x + K[2][1] * dif.y + K[2][2] * dif_2;
            const float rx2 = Rr[kx], ry2 = Rr[ky], rz2 = Rr[kz];
            const float d2 = Da[0][cx] * ayz_2 + rx2 * (Da[1][cy] * A[2][cz] + ry2 * Da[2][cz]);
            const float e2 = th.rho_a[2] * d2 + th.rho_a_dev[2] * (rx2 * ry2 * rz2);
            s_e[2] += e2; s_F[2] += F2;
            const float kv2 = species_val(2, i, cx - 1);
            const float out2 = kv2 + Real(2) * beta[2] * (e2 - kv2) + (beta[2] - Real(1)) * F2;
            if (active) codec_store<Store, Real>(p, pop_at(2 * Q + slot, node), 0, 2, EQ ? out2 - e2 : out2);
          }
        }
      });
      s_e[0] += se2.x; s_e[1] += se2.y;
      s_F[0] += sF2.x; s_F[1] += sF2.y;
    } else if constexpr (LBM_SPECIES_AXIS_TABLES) {
      // Unrolled velocities, every product-form factor taken from per-axis
      // tables: each 1-D factor has one value per axis and c in {-1, 0, +1},
      // formed once per species instead of once per velocity.
      //   A = Psi_c(u, z)   T = Psi_c(u) - Psi_c(u + V)   D = A - Psi_c(0, zr)   R = Psi_c(0, zr)
      Real A[M][3][3], Tt[M][3][3], Da[M][3][3], Rr[M][2];
#pragma unroll
      for (int b = 0; b < M; ++b) {
        const Real z = zr[b] + dz[b];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
#pragma unroll
          for (int c = -1; c <= 1; ++c) {
            A[b][ax][c + 1] = pf_a<Real>(c, th.u_sp[ax], x2[ax], z);
            Tt[b][ax][c + 1] = pf_v<Real>(c, V[b][ax], ev[b][ax]);
            Da[b][ax][c + 1] = pf_da<Real>(c, th.u_sp[ax], x2[ax], dz[b]);
          }
        Rr[b][0] = pf_r<Real>(0, zr[b]);
        Rr[b][1] = pf_r<Real>(1, zr[b]);
      }
      static_for<0, Q>([&](auto I_) {
        constexpr int i = decltype(I_)::value;
        if constexpr (i != 13) {
          constexpr int cx = cx_of(i) + 1, cy = cy_of(i) + 1, cz = cz_of(i) + 1;
          long long node; int slot;
          aa_write_loc<WALL>(PAR, nbw, nw, i, node, slot);
          Real Dif[M];
#pragma unroll
          for (int b = 0; b < M; ++b) {
            const Real ayz = A[b][1][cy] * A[b][2][cz];
            const Real sx = A[b][0][cx] - Tt[b][0][cx], sy = A[b][1][cy] - Tt[b][1][cy];
            Dif[b] = th.rho_a[b] * (Tt[b][0][cx] * ayz + sx * (Tt[b][1][cy] * A[b][2][cz] + sy * Tt[b][2][cz]));
          }
#pragma unroll
          for (int a = 0; a < M; ++a) {
            Real F = Real(0);
#pragma unroll
            for (int b = 0; b < M; ++b) F += p.Cab[a][b] * Dif[b];
            F *= tY[a];
            const Real rx = Rr[a][cx == 1 ? 0 : 1], ry = Rr[a][cy == 1 ? 0 : 1], rz = Rr[a][cz == 1 ? 0 : 1];
            const Real d = Da[a][0][cx] * A[a][1][cy] * A[a][2][cz]
                         + rx * (Da[a][1][cy] * A[a][2][cz] + ry * Da[a][2][cz]);
            const Real e = th.rho_a[a] * d + th.rho_a_dev[a] * (rx * ry * rz);
            s_e[a] += e; s_F[a] += F;
            const Real kv = species_val(a, i, cx - 1);
            const Real out = kv + Real(2) * beta[a] * (e - kv) + (beta[a] - Real(1)) * F;
            if (active) codec_store<Store, Real>(p, pop_at(a * Q + slot, node), 0, a, EQ ? out - e : out);
          }
        }
      });
    } else {
      static_for<0, Q>([&](auto I_) {
        constexpr int i = decltype(I_)::value;
        if constexpr (i != 13) {
          long long node; int slot;
          aa_write_loc<WALL>(PAR, nbw, nw, i, node, slot);
          species_velocity(i, cx_of(i), cy_of(i), cz_of(i), node, slot);
        }
      });
    }
    long long node; int slot;
    aa_write_loc<WALL>(PAR, nbw, nw, 13, node, slot);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      const Real e = th.rho_a_dev[a] - s_e[a];
      const Real kv = species_val(a, 13, 0);
      const Real out = kv + Real(2) * beta[a] * (e - kv) - (beta[a] - Real(1)) * s_F[a];
      if (active) codec_store<Store, Real>(p, pop_at(a * Q + slot, node), 0, a, EQ ? out - e : out);
    }
  }
  if constexpr (CL) mlp.teardown();
}

// LD = 1: bulk row loads; needs Store == Real, nx a multiple of the block
// size and a grid whose blocks are whole row segments (checked by the host).
// WALL = 1: bounce-back walls normal to x (with LD = 0); WALL = 2: the
// opposed-jets frame (with LD = 0).
template <int M, class Real, class Store, int PAR, int CL = 0, int LD = 0, int WALL = 0>
__global__ void __launch_bounds__(collide_block<M, Real, CL, Store>(), collide_min_blocks<M, Real, CL, Store>())
collide_kernel(const __grid_constant__ DevParams<Real> p, Store* __restrict__ pops, Real* __restrict__ side,
               unsigned* __restrict__ err, const unsigned char* __restrict__ mlp_img,
               unsigned long long* __restrict__ mlp_stats, const __grid_constant__ PlaneOffsets po) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  collide_node<M, Real, Store, PAR, CL, LD, WALL == 1, LBM_PLANE_OFFSETS != 0, WALL == 2>(
      p, pops, side, err, mlp_img, mlp_stats, gtid(), smem_raw, po.off);
}

}  // namespace lbm
