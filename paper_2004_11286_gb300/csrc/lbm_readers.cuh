// lbm_readers.cuh -- kernels that read or replace the state between steps:
// observables (get_moments) and natural-layout copies (checkpoint interface).
// Readers add the pending deferred terms of the last step, so what they see
// is the exact post-streaming state.
#pragma once

#include "lbm_stencil.cuh"
#include "lbm_mlp.cuh"

namespace lbm {

// FP64 species and momentum-lattice moments of node n read again from the
// stored populations (with their pending terms and shifts), for the FP64
// re-solve of an ill-conditioned system in the FP32 paths (Eqs. rhoMATCH,
// uMATCH or rhoSPEC, uSPEC).  Out of line: only those nodes run it.
template <int M, class Real, class Store>
__device__ __noinline__ void state_moments64(const DevParams<Real>& p, const Store* __restrict__ pops,
                                             const Real* __restrict__ side, int parity, long long n,
                                             SpMoments64<M>* out) {
  const long long N = p.N;
  const Nbr nb = make_nbr(p, n);
  SpMoments64<M> m;
  double rf = 0.0, jf[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int a = 0; a < M; ++a) { m.rho_a[a] = 0.0; m.ja[a][0] = m.ja[a][1] = m.ja[a][2] = 0.0; }
  static_for<0, Q>([&](auto I_) {
    constexpr int i = decltype(I_)::value;
    constexpr int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
    long long node; int slot;
    aa_read_loc<true>(parity, nb, n, i, node, slot);
    Real cf, cg, sh[M + 2];
    incoming_terms<M, Real, Store, i>(p, side, nb, n, parity, cf, cg, sh);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      const double v = (double)codec_load<Store, Real>(p, pops, (a * Q + slot) * N + node, a) + (double)sh[a];
      m.rho_a[a] += v;
      m.ja[a][0] += cx * v; m.ja[a][1] += cy * v; m.ja[a][2] += cz * v;
    }
    const double fv = (double)codec_load<Store, Real>(p, pops, (M * Q + slot) * N + node, M) + (double)cf
                    + (double)sh[M];
    rf += fv;
    jf[0] += cx * fv; jf[1] += cy * fv; jf[2] += cz * fv;
  });
#pragma unroll
  for (int a = 0; a < M; ++a) m.rho_a[a] += p.RL64[a];
  if (!p.weak) {
    const double rho = p.RL64[M] + rf;
    double ro = 0.0, o[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < M; ++a)
      if (a != p.slaved) { ro += m.rho_a[a]; o[0] += m.ja[a][0]; o[1] += m.ja[a][1]; o[2] += m.ja[a][2]; }
#pragma unroll
    for (int a = 0; a < M; ++a)
      if (a == p.slaved) {
        m.rho_a[a] = rho - ro;
#pragma unroll
        for (int c = 0; c < 3; ++c) m.ja[a][c] = jf[c] - o[c];
      }
    m.rho_sp = rho;
#pragma unroll
    for (int c = 0; c < 3; ++c) m.u[c] = jf[c] / rho;
  } else {
    double rs = 0.0, js[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < M; ++a) { rs += m.rho_a[a]; js[0] += m.ja[a][0]; js[1] += m.ja[a][1]; js[2] += m.ja[a][2]; }
    m.rho_sp = rs;
#pragma unroll
    for (int c = 0; c < 3; ++c) m.u[c] = js[c] / rs;
  }
  *out = m;
}

// Observables: rho, u, T, P, X_a, Y_a, V_a (Sec. 2.1, Eq. temperature2, Eq. transform12).
template <int M, class Real, class Store>
__global__ void __launch_bounds__(BLOCK)
moments_kernel(const DevParams<Real> p, const Store* __restrict__ pops, const Real* __restrict__ side,
               int parity, double* __restrict__ out) {
  const long long n = gtid();
  if (n >= p.N) return;
  const long long N = p.N;
  const Nbr nb = make_nbr(p, n);
  Real rdev[M], ja[M][3], rho_dev, j[3], rhoE_dev;
  load_state_moments<M, Real, Store>(p, pops, side, parity, nb, n, rdev, ja, rho_dev, j, rhoE_dev);
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
  auto moments64 = [&](SpMoments64<M>& m) { state_moments64<M, Real, Store>(p, pops, side, parity, n, &m); };
  sm_solve<M, Real>(p, th, itab, ja, J, moments64);
  // rho, T and P leave as the reference value plus the state's deviation,
  // summed in FP64, so the output carries the deviation's own precision
  // rather than the rounding of the full value in the arithmetic type.
  out[0 * N + n] = (double)p.RL[M] + (double)th.rho_dev;
  out[1 * N + n] = (double)th.u[0];
  out[2 * N + n] = (double)th.u[1];
  out[3 * N + n] = (double)th.u[2];
  out[4 * N + n] = (double)p.Tr + (double)th.dT;
  out[5 * N + n] = (double)p.Pr + (double)th.dP;
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

// Natural-layout full populations: f = b + d (+ the pending deferred term).
template <int M, class Real, class Store>
__global__ void __launch_bounds__(BLOCK_LIGHT)
get_pops_kernel(const DevParams<Real> p, const Store* __restrict__ pops, const Real* __restrict__ side,
                const double* __restrict__ base, int parity, double* __restrict__ out) {
  const long long n = gtid();
  if (n >= p.N) return;
  const long long N = p.N;
  const Nbr nb = make_nbr(p, n);
  static_for<0, Q>([&](auto I_) {
    constexpr int i = decltype(I_)::value;
    long long node; int slot;
    aa_read_loc<true>(parity, nb, n, i, node, slot);
    Real cf, cg, sh[M + 2];
    incoming_terms<M, Real, Store, i>(p, side, nb, n, parity, cf, cg, sh);
    for (int L = 0; L < M + 2; ++L) {
      double v = (double)codec_load<Store, Real>(p, pops, (L * Q + slot) * N + node, L) + (double)sh[L];
      if (L == M) v += (double)cf;
      if (L == M + 1) v += (double)cg;
      out[(L * Q + i) * N + n] = base[L * Q + i] + v;
    }
  });
}

// 16-bit storage: each node's equilibrium record (lbm_eqcodec.cuh) from
// natural-layout full populations, into record buffer `buf`.
template <int M>
__global__ void __launch_bounds__(BLOCK_LIGHT)
rec_from_pops_kernel(const DevParams<double> p, float* __restrict__ side, int buf, const double* __restrict__ in) {
  const long long n = gtid();
  if (n >= p.N) return;
  const long long N = p.N;
  double ra[M], jsp[3] = {0.0, 0.0, 0.0}, rho = 0.0, j[3] = {0.0, 0.0, 0.0}, rhoE = 0.0;
#pragma unroll
  for (int a = 0; a < M; ++a) ra[a] = 0.0;
  for (int i = 0; i < Q; ++i) {
    const int c[3] = {cx_of(i), cy_of(i), cz_of(i)};
    for (int a = 0; a < M; ++a) {
      const double v = in[(a * Q + i) * N + n];
      ra[a] += v;
      for (int d = 0; d < 3; ++d) jsp[d] += c[d] * v;
    }
    const double f = in[(M * Q + i) * N + n];
    rho += f;
    for (int d = 0; d < 3; ++d) j[d] += c[d] * f;
    rhoE += in[((M + 1) * Q + i) * N + n];
  }
  double usp[3];
  if (!p.weak) {
    double o = 0.0;
    for (int a = 0; a < M; ++a) if (a != p.slaved) o += ra[a];
    ra[p.slaved] = rho - o;                                     // Eq. (rhoMATCH)
    for (int d = 0; d < 3; ++d) usp[d] = j[d] / rho;
  } else {
    double rs = 0.0;
    for (int a = 0; a < M; ++a) rs += ra[a];
    for (int d = 0; d < 3; ++d) usp[d] = jsp[d] / rs;          // Eq. (uSPEC)
  }
  store_rec<M>(eq_rec_buf(side, N, p.rec_w, buf), n, p.rec_w, p.weak, eq_record64<M>(p, ra, rho, j, rhoE, usp));
}

// Replaces the state by natural-layout full populations (no terms pending).
// With 16-bit storage the senders' records must be in place (rec_from_pops_kernel)
// and no deferred terms pending.
template <int M, class Real, class Store>
__global__ void __launch_bounds__(BLOCK_LIGHT)
set_pops_kernel(const DevParams<Real> p, Store* __restrict__ pops, const Real* __restrict__ side,
                const double* __restrict__ base, int parity, const double* __restrict__ in) {
  const long long n = gtid();
  if (n >= p.N) return;
  const long long N = p.N;
  const Nbr nb = make_nbr(p, n);
  static_for<0, Q>([&](auto I_) {
    constexpr int i = decltype(I_)::value;
    long long node; int slot;
    aa_read_loc<true>(parity, nb, n, i, node, slot);
    Real sh[M + 2];
#pragma unroll
    for (int L = 0; L < M + 2; ++L) sh[L] = Real(0);
    if constexpr (kEqCodec<Store, Real>) {
      Real cf, cg;
      eq_incoming<M, i, true>(p, side, nb, n, parity, cf, cg, sh);
    }
    for (int L = 0; L < M + 2; ++L)
      codec_store<Store, Real>(p, pops, (L * Q + slot) * N + node, L,
                               (Real)((in[(L * Q + i) * N + n] - base[L * Q + i]) - (double)sh[L]));
  });
}

// Training pairs of the learned closure at every node: the network's
// features (lbm_mlp.cuh) and its exact target, the correction of the exact
// normalised fluxes J_a / s of the J-form system of Eq. (transform12)
// (solved in FP64) to their one-sweep Jacobi estimate.
template <int M, class Real, class Store>
__global__ void __launch_bounds__(BLOCK)
closure_samples_kernel(const DevParams<Real> p, const Store* __restrict__ pops, const Real* __restrict__ side,
                       int parity, float* __restrict__ feat, float* __restrict__ tgt) {
  using Dm = MlpDims<M>;
  const long long n = gtid();
  if (n >= p.N) return;
  const Nbr nb = make_nbr(p, n);
  Real rdev[M], ja[M][3], rho_dev, j[3], rhoE_dev;
  load_state_moments<M, Real, Store>(p, pops, side, parity, nb, n, rdev, ja, rho_dev, j, rhoE_dev);
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
  Real itab[M][M], r[M][3], sr = Real(0);
  const Real tm = p.R_U * th.T * th.m;
#pragma unroll
  for (int a = 0; a < M; ++a) {
#pragma unroll
    for (int b = 0; b < M; ++b) itab[a][b] = tm * p.Cab[a][b];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      r[a][c] = ja[a][c] - th.rho_a[a] * th.u_sp[c];
      sr = fmax(sr, fabs(r[a][c]));
    }
  }
  const Real inv_s = sr > Real(0) ? Real(1) / sr : Real(0);
  float f[Dm::F];
  sm_feature_values<M, Real>(p, th, itab, r, inv_s, f);
#pragma unroll
  for (int k = 0; k < Dm::F; ++k) feat[n * Dm::F + k] = f[k];
  double A64[M][M], r64[M][3], J64[M][3];
  const double T = (double)th.T, m = (double)th.m;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    double diag = 1.0;
#pragma unroll
    for (int b = 0; b < M; ++b) {
      if (b != a) {
        const double it = (double)p.R_U * T * m * p.Cab64[a][b];
        diag += 0.5 * it * (double)th.Y[b];
        A64[a][b] = -0.5 * it * (double)th.Y[a];
      }
    }
    A64[a][a] = diag;
#pragma unroll
    for (int c = 0; c < 3; ++c) r64[a][c] = (double)(r[a][c] * inv_s);
  }
  double J0[M][3];                       // one-sweep Jacobi estimate (before the elimination)
#pragma unroll
  for (int a = 0; a < M; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) J0[a][c] = r64[a][c] / A64[a][a];
  sm_eliminate<M, double>(A64, r64, J64);
#pragma unroll
  for (int k = 0; k < Dm::O; ++k)
    tgt[n * Dm::O + k] = k < 3 * M ? (float)(J64[k / 3][k % 3] - J0[k / 3][k % 3]) : 0.0f;
}

}  // namespace lbm
