// lbm_kernels.cuh -- the step's launch sequence, initialisation, conservation
// sums and the host launchers (templated; instantiated per species count and
// precision in inst_m*_*.cu).
//
// One time step is three launches:
//   collide_kernel  adds the deferred non-local terms of the previous step to
//                   the arriving populations, then moments, closure,
//                   Stefan-Maxwell solve, species/f/g collisions and the
//                   in-place AA write; writes this node's side fields
//                   (lbm_collide.cuh)
//   grad_GK_kernel  G_alpha = (1/omega - 1/2) d_alpha Phi_alpha, K = s grad C_p
//   grad_X_kernel   X_alpha = -d_alpha G_alpha             (Eq. Xalpha; lbm_stencil.cuh)
// All non-local inputs are built from time-t moments (synchronous), and each
// population carries its full time-t collision before it is used.
#pragma once

#include "lbm_collide.cuh"
#include "lbm_batch.cuh"
#include "lbm_readers.cuh"
#include "lbm_frame.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// Equilibrium initialisation (Eqs. 27eq, fixed, feq, gieq), evaluated in FP64
// as full populations and stored as deviations from the base table.
// ---------------------------------------------------------------------------
// 16-bit storage: the record of every node from the fields (into buffer 1,
// which the first step, of parity 0, reads).
template <int M>
__global__ void __launch_bounds__(BLOCK_LIGHT)
init_rec_kernel(const DevParams<double> p, float* __restrict__ side, const double* __restrict__ Xin,
                const double* __restrict__ uin, const double* __restrict__ Tin, const double* __restrict__ Pin) {
  const long long n = gtid();
  if (n >= p.N) return;
  const long long N = p.N;
  double X[M], u[3], m = 0.0;
#pragma unroll
  for (int a = 0; a < M; ++a) { X[a] = Xin[a * N + n]; m += X[a] * p.mass[a]; }
#pragma unroll
  for (int c = 0; c < 3; ++c) u[c] = uin[c * N + n];
  const double T = Tin[n], rho = Pin[n] * m / (p.R_U * T);
  double ra[M], Umix = 0.0;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    const double Y = X[a] * p.mass[a] / m;
    ra[a] = Y * rho;
    Umix += Y * U_a64(p, a, T);
  }
  const double j[3] = {rho * u[0], rho * u[1], rho * u[2]};
  const double rhoE = rho * (Umix + 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  store_rec<M>(eq_rec_buf(side, N, p.rec_w, 1), n, p.rec_w, p.weak, eq_record64<M>(p, ra, rho, j, rhoE, u));
}

// With 16-bit storage the stored value of each population is its deviation
// minus the shift of its sender's record (init_rec_kernel; p32 gives the
// FP32 constants the shifts are formed with).
template <int M, class Store>
__global__ void __launch_bounds__(BLOCK_LIGHT)
init_kernel(const DevParams<double> p, const DevParams<float> p32, Store* __restrict__ pops,
            const float* __restrict__ side, const double* __restrict__ base,
            const double* __restrict__ Xin, const double* __restrict__ uin,
            const double* __restrict__ Tin, const double* __restrict__ Pin) {
  const long long n = gtid();
  if (n >= p.N) return;
  const long long N = p.N;
  // shifts [i][L] of the senders' equilibria (zero without the shifted codec)
  float sh[Q][M + 2];
  if constexpr (kEqCodec<Store, float>) {
    const Nbr nb = make_nbr(p, n);
    static_for<0, Q>([&](auto I_) {
      constexpr int i = decltype(I_)::value;
      float cf, cg;
      eq_incoming<M, i, true>(p32, side, nb, n, 0, cf, cg, sh[i]);
    });
  } else {
    for (int i = 0; i < Q; ++i)
      for (int L = 0; L < M + 2; ++L) sh[i][L] = 0.0f;
  }
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
  double Umix = Cv * T, Hmix = Cp * T;                    // constant heats
  if (p.tvar) {                                           // Eqs. specUa, specHa, Umix, specH
    Umix = 0.0; Hmix = 0.0;
#pragma unroll
    for (int a = 0; a < M; ++a) { Umix += Y[a] * U_a64(p, a, T); Hmix += Y[a] * H_a64(p, a, T); }
  }
  const double rhoE = rho * (Umix + 0.5 * usq);
#pragma unroll
  for (int a = 0; a < M; ++a) {
    const double ra = Y[a] * rho, ze = p.R_a[a] * T;
    const Triplet<double> tx = psi_triplet(u[0], ze), ty = psi_triplet(u[1], ze), tz = psi_triplet(u[2], ze);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double v = ra * tri(tx, cx_of(i)) * tri(ty, cy_of(i)) * tri(tz, cz_of(i));
      codec_store<Store, double>(p, pops, (a * Q + i) * N + n, a, v - base[a * Q + i] - (double)sh[i][a]);
    }
  }
  {
    const double ze = R * T;
    const Triplet<double> tx = psi_triplet(u[0], ze), ty = psi_triplet(u[1], ze), tz = psi_triplet(u[2], ze);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double v = rho * tri(tx, cx_of(i)) * tri(ty, cy_of(i)) * tri(tz, cz_of(i));
      codec_store<Store, double>(p, pops, (M * Q + i) * N + n, M, v - base[M * Q + i] - (double)sh[i][M]);
    }
  }
  {
    const double theta = R * T, hk = Hmix + 0.5 * usq;
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
      codec_store<Store, double>(p, pops, ((M + 1) * Q + i) * N + n, M + 1,
                                 v - base[(M + 1) * Q + i] - (double)sh[i][M + 1]);
    });
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
diag_partial_kernel(const DevParams<Real> p, const Store* __restrict__ pops, const Real* __restrict__ side,
                    int parity, double* __restrict__ partials) {
  constexpr int NV = M + 5;
  __shared__ double red[DIAG_BLOCK / 32][NV];
  const long long n = gtid();
  // A node's 27 deviations are summed in the arithmetic type (they are the
  // stored values, already of that precision), the nodes' sums in FP64.
  double v[NV];
#pragma unroll
  for (int s = 0; s < NV; ++s) v[s] = 0.0;
  if (n < p.N) {
    const long long N = p.N;
    const Nbr nb = make_nbr(p, n);
    Real w[NV];
#pragma unroll
    for (int s = 0; s < NV; ++s) w[s] = Real(0);
    static_for<0, Q>([&](auto I_) {
      constexpr int i = decltype(I_)::value;
      long long node; int slot;
      aa_read_loc<true>(parity, nb, n, i, node, slot);
      Real cf, cg, sh[M + 2];
      incoming_terms<M, Real, Store, i>(p, side, nb, n, parity, cf, cg, sh);
#pragma unroll
      for (int a = 0; a < M; ++a) w[a] += codec_load<Store, Real>(p, pops, (a * Q + slot) * N + node, a) + sh[a];
      const Real fv = codec_load<Store, Real>(p, pops, (M * Q + slot) * N + node, M) + cf + sh[M];
      w[M] += fv;
      if constexpr (cx_of(i) != 0) w[M + 1] += cx_of(i) * fv;
      if constexpr (cy_of(i) != 0) w[M + 2] += cy_of(i) * fv;
      if constexpr (cz_of(i) != 0) w[M + 3] += cz_of(i) * fv;
      w[M + 4] += codec_load<Store, Real>(p, pops, ((M + 1) * Q + slot) * N + node, M + 1) + cg + sh[M + 1];
    });
#pragma unroll
    for (int s = 0; s < NV; ++s) v[s] = (double)w[s];
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
  static constexpr bool EQ = kEqCodec<Store, Real>;
  static cudaError_t init(const LaunchCtx& c, const double* X, const double* u, const double* T,
                          const double* Pr) {
    if constexpr (EQ)
      init_rec_kernel<M><<<grid_for(c.N, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(*c.p64, (float*)c.side, X, u, T, Pr);
    init_kernel<M, Store><<<grid_for(c.N, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(
        *c.p64, *c.p32, (Store*)c.pops, (const float*)c.side, c.base, X, u, T, Pr);
    return cudaGetLastError();
  }
  template <int CL, int LD, int WALL = 0>
  static void collide_launch(const LaunchCtx& c, int parity, Real* side) {
    constexpr int BS = collide_block<M, Real, CL, Store>();
    constexpr size_t smem = collide_smem<M, Real, CL, LD, Store>();
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(collide_kernel<M, Real, Store, 0, CL, LD, WALL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      cudaFuncSetAttribute(collide_kernel<M, Real, Store, 1, CL, LD, WALL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      attr = true;
    }
    PlaneOffsets po;
    for (int k = 0; k < (M + 2) * Q; ++k) po.off[k] = (long long)k * c.N * (long long)sizeof(Store);
    if (parity == 0)
      collide_kernel<M, Real, Store, 0, CL, LD, WALL><<<grid_for(c.N, BS), BS, smem, c.stream>>>(
          P(c), (Store*)c.pops, side, c.err, c.mlp_img, c.mlp_stats, po);
    else
      collide_kernel<M, Real, Store, 1, CL, LD, WALL><<<grid_for(c.N, BS), BS, smem, c.stream>>>(
          P(c), (Store*)c.pops, side, c.err, c.mlp_img, c.mlp_stats, po);
  }
  // Bulk row loads where the blocks are whole row segments and the stage
  // holds the stored type (FP64, FP32).
  template <int CL>
  static void collide(const LaunchCtx& c, int parity, Real* side) {
    // Walls normal to x (bounce-back), the opposed-jets frame: register
    // loads, exact closure (the host refuses both with the network closure).
    if constexpr (CL == 0) {
      if (P(c).wall_x) {
        collide_launch<0, 0, 1>(c, parity, side);
        return;
      }
      if constexpr (!EQ) {
        if (P(c).frame) {
          collide_launch<0, 0, 2>(c, parity, side);
          return;
        }
      }
    }
    if constexpr (CL == 0 && LBM_COLLIDE_BULK && M >= LBM_COLLIDE_BULK_MIN_M && std::is_same<Real, Store>::value) {
      if (P(c).nx % collide_block<M, Real, 0, Store>() == 0) {
        collide_launch<0, 1>(c, parity, side);
        return;
      }
    }
    collide_launch<CL, 0>(c, parity, side);
  }
  static cudaError_t step(const LaunchCtx& c, int parity) {
    Real* side = (Real*)c.side;
    if (c.ev) cudaEventRecord(c.ev[0], c.stream);
    if constexpr (kMlpOk<M, Real>) {
      if (c.closure) collide<1>(c, parity, side);
      else collide<0>(c, parity, side);
    } else {
      collide<0>(c, parity, side);
    }
    // opposed-jets frame: the populations and side fields of the frame nodes
    const bool frame = P(c).frame != 0;
    const unsigned fgrid = frame ? grid_for(frame_count(P(c)), BLOCK_LIGHT) : 0u;
    if (frame) {
      frame_pops_kernel<M, Real, Store><<<fgrid, BLOCK_LIGHT, 0, c.stream>>>(P(c), (Store*)c.pops, c.jet, c.base,
                                                                             parity);
      frame_side_kernel<Real><<<fgrid, BLOCK_LIGHT, 0, c.stream>>>(P(c), side, 0);
    }
    if (c.ev) cudaEventRecord(c.ev[1], c.stream);
    // Row-blocked stencils (ROWV nodes per thread) where rows split evenly.
    const bool rows = P(c).nx % ROWV == 0 && !P(c).tvar;
    if (rows) grad_GK_row_kernel<Real><<<grid_for(c.N / ROWV, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(P(c), side);
    else grad_GK_kernel<Real><<<grid_for(c.N, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(P(c), side);
    if (frame) frame_side_kernel<Real><<<fgrid, BLOCK_LIGHT, 0, c.stream>>>(P(c), side, 1);
    if (c.ev) cudaEventRecord(c.ev[2], c.stream);
    if (rows) grad_X_row_kernel<Real><<<grid_for(c.N / ROWV, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(P(c), side);
    else grad_X_kernel<Real><<<grid_for(c.N, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(P(c), side);
    if (frame) frame_side_kernel<Real><<<fgrid, BLOCK_LIGHT, 0, c.stream>>>(P(c), side, 2);
    if (c.ev) cudaEventRecord(c.ev[3], c.stream);
    return cudaGetLastError();
  }
  static cudaError_t batch_prepare() {
    constexpr size_t smem = collide_smem<M, Real, 0, 0, Store>();
    cudaFuncSetAttribute(collide_batch_kernel<M, Real, Store, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(collide_batch_kernel<M, Real, Store, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaGetLastError();
  }
  static cudaError_t batch_step(const BatchCtx& b, int parity) {
    constexpr int BS = collide_block<M, Real, 0, Store>();
    constexpr size_t smem = collide_smem<M, Real, 0, 0, Store>();
    const DevParams<Real>* prm = static_cast<const DevParams<Real>*>(b.params);
    if (parity == 0)
      collide_batch_kernel<M, Real, Store, 0><<<b.grid_c, BS, smem, b.stream>>>(prm, b.pops, b.side, b.tiles_c,
                                                                                 b.ntiles_c, b.err);
    else
      collide_batch_kernel<M, Real, Store, 1><<<b.grid_c, BS, smem, b.stream>>>(prm, b.pops, b.side, b.tiles_c,
                                                                                 b.ntiles_c, b.err);
    grad_GK_batch_kernel<Real><<<b.grid_l, b.block_l, 0, b.stream>>>(b.geom, b.side, b.tiles_l, b.ntiles_l);
    grad_X_batch_kernel<Real><<<b.grid_l, b.block_l, 0, b.stream>>>(b.geom, b.side, b.tiles_l, b.ntiles_l);
    return cudaGetLastError();
  }
  static cudaError_t samples(const LaunchCtx& c, int parity, float* feat, float* tgt) {
    closure_samples_kernel<M, Real, Store><<<grid_for(c.N, BLOCK), BLOCK, 0, c.stream>>>(
        P(c), (const Store*)c.pops, (const Real*)c.side, parity, feat, tgt);
    return cudaGetLastError();
  }
  static cudaError_t mlp_forward(const LaunchCtx& c, const float* feat, float* out, long long n) {
    constexpr int smem = mlp_smem<M, 1>();
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(mlp_forward_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      attr = true;
    }
    if (n > 0)
      mlp_forward_kernel<M><<<grid_for(n, MLP_TILE), MLP_TILE, smem, c.stream>>>(c.mlp_img, feat, out, n, c.err);
    return cudaGetLastError();
  }
  static cudaError_t mlp_pack(const LaunchCtx& c, const float* w, unsigned char* img) {
    mlp_pack_kernel<M><<<grid_for(MlpDims<M>::NW, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(w, img);
    return cudaGetLastError();
  }
  static cudaError_t moments(const LaunchCtx& c, int parity, double* out) {
    moments_kernel<M, Real, Store><<<grid_for(c.N, BLOCK), BLOCK, 0, c.stream>>>(
        P(c), (const Store*)c.pops, (const Real*)c.side, parity, out);
    return cudaGetLastError();
  }
  static cudaError_t get_pops(const LaunchCtx& c, int parity, double* out) {
    get_pops_kernel<M, Real, Store><<<grid_for(c.N, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(
        P(c), (const Store*)c.pops, (const Real*)c.side, c.base, parity, out);
    return cudaGetLastError();
  }
  static cudaError_t set_pops(const LaunchCtx& c, int parity, const double* in) {
    if constexpr (EQ)
      rec_from_pops_kernel<M><<<grid_for(c.N, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(*c.p64, (float*)c.side,
                                                                                       1 - parity, in);
    set_pops_kernel<M, Real, Store><<<grid_for(c.N, BLOCK_LIGHT), BLOCK_LIGHT, 0, c.stream>>>(
        P(c), (Store*)c.pops, (const Real*)c.side, c.base, parity, in);
    return cudaGetLastError();
  }
  static cudaError_t diag(const LaunchCtx& c, int parity, double* d_sums) {
    const unsigned nb = grid_for(c.N, DIAG_BLOCK);
    diag_partial_kernel<M, Real, Store><<<nb, DIAG_BLOCK, 0, c.stream>>>(
        P(c), (const Store*)c.pops, (const Real*)c.side, parity, c.partials);
    diag_final_kernel<<<1, DIAG_BLOCK, 0, c.stream>>>(c.partials, (int)nb, M + 5, d_sums);
    return cudaGetLastError();
  }
  static cudaError_t jet_table(const LaunchCtx& c, double* buf) {
    DevParams<double> q = *c.p64;
    q.N = 2; q.nx = 2; q.ny = 1; q.nz = 1; q.wall_x = 0; q.frame = 0;
    const size_t S = M + 2;
    double* out = buf;
    const double* zero = buf + S * Q * 2;
    const double* X = zero + S * Q;
    const double* u = X + 2 * M;
    const double* T = u + 6;
    const double* Pr = T + 2;
    init_kernel<M, double><<<1, BLOCK_LIGHT, 0, c.stream>>>(q, *c.p32, out, nullptr, zero, X, u, T, Pr);
    return cudaGetLastError();
  }
  static KernelSet make() {
    KernelSet k;
    k.init = &init; k.step = &step; k.moments = &moments; k.get_pops = &get_pops;
    k.set_pops = &set_pops; k.diag = &diag;
    k.samples = &samples; k.mlp_forward = &mlp_forward; k.mlp_pack = &mlp_pack;
    k.batch_prepare = &batch_prepare; k.batch_step = &batch_step; k.jet_table = &jet_table;
    k.launches_per_step = 3;
    k.setup_launches = EQ ? 2 : 1;
    k.collide_bs = collide_block<M, Real, 0, Store>();
    k.mlp_F = MlpDims<M>::F; k.mlp_O = MlpDims<M>::O; k.mlp_nw = MlpDims<M>::NW;
    k.mlp_img_bytes = MlpDims<M>::IMG_BYTES;
    k.mlp_step_ok = kMlpOk<M, Real> ? 1 : 0;
    return k;
  }
};

}  // namespace lbm
