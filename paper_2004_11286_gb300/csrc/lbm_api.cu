// lbm_api.cu -- C ABI (include/lbm_mix.h): parameter validation, constant
// tables, buffer binding, launch sequencing and error latching.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm_mix.h"
#include "lbm_device.cuh"
#include "lbm_eqcodec.cuh"
#include "lbm_dispatch.h"
#include "lbm_train.h"

namespace {

thread_local std::string g_create_error;

const lbm::KernelSet* select_kernels(int M, int prec) {
#define LBM_PICK(MM)                                   \
  case MM:                                             \
    switch (prec) {                                    \
      case LBM_PREC_FP64: return lbm::kernel_set_m##MM##_f64();        \
      case LBM_PREC_FP32: return lbm::kernel_set_m##MM##_f32();        \
      case LBM_PREC_FP16_STORE: return lbm::kernel_set_m##MM##_f16();  \
      case LBM_PREC_BF16_STORE: return lbm::kernel_set_m##MM##_bf16(); \
      default: return nullptr;                         \
    }
  switch (M) {
    LBM_PICK(1)
    LBM_PICK(2)
    LBM_PICK(3)
    LBM_PICK(4)
    LBM_PICK(5)
    LBM_PICK(6)
    LBM_PICK(7)
    LBM_PICK(8)
    default: return nullptr;
  }
#undef LBM_PICK
}

size_t store_elem_bytes(int prec) { return prec == LBM_PREC_FP64 ? 8 : (prec == LBM_PREC_FP32 ? 4 : 2); }
size_t side_elem_bytes(int prec) { return prec == LBM_PREC_FP64 ? 8 : 4; }

template <class Real>
void fill_params(lbm::DevParams<Real>& d, const lbm::DevParams<double>& s) {
  d.N = s.N; d.nx = s.nx; d.ny = s.ny; d.nz = s.nz; d.M = s.M; d.slaved = s.slaved; d.weak = s.weak;
  d.wall_x = s.wall_x;
  d.frame = s.frame; d.jet_y0 = s.jet_y0; d.jet_y1 = s.jet_y1;
  d.omega_is_fixed = s.omega_is_fixed; d.omega1_is_fixed = s.omega1_is_fixed;
  d.omega_fixed = (Real)s.omega_fixed; d.omega1_fixed = (Real)s.omega1_fixed;
  d.R_U = (Real)s.R_U; d.cond_bound = (Real)s.cond_bound; d.closure_bound = (Real)s.closure_bound;
  for (int a = 0; a < lbm::MAXM; ++a) {
    d.mass[a] = (Real)s.mass[a]; d.inv_mass[a] = (Real)s.inv_mass[a]; d.R_a[a] = (Real)s.R_a[a];
    d.Cv_a[a] = (Real)s.Cv_a[a]; d.Cp_a[a] = (Real)s.Cp_a[a]; d.mu[a] = (Real)s.mu[a];
    d.lam[a] = (Real)s.lam[a]; d.inv_lam[a] = (Real)s.inv_lam[a];
    for (int b = 0; b < lbm::MAXM; ++b) {
      d.phi[a][b] = (Real)s.phi[a][b]; d.Cab[a][b] = (Real)s.Cab[a][b]; d.Cab64[a][b] = s.Cab64[a][b];
    }
  }
  for (int L = 0; L < lbm::MAXM + 2; ++L) {
    d.RL[L] = (Real)s.RL[L]; d.scale[L] = (Real)s.scale[L]; d.inv_scale[L] = (Real)s.inv_scale[L];
    d.RL64[L] = s.RL[L];
  }
  for (int L = 0; L < lbm::MAXM + 2; ++L)
    for (int k = 0; k < 4; ++k) d.bref[L][k] = (Real)s.bref[L][k];
  d.rec_w = s.rec_w;
  d.tvar = s.tvar; d.nterm = s.nterm; d.Ur = (Real)s.Ur;
  for (int a = 0; a < lbm::MAXM; ++a) {
    d.Uar[a] = (Real)s.Uar[a];
    for (int k = 0; k < 3; ++k) { d.cvp[a][k] = (Real)s.cvp[a][k]; d.Uc[a][k] = (Real)s.Uc[a][k]; d.Hc[a][k] = (Real)s.Hc[a][k]; }
  }
  for (int a = 0; a < lbm::MAXM; ++a) d.Yr[a] = (Real)s.Yr[a];
  d.Tr = (Real)s.Tr; d.Rr = (Real)s.Rr; d.thr = (Real)s.thr; d.Pr = (Real)s.Pr; d.Cvr = (Real)s.Cvr;
  d.cE = (Real)s.cE; d.cPi = (Real)s.cPi; d.cS = (Real)s.cS; d.Rsp = (Real)s.Rsp;
}

// Reductions used to pick the reference state: per-block partial sums of
// nv values per node, then a fixed-order final sum (deterministic).
constexpr int RED_BLOCK = 256;
constexpr int RED_MAXV = 16;

__device__ __forceinline__ double red_warp(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void red_block_store(double (&v)[RED_MAXV], int nv, double* partials) {
  __shared__ double red[RED_BLOCK / 32][RED_MAXV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int s = 0; s < nv; ++s) {
    const double t = red_warp(v[s]);
    if (lane == 0) red[wid][s] = t;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double t = 0.0;
    for (int w = 0; w < RED_BLOCK / 32; ++w) t += red[w][threadIdx.x];
    partials[(long long)blockIdx.x * nv + threadIdx.x] = t;
  }
}

// sums of X_a (a < M), T and P over the nodes
__global__ void __launch_bounds__(RED_BLOCK)
field_partials_kernel(const double* __restrict__ X, const double* __restrict__ T, const double* __restrict__ P,
                      int M, long long N, double* __restrict__ partials) {
  double v[RED_MAXV];
  for (int s = 0; s < RED_MAXV; ++s) v[s] = 0.0;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n < N) {
    for (int a = 0; a < M; ++a) v[a] = X[a * N + n];
    v[M] = T[n];
    v[M + 1] = P[n];
  }
  red_block_store(v, M + 2, partials);
}

// zeroth moments of each of the S lattices of natural-layout full populations
__global__ void __launch_bounds__(RED_BLOCK)
pops_partials_kernel(const double* __restrict__ in, int S, long long N, double* __restrict__ partials) {
  double v[RED_MAXV];
  for (int s = 0; s < RED_MAXV; ++s) v[s] = 0.0;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n < N)
    for (int L = 0; L < S; ++L)
      for (int i = 0; i < 27; ++i) v[L] += in[((long long)L * 27 + i) * N + n];
  red_block_store(v, S, partials);
}

__global__ void __launch_bounds__(RED_BLOCK)
red_final_kernel(const double* __restrict__ partials, int nblocks, int nv, double* __restrict__ sums) {
  __shared__ double sh[RED_BLOCK];
  for (int s = 0; s < nv; ++s) {
    double t = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += RED_BLOCK) t += partials[(long long)b * nv + s];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int w = RED_BLOCK / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) sums[s] = sh[0];
    __syncthreads();
  }
}

// z-face halo of a slab: `nfields` fields of `stride` elements each, of which
// the `seg` elements from offset `off` are copied to (pack) or from (unpack)
// the contiguous buffer.
template <class T>
__global__ void __launch_bounds__(256)
halo_copy_kernel(T* __restrict__ state, T* __restrict__ buf, long long nfields, long long stride, long long off,
                 long long seg, int unpack) {
  const long long total = nfields * seg;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const long long f = k / seg, e = k - f * seg;
    T* s = state + f * stride + off + e;
    if (unpack) *s = buf[k]; else buf[k] = *s;
  }
}

template <class T>
cudaError_t halo_copy(void* state, void* buf, long long nfields, long long stride, long long off, long long seg,
                      int unpack, cudaStream_t stream) {
  const long long total = nfields * seg;
  if (total <= 0) return cudaSuccess;
  const long long want = (total + 255) / 256;
  const unsigned grid = (unsigned)(want < 65536 ? want : 65536);
  halo_copy_kernel<T><<<grid, 256, 0, stream>>>((T*)state, (T*)buf, nfields, stride, off, seg, unpack);
  return cudaGetLastError();
}

}  // namespace

// Message reported by lbm_mix_last_error(NULL) for calls without a handle.
void lbm_set_thread_error(const std::string& msg) { g_create_error = msg; }

struct lbm_mix {
  int M = 0, prec = 0, device = 0;
  long long N = 0;
  cudaStream_t stream = nullptr;
  const lbm::KernelSet* ks = nullptr;
  lbm::DevParams<double> p64{};
  lbm::DevParams<float> p32{};
  double base[(lbm::MAXM + 2) * 27] = {};   // host copy of the reference rest equilibria
  double* d_base = nullptr;
  double* d_jet = nullptr;     // opposed-jets frame: inlet equilibria (KernelSet::jet_table)
  bool has_reference = false;
  bool fixed_reference = false;    // set by lbm_mix_set_reference: init_fields keeps it
  void* pops = nullptr;
  size_t pops_bytes = 0;
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  bool owns_buffers = false;
  unsigned* d_err = nullptr;
  double* d_partials = nullptr;
  double* d_sums = nullptr;
  double* d_stage = nullptr;
  size_t stage_bytes = 0;
  long long steps = 0;
  long long launches = 0;
  long long param_version = 0;   // bumped whenever the reference state (and so the parameter block) changes
  bool initialized = false;
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;   // 4 per recorded step
  size_t ev_used = 0;
  std::string err;
  // learned closure: FP32 master weights, Adam moments, gradient, bf16 image,
  // accept/fallback counters, mini-batch scratch
  int closure = 0;
  float *d_w = nullptr, *d_m = nullptr, *d_v = nullptr, *d_g = nullptr;
  unsigned char* d_img = nullptr;
  unsigned long long* d_stats = nullptr;
  double* d_loss = nullptr;
  int adam_t = 0;
  lbm::MlpScratch z{};
  float* z_base = nullptr;
  long long z_rows = 0;

  size_t need_pops() const { return (size_t)(M + 2) * 27 * (size_t)N * store_elem_bytes(prec); }
  // side planes, then (16-bit storage) the two buffers of equilibrium records
  size_t need_scratch() const {
    if (p64.rec_w == 0) return (size_t)lbm::NSIDE * (size_t)N * side_elem_bytes(prec);
    return ((size_t)lbm::eq_rec_offset(N) + 2 * (size_t)p64.rec_w * (size_t)N) * sizeof(float);
  }
  lbm::LaunchCtx ctx() {
    lbm::LaunchCtx c;
    c.N = N; c.stream = stream; c.pops = pops; c.side = scratch; c.err = d_err;
    c.partials = d_partials; c.p64 = &p64; c.p32 = &p32; c.base = d_base; c.ev = nullptr;
    c.closure = closure; c.mlp_img = d_img; c.mlp_stats = d_stats;
    c.jet = d_jet;
    return c;
  }
  lbm_status fail(lbm_status s, const std::string& m) { err = m; return s; }
  lbm_status cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return LBM_OK;
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return LBM_ERR_CUDA;
  }
  lbm_status ensure_stage(size_t bytes) {
    if (bytes <= stage_bytes) return LBM_OK;
    if (d_stage) { cudaStreamSynchronize(stream); cudaFree(d_stage); d_stage = nullptr; stage_bytes = 0; }
    lbm_status s = cuda(cudaMalloc(&d_stage, bytes), "cudaMalloc(staging)");
    if (s == LBM_OK) stage_bytes = bytes;
    return s;
  }
  lbm_status check_flag() {
    unsigned flag = 0;
    lbm_status s = cuda(cudaMemcpyAsync(&flag, d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, stream),
                        "read error flag");
    if (s != LBM_OK) return s;
    s = cuda(cudaStreamSynchronize(stream), "stream synchronize");
    if (s != LBM_OK) return s;
    if (flag & 4u) return fail(LBM_ERR_TIMEOUT, "a tensor-core completion wait timed out");
    if (flag) return fail(LBM_ERR_NONFINITE, "a node reached non-positive density or temperature (or NaN)");
    return LBM_OK;
  }
  lbm::MlpShape mlp_shape() const { return lbm::MlpShape{128, ks->mlp_F, ks->mlp_O, 3 * M}; }
  // Mini-batch scratch for `rows` samples (grown on demand).
  lbm_status ensure_train_scratch(long long rows) {
    if (rows <= z_rows) return LBM_OK;
    if (z_base) { cudaStreamSynchronize(stream); cudaFree(z_base); z_base = nullptr; z_rows = 0; }
    const long long H = 128, O = ks->mlp_O;
    lbm_status st = cuda(cudaMalloc(&z_base, sizeof(float) * (size_t)rows * (6 * H + 2 * O)), "cudaMalloc(training)");
    if (st != LBM_OK) return st;
    float* q = z_base;
    z.h1 = q; q += rows * H; z.a1 = q; q += rows * H; z.h2 = q; q += rows * H; z.a2 = q; q += rows * H;
    z.d1 = q; q += rows * H; z.d2 = q; q += rows * H; z.out = q; q += rows * O; z.dout = q;
    z_rows = rows;
    return LBM_OK;
  }
  lbm_status repack() {
    return cuda(ks->mlp_pack(ctx(), d_w, d_img), "pack network image");
  }
  // Reference rest state (mass fractions Y, temperature T, density rho):
  // base tables of every lattice, their sums RL and the derived constants.
  lbm_status set_reference(const double* Y, double T, double rho) {
    if (!(T > 0.0) || !(rho > 0.0) || !std::isfinite(T) || !std::isfinite(rho))
      return fail(LBM_ERR_ARG, "reference state has non-positive temperature or density");
    lbm::DevParams<double>& d = p64;
    const int S = M + 2;
    auto w1 = [](int c, double z) { return c == 0 ? 1.0 - z : 0.5 * z; };
    auto W = [&](int i, double z) {
      return w1(lbm::cx_of(i), z) * w1(lbm::cy_of(i), z) * w1(lbm::cz_of(i), z);
    };
    double inv_m = 0.0, Cv = 0.0, Umix = 0.0;
    for (int a = 0; a < M; ++a) {
      inv_m += Y[a] * d.inv_mass[a]; Cv += Y[a] * d.Cv_a[a];
      Umix += Y[a] * lbm::U_a64(d, a, T);                    // Eqs. specUa, Umix
    }
    const double R = d.R_U * inv_m, th = R * T;
    for (int a = 0; a < M; ++a)
      for (int i = 0; i < 27; ++i) base[a * 27 + i] = Y[a] * rho * W(i, d.R_a[a] * T);     // Eq. (27eq) at rest
    for (int i = 0; i < 27; ++i) base[M * 27 + i] = rho * W(i, th);                      // Eq. (feq) at rest
    const double rhoE = rho * (d.tvar ? Umix : Cv * T), P = rho * th, Z = 0.5 * (1.0 - 3.0 * th) * P;
    for (int i = 0; i < 27; ++i) {                                                       // Eq. (gieq) at rest
      const int c2 = lbm::c2_of(i);
      const double E = rhoE - 1.5 * P + 0.5 * c2 * rho;
      const double BZ = c2 == 0 ? 3.0 * Z : (c2 == 1 ? -0.5 * Z : 0.0);
      base[(M + 1) * 27 + i] = W(i, th) * E + BZ;
    }
    for (int L = 0; L < lbm::MAXM + 2; ++L) {
      d.RL[L] = 0.0; d.scale[L] = 1.0; d.inv_scale[L] = 1.0;
      for (int k = 0; k < 4; ++k) d.bref[L][k] = 0.0;
    }
    for (int L = 0; L < S; ++L) {
      double sum = 0.0;
      for (int i = 0; i < 27; ++i) sum += base[L * 27 + i];
      d.RL[L] = sum;
      // 16-bit storage holds the non-equilibrium part f - f^eq of each
      // population, scaled per lattice: FP16 by 2^12 / RL (the part is a
      // small fraction of RL, so this keeps it in FP16's normal range),
      // BF16 by 1 / RL (its exponent range makes the scale immaterial).
      if (prec == LBM_PREC_FP16_STORE || prec == LBM_PREC_BF16_STORE) {
        const double s = (prec == LBM_PREC_FP16_STORE ? 4096.0 : 1.0) / std::fabs(sum);
        d.scale[L] = s;
        d.inv_scale[L] = 1.0 / s;
      }
      for (int i = 0; i < 27; ++i) d.bref[L][lbm::c2_of(i)] = base[L * 27 + i];
    }
    double Rsp = 0.0;
    for (int a = 0; a < M; ++a) Rsp += d.RL[a];
    double im = 0.0, cv = 0.0;
    for (int a = 0; a < lbm::MAXM; ++a) {
      d.Yr[a] = a < M ? d.RL[a] / Rsp : 0.0;
      if (a < M) { im += d.Yr[a] * d.inv_mass[a]; cv += d.Yr[a] * d.Cv_a[a]; }
    }
    d.Rsp = Rsp;
    d.Tr = T;
    d.Rr = d.R_U * im;
    d.thr = d.Rr * T;
    d.Pr = d.RL[M] * d.thr;
    d.Cvr = cv;
    d.cE = d.RL[M + 1] - d.RL[M] * cv * T;
    if (d.tvar) {
      // temperature-dependent heats: U_a(T_r), the reference mixture's U(T_r)
      double ur = 0.0;
      for (int a = 0; a < lbm::MAXM; ++a) {
        d.Uar[a] = a < M ? lbm::U_a64(d, a, T) : 0.0;
        if (a < M) ur += d.Yr[a] * d.Uar[a];
      }
      d.Ur = ur;
      d.cE = d.RL[M + 1] - d.RL[M] * ur;
    }
    double pix = 0.0;
    for (int i = 0; i < 27; ++i) pix += base[M * 27 + i] * (double)(lbm::cx_of(i) * lbm::cx_of(i));
    d.cPi = pix - d.RL[M] * d.thr;
    d.cS = d.RL[M] - Rsp;
    fill_params<float>(p32, d);
    p32.rho_eps = 1e-7f;
    lbm_status st = cuda(cudaMemcpyAsync(d_base, base, sizeof(double) * S * 27, cudaMemcpyHostToDevice, stream),
                         "upload reference table");
    if (st != LBM_OK) return st;
    st = cuda(cudaStreamSynchronize(stream), "synchronize");
    if (st == LBM_OK) has_reference = true;
    ++param_version;
    return st;
  }
  // Host sums of nv reduced values (partials from the kernels above).
  lbm_status reduce_to_host(int nblocks, int nv, double* out) {
    red_final_kernel<<<1, RED_BLOCK, 0, stream>>>(d_partials, nblocks, nv, d_sums);
    lbm_status st = cuda(cudaGetLastError(), "reduction kernel");
    if (st != LBM_OK) return st;
    launches += 2;
    st = cuda(cudaMemcpyAsync(out, d_sums, sizeof(double) * nv, cudaMemcpyDeviceToHost, stream), "copy sums");
    if (st != LBM_OK) return st;
    return cuda(cudaStreamSynchronize(stream), "synchronize");
  }
  lbm_status reference_from_fields(const double* dX, const double* dT, const double* dP) {
    const int nb = (int)((N + RED_BLOCK - 1) / RED_BLOCK);
    field_partials_kernel<<<nb, RED_BLOCK, 0, stream>>>(dX, dT, dP, M, N, d_partials);
    double sums[RED_MAXV];
    lbm_status st = reduce_to_host(nb, M + 2, sums);
    if (st != LBM_OK) return st;
    double Xm[lbm::MAXM], mbar = 0.0, xs = 0.0;
    for (int a = 0; a < M; ++a) { Xm[a] = sums[a] / (double)N; xs += Xm[a]; }
    for (int a = 0; a < M; ++a) { Xm[a] /= xs; mbar += Xm[a] * p64.mass[a]; }
    const double T = sums[M] / (double)N, P = sums[M + 1] / (double)N;
    double Y[lbm::MAXM];
    for (int a = 0; a < M; ++a) Y[a] = Xm[a] * p64.mass[a] / mbar;
    const double rho = P * mbar / (p64.R_U * T);
    return set_reference(Y, T, rho);
  }
  lbm_status reference_from_pops(const double* dpops) {
    const int nb = (int)((N + RED_BLOCK - 1) / RED_BLOCK);
    pops_partials_kernel<<<nb, RED_BLOCK, 0, stream>>>(dpops, M + 2, N, d_partials);
    double sums[RED_MAXV];
    lbm_status st = reduce_to_host(nb, M + 2, sums);
    if (st != LBM_OK) return st;
    double r[lbm::MAXM], tot = 0.0;
    for (int a = 0; a < M; ++a) r[a] = sums[a] / (double)N;
    const double rho = sums[M] / (double)N, rhoE = sums[M + 1] / (double)N;
    if (!p64.weak) {
      double others = 0.0;
      for (int a = 0; a < M; ++a) if (a != p64.slaved) others += r[a];
      if (rho - others > 0.0) r[p64.slaved] = rho - others;
    }
    for (int a = 0; a < M; ++a) tot += r[a];
    double Y[lbm::MAXM];
    for (int a = 0; a < M; ++a) Y[a] = r[a] / tot;
    return set_reference(Y, lbm::T_from_energy64(p64, Y, M, rhoE / rho), rho);
  }
  // No deferred non-local terms are pending for a state set from outside.
  lbm_status clear_pending() {
    const size_t es = side_elem_bytes(prec);
    return cuda(cudaMemsetAsync((char*)scratch + (size_t)lbm::SP_K * N * es, 0,
                                (size_t)(lbm::NSIDE - lbm::SP_K) * N * es, stream), "clear deferred terms");
  }
  lbm_status ready() {
    if (!pops || !scratch) return fail(LBM_ERR_STATE, "buffers not bound");
    return LBM_OK;
  }
};

// An ensemble of independent domains stepped together (one launch per kernel
// for all of them).  Each domain is a full handle (its own constants,
// reference state and buffers, carved from two shared allocations); the
// batch keeps device tables of their parameter blocks, geometry, buffer
// pointers and tiles, the launch shapes chosen by the autotuner, and a CUDA
// graph of two consecutive steps (both AA parities).
struct lbm_mix_batch {
  int nd = 0, M = 0, prec = 0;
  cudaStream_t user = nullptr;      // caller's stream
  cudaStream_t stream = nullptr;    // internal stream (capturable)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<lbm_mix*> dom;
  const lbm::KernelSet* ks = nullptr;
  void* pops_all = nullptr;
  void* side_all = nullptr;
  size_t pops_total = 0, side_total = 0;
  void* d_params = nullptr;
  size_t param_bytes = 0;            // one parameter block
  lbm::BatchGeom* d_geom = nullptr;
  void** d_ptrs = nullptr;           // [nd] pops, then [nd] side
  int2* d_tiles = nullptr;           // collide tiles, then stencil tiles for 128 and 256 threads
  int ntiles_c = 0, ntiles_128 = 0, ntiles_256 = 0;
  int grid_c = 0, grid_l = 0, block_l = 256;
  int sm_count = 0;
  unsigned* d_err = nullptr;
  std::vector<long long> uploaded;   // parameter versions on the device
  cudaGraphExec_t graph = nullptr;
  bool use_graph = true;
  // mode 0: persistent launches over the tiles of all domains;
  // mode 1: each domain's own kernels, domains spread over `nbranch`
  //         concurrent branches of the graph.
  int mode = 0, nbranch = 8;
  std::vector<cudaStream_t> branches;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  long long steps = 0, nodes = 0;
  std::string err;

  lbm_status fail(lbm_status st, const std::string& m) { err = m; return st; }
  lbm_status cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return LBM_OK;
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return LBM_ERR_CUDA;
  }
  const int2* tiles_l() const { return d_tiles + ntiles_c + (block_l == 128 ? 0 : ntiles_128); }
  int ntiles_l() const { return block_l == 128 ? ntiles_128 : ntiles_256; }
  lbm::BatchCtx ctx() const {
    lbm::BatchCtx c;
    c.stream = stream; c.params = d_params; c.geom = d_geom;
    c.pops = d_ptrs; c.side = d_ptrs + nd;
    c.tiles_c = d_tiles; c.ntiles_c = ntiles_c; c.grid_c = grid_c;
    c.tiles_l = tiles_l(); c.ntiles_l = ntiles_l(); c.grid_l = grid_l; c.block_l = block_l;
    c.err = d_err;
    return c;
  }
  void drop_graph() {
    if (graph) { cudaGraphExecDestroy(graph); graph = nullptr; }
  }
  // Parameter blocks of domains whose reference state changed since the last upload.
  lbm_status upload_params() {
    for (int d = 0; d < nd; ++d) {
      if (uploaded[d] == dom[d]->param_version) continue;
      const void* src = prec == LBM_PREC_FP64 ? (const void*)&dom[d]->p64 : (const void*)&dom[d]->p32;
      lbm_status st = cuda(cudaMemcpyAsync((char*)d_params + (size_t)d * param_bytes, src, param_bytes,
                                           cudaMemcpyHostToDevice, stream), "upload parameter block");
      if (st != LBM_OK) return st;
      uploaded[d] = dom[d]->param_version;
    }
    return cuda(cudaStreamSynchronize(stream), "synchronize");   // the host blocks must stay valid
  }
  // One domain's step (its own kernels, parameter block by value) on stream s.
  cudaError_t domain_step(int d, cudaStream_t s, int parity) {
    lbm::LaunchCtx c = dom[d]->ctx();
    c.stream = s;
    return ks->step(c, parity);
  }
  lbm_status ensure_branches() {
    if ((int)branches.size() >= nbranch) return LBM_OK;
    if (!fork && cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess)
      return fail(LBM_ERR_CUDA, "event creation failed");
    while ((int)branches.size() < nbranch) {
      cudaStream_t s;
      cudaEvent_t e;
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return fail(LBM_ERR_CUDA, "stream creation failed");
      branches.push_back(s);
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(LBM_ERR_CUDA, "event creation failed");
      joins.push_back(e);
    }
    return LBM_OK;
  }
  lbm_status build_graph() {
    drop_graph();
    if (mode == 1) {
      lbm_status st = ensure_branches();
      if (st != LBM_OK) return st;
    }
    cudaGraph_t g = nullptr;
    lbm_status st = cuda(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (st != LBM_OK) return st;
    cudaError_t e = cudaSuccess;
    if (mode == 0) {
      const lbm::BatchCtx c = ctx();
      e = ks->batch_step(c, 0);
      if (e == cudaSuccess) e = ks->batch_step(c, 1);
    } else {
      e = cudaEventRecord(fork, stream);
      for (int k = 0; k < nbranch && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(branches[k], fork, 0);
      for (int d = 0; d < nd && e == cudaSuccess; ++d) {
        e = domain_step(d, branches[d % nbranch], 0);
        if (e == cudaSuccess) e = domain_step(d, branches[d % nbranch], 1);
      }
      for (int k = 0; k < nbranch && e == cudaSuccess; ++k) {
        e = cudaEventRecord(joins[k], branches[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, joins[k], 0);
      }
    }
    cudaError_t e2 = cudaStreamEndCapture(stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda(e != cudaSuccess ? e : e2, "capture step graph");
    }
    st = cuda(cudaGraphInstantiate(&graph, g, 0), "instantiate step graph");
    cudaGraphDestroy(g);
    return st;
  }
  cudaError_t eager_step(int parity) {
    if (mode == 0) return ks->batch_step(ctx(), parity);
    for (int d = 0; d < nd; ++d) {
      cudaError_t e = domain_step(d, stream, parity);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  // nsteps steps of every domain on the internal stream (graph replays of two
  // steps where the parity allows, single launches otherwise).
  lbm_status run(int nsteps, bool graphs) {
    int done = 0;
    while (done < nsteps) {
      const int parity = (int)((steps + done) & 1);
      if (graphs && parity == 0 && nsteps - done >= 2) {
        if (!graph) {
          lbm_status st = build_graph();
          if (st != LBM_OK) return st;
        }
        lbm_status st = cuda(cudaGraphLaunch(graph, stream), "graph launch");
        if (st != LBM_OK) return st;
        done += 2;
      } else {
        lbm_status st = cuda(eager_step(parity), "batched step kernels");
        if (st != LBM_OK) return st;
        done += 1;
      }
    }
    return LBM_OK;
  }
  void advance(int nsteps) {
    steps += nsteps;
    for (lbm_mix* h : dom) {
      h->steps += nsteps;
      h->launches += (long long)nsteps * ks->launches_per_step;
    }
  }
};

extern "C" {

int lbm_mix_num_outputs(int M) { return 6 + 5 * M; }

lbm_status lbm_mix_create(const lbm_mix_params* p, void* cuda_stream, lbm_mix_t* out) {
  auto bad = [&](const std::string& m) { g_create_error = m; return LBM_ERR_ARG; };
  if (!out) return bad("out is NULL");
  *out = nullptr;
  if (!p) return bad("params is NULL");
  const int M = p->M;
  if (M < 1 || M > lbm::MAXM) return bad("M must be in 1..8");
  if (!p->molar_mass || !p->cv_molar || !p->D) return bad("molar_mass, cv_molar and D are required");
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return bad("grid dimensions must be >= 1");
  if ((long long)p->nx * p->ny * p->nz >= (1LL << 31)) return bad("grids must have fewer than 2^31 nodes");
  if (!(p->R_U > 0.0)) return bad("R_U must be > 0");
  for (int s = 0; s < 6; ++s)
    if (p->bc[s] < LBM_BC_PERIODIC || p->bc[s] > LBM_BC_OUTLET) return bad("unknown boundary type");
  // Built: periodic everywhere; bounce-back walls on both x faces with
  // periodic y and z (the closed tube); the opposed-jets frame (jets on both
  // x faces, outlets on both y faces, periodic z).
  const bool walls = p->bc[0] == LBM_BC_BOUNCEBACK;
  const bool jets = p->bc[0] == LBM_BC_JET;
  for (int s = 0; s < 6; ++s) {
    const int want = (s < 2 && walls) ? LBM_BC_BOUNCEBACK
                   : (jets && s < 2) ? LBM_BC_JET : (jets && s < 4) ? LBM_BC_OUTLET : LBM_BC_PERIODIC;
    if (p->bc[s] != want) {
      g_create_error = "boundaries built: all periodic; bounce-back on both x faces with y, z periodic; "
                       "jets on both x faces with outlets on both y faces and z periodic";
      return LBM_ERR_UNSUPPORTED;
    }
  }
  if (jets) {
    if (p->nx < 3 || p->ny < 3) return bad("the jets frame needs nx, ny >= 3");
    if (!(p->jet_y0 >= 1 && p->jet_y0 <= p->jet_y1 && p->jet_y1 <= p->ny - 1))
      return bad("nozzle rows need 1 <= jet_y0 <= jet_y1 <= ny - 1");
    if (!p->jet_X) return bad("jet_X is required with LBM_BC_JET");
    for (int k = 0; k < 2; ++k) {
      if (!(p->jet_T[k] > 0.0) || !(p->jet_P[k] > 0.0)) return bad("inlet T and P must be > 0");
      if (!std::isfinite(p->jet_u[k])) return bad("inlet velocity must be finite");
      for (int a = 0; a < M; ++a)
        if (!(p->jet_X[k * M + a] >= 0.0)) return bad("inlet mole fractions must be >= 0");
    }
    if (!(p->precision == LBM_PREC_FP64 || p->precision == LBM_PREC_FP32) || p->closure == LBM_CLOSURE_MLP ||
        p->cv_poly) {
      g_create_error = "the jets frame runs with FP64 or FP32 storage, the exact closure and constant heats";
      return LBM_ERR_UNSUPPORTED;
    }
  }
  if (p->precision < LBM_PREC_FP64 || p->precision > LBM_PREC_BF16_STORE) return bad("unknown precision");
  if (p->coupling != LBM_COUPLE_STRONG && p->coupling != LBM_COUPLE_WEAK) return bad("unknown coupling");
  if (p->closure != LBM_CLOSURE_EXACT && p->closure != LBM_CLOSURE_MLP) return bad("unknown closure");
  const int slaved = p->slaved_species < 0 ? M - 1 : p->slaved_species;
  if (slaved >= M) return bad("slaved_species out of range");
  for (int a = 0; a < M; ++a) {
    if (!(p->molar_mass[a] > 0.0) || !std::isfinite(p->molar_mass[a])) return bad("molar masses must be > 0");
    if (!(p->cv_molar[a] > 0.0)) return bad("cv_molar must be > 0");
  }
  double D[lbm::MAXM][lbm::MAXM];
  for (int a = 0; a < M; ++a)
    for (int b = 0; b < M; ++b) {
      D[a][b] = p->D[a * M + b];
      if (a != b && !(D[a][b] > 0.0)) return bad("off-diagonal D_ab must be > 0");
      if (a != b && std::fabs(D[a][b] - p->D[b * M + a]) > 1e-14 * std::fabs(D[a][b])) return bad("D must be symmetric");
    }
  for (int a = 0; a < M; ++a) {
    if (D[a][a] > 0.0) continue;
    if (M == 1) return bad("M = 1 needs D_11 > 0");
    double s = 0.0;
    for (int b = 0; b < M; ++b) if (b != a) s += std::log(D[a][b]);
    D[a][a] = std::exp(s / (M - 1));   // geometric mean of the row's off-diagonal entries
  }
  if (!(p->omega_fixed > 0.0)) {
    if (!p->mu) return bad("mu is required unless omega_fixed > 0");
    for (int a = 0; a < M; ++a) if (!(p->mu[a] > 0.0)) return bad("mu_a must be > 0");
  } else if (!(p->omega_fixed < 2.0)) return bad("omega_fixed must be in (0, 2)");
  if (!(p->omega1_fixed > 0.0)) {
    if (!p->lambda) return bad("lambda is required unless omega1_fixed > 0");
    for (int a = 0; a < M; ++a) if (!(p->lambda[a] > 0.0)) return bad("lambda_a must be > 0");
  } else if (!(p->omega1_fixed < 2.0)) return bad("omega1_fixed must be in (0, 2)");

  const bool tvar = p->cv_poly != nullptr;
  if (tvar) {
    if (p->cv_terms < 1 || p->cv_terms > 3) return bad("cv_terms must be 1..3 with cv_poly");
    if (!(p->precision == LBM_PREC_FP64 || p->precision == LBM_PREC_FP32)) {
      g_create_error = "temperature-dependent heats run with FP64 or FP32 storage";
      return LBM_ERR_UNSUPPORTED;
    }
    if (walls || p->closure == LBM_CLOSURE_MLP) {
      g_create_error = "temperature-dependent heats run on periodic grids with the exact closure";
      return LBM_ERR_UNSUPPORTED;
    }
    for (int a = 0; a < M; ++a)
      if (!(p->cv_poly[a * p->cv_terms] > 0.0)) return bad("cv_poly: the heat at T = 0 must be > 0");
  }

  const lbm::KernelSet* ks = select_kernels(M, p->precision);
  if (!ks) { g_create_error = "no kernels built for this (M, precision)"; return LBM_ERR_UNSUPPORTED; }
  if (p->closure == LBM_CLOSURE_MLP && !ks->mlp_step_ok) {
    g_create_error = "the learned closure runs only in the FP32-arithmetic precisions with M >= 2";
    return LBM_ERR_UNSUPPORTED;
  }
  if (p->closure == LBM_CLOSURE_MLP && walls) {
    g_create_error = "the learned closure runs on periodic grids only";
    return LBM_ERR_UNSUPPORTED;
  }

  lbm_mix* h = new (std::nothrow) lbm_mix();
  if (!h) return bad("out of host memory");
  h->M = M; h->prec = p->precision; h->ks = ks;
  h->N = (long long)p->nx * p->ny * p->nz;
  h->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&h->device);

  lbm::DevParams<double>& d = h->p64;
  d.N = h->N; d.nx = p->nx; d.ny = p->ny; d.nz = p->nz; d.M = M; d.slaved = slaved;
  d.weak = p->coupling == LBM_COUPLE_WEAK;
  d.wall_x = walls ? 1 : 0;
  d.frame = jets ? 1 : 0;
  d.jet_y0 = jets ? p->jet_y0 : 0; d.jet_y1 = jets ? p->jet_y1 : 0;
  d.omega_is_fixed = p->omega_fixed > 0.0; d.omega1_is_fixed = p->omega1_fixed > 0.0;
  d.omega_fixed = p->omega_fixed; d.omega1_fixed = p->omega1_fixed; d.R_U = p->R_U;
  d.cond_bound = p->fp64_cond_bound > 0.0 ? p->fp64_cond_bound : 1e3;
  d.closure_bound = p->closure_residual_bound > 0.0 ? p->closure_residual_bound : 1e-2;
  h->closure = p->closure == LBM_CLOSURE_MLP;
  for (int a = 0; a < lbm::MAXM; ++a) {
    const bool on = a < M;
    const double ma = on ? p->molar_mass[a] : 1.0;
    d.mass[a] = ma; d.inv_mass[a] = 1.0 / ma; d.R_a[a] = p->R_U / ma;     // Eq. (Ra)
    d.Cv_a[a] = on ? p->cv_molar[a] * p->R_U / ma : 0.0;                    // C_{a,v} = C-bar/m_a
    d.Cp_a[a] = d.Cv_a[a] + d.R_a[a];                                       // Mayer
    d.mu[a] = (on && p->mu) ? p->mu[a] : 1.0;
    d.lam[a] = (on && p->lambda) ? p->lambda[a] : 1.0;
    d.inv_lam[a] = 1.0 / d.lam[a];
  }
  for (int a = 0; a < lbm::MAXM; ++a)
    for (int b = 0; b < lbm::MAXM; ++b) {
      if (a < M && b < M) {
        // Eq. (wilkePhi)
        d.phi[a][b] = std::pow(1.0 + std::sqrt((d.mu[a] / d.mu[b]) * std::sqrt(d.mass[b] / d.mass[a])), 2.0)
                    / (std::sqrt(8.0) * std::sqrt(1.0 + d.mass[a] / d.mass[b]));
        d.Cab[a][b] = 1.0 / (D[a][b] * d.mass[a] * d.mass[b]);             // Eq. (tauab)
      } else {
        d.phi[a][b] = 0.0; d.Cab[a][b] = 0.0;
      }
      d.Cab64[a][b] = d.Cab[a][b];
    }
  d.tvar = tvar ? 1 : 0;
  d.nterm = tvar ? p->cv_terms : 1;
  for (int a = 0; a < lbm::MAXM; ++a) {
    for (int k = 0; k < 3; ++k) {
      // per mass: C_{a,v}(T) = (R_U / m_a) sum_k c_ak T^k; U_a = T sum_k c_ak T^k R_U / (m_a (k + 1))
      const double c = (a < M) ? (tvar ? (k < p->cv_terms ? p->cv_poly[a * p->cv_terms + k] : 0.0)
                                       : (k == 0 ? p->cv_molar[a] : 0.0)) : 0.0;
      d.cvp[a][k] = c * p->R_U / d.mass[a];
      d.Uc[a][k] = d.cvp[a][k] / (k + 1);
      d.Hc[a][k] = d.Uc[a][k] + (k == 0 && a < M ? d.R_a[a] : 0.0);
    }
    d.Uar[a] = 0.0;
  }
  d.Ur = 0.0;
  d.rho_eps = 1e-14;
  const bool store16 = p->precision == LBM_PREC_FP16_STORE || p->precision == LBM_PREC_BF16_STORE;
  d.rec_w = store16 ? lbm::eq_rec_width(M, d.weak) : 0;
  fill_params<float>(h->p32, d);
  h->p32.rho_eps = 1e-7f;

  const long long nblocks = (h->N + 255) / 256;
  cudaError_t e = cudaMalloc(&h->d_err, 256);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_partials, (size_t)nblocks * 16 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_base, sizeof(double) * (lbm::MAXM + 2) * 27);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_sums, 16 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, 256, h->stream);
  // the closure network: zero weights (every node falls back until trained)
  const size_t nw = (size_t)ks->mlp_nw;
  if (e == cudaSuccess) e = cudaMalloc(&h->d_w, 4 * nw * sizeof(float));
  if (e == cudaSuccess) {
    h->d_m = h->d_w + nw; h->d_v = h->d_m + nw; h->d_g = h->d_v + nw;
    e = cudaMemsetAsync(h->d_w, 0, 4 * nw * sizeof(float), h->stream);
  }
  if (e == cudaSuccess) e = cudaMalloc(&h->d_img, (size_t)ks->mlp_img_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_stats, 2 * sizeof(unsigned long long) + sizeof(double));
  if (e == cudaSuccess) {
    h->d_loss = reinterpret_cast<double*>(h->d_stats + 2);
    e = cudaMemsetAsync(h->d_stats, 0, 2 * sizeof(unsigned long long), h->stream);
  }
  if (e == cudaSuccess) e = ks->mlp_pack(h->ctx(), h->d_w, h->d_img);
  if (e == cudaSuccess && jets) {
    // the complete equilibria of the two inlet states (the library's own FP64
    // initial-state kernel on a two-node grid)
    const int S = M + 2;
    const size_t n_out = (size_t)S * 27 * 2, n_zero = (size_t)S * 27, n_in = (size_t)M * 2 + 6 + 2 + 2;
    std::vector<double> in(n_in, 0.0);
    for (int k = 0; k < 2; ++k) {
      for (int a = 0; a < M; ++a) in[(size_t)a * 2 + k] = p->jet_X[k * M + a];
      in[(size_t)M * 2 + 0 * 2 + k] = p->jet_u[k];
      in[(size_t)M * 2 + 6 + k] = p->jet_T[k];
      in[(size_t)M * 2 + 8 + k] = p->jet_P[k];
    }
    e = cudaMalloc(&h->d_jet, (n_out + n_zero + n_in) * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_jet, 0, (n_out + n_zero) * sizeof(double), h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->d_jet + n_out + n_zero, in.data(), n_in * sizeof(double), cudaMemcpyHostToDevice,
                          h->stream);
    if (e == cudaSuccess) e = ks->jet_table(h->ctx(), h->d_jet);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);      // `in` leaves scope
    h->launches += 1;
  }
  if (e != cudaSuccess) {
    g_create_error = std::string("CUDA: ") + cudaGetErrorString(e);
    if (h->d_err) cudaFree(h->d_err);
    if (h->d_partials) cudaFree(h->d_partials);
    if (h->d_sums) cudaFree(h->d_sums);
    if (h->d_base) cudaFree(h->d_base);
    if (h->d_w) cudaFree(h->d_w);
    if (h->d_img) cudaFree(h->d_img);
    if (h->d_stats) cudaFree(h->d_stats);
    if (h->d_jet) cudaFree(h->d_jet);
    delete h;
    return LBM_ERR_CUDA;
  }
  *out = h;
  return LBM_OK;
}

lbm_status lbm_mix_required_bytes(lbm_mix_t h, size_t* pops_bytes, size_t* scratch_bytes) {
  if (!h) return LBM_ERR_ARG;
  if (pops_bytes) *pops_bytes = h->need_pops();
  if (scratch_bytes) *scratch_bytes = h->need_scratch();
  return LBM_OK;
}

lbm_status lbm_mix_bind_buffers(lbm_mix_t h, void* pops, size_t pops_bytes, void* scratch, size_t scratch_bytes) {
  if (!h) return LBM_ERR_ARG;
  if (!pops || !scratch) return h->fail(LBM_ERR_ARG, "NULL buffer");
  if (pops_bytes < h->need_pops()) return h->fail(LBM_ERR_ARG, "population buffer too small");
  if (scratch_bytes < h->need_scratch()) return h->fail(LBM_ERR_ARG, "scratch buffer too small");
  if (((uintptr_t)pops & 255) || ((uintptr_t)scratch & 255)) return h->fail(LBM_ERR_ARG, "buffers must be 256-byte aligned");
  if (h->owns_buffers) { cudaFree(h->pops); cudaFree(h->scratch); h->owns_buffers = false; }
  h->pops = pops; h->pops_bytes = pops_bytes; h->scratch = scratch; h->scratch_bytes = scratch_bytes;
  h->initialized = false;
  return LBM_OK;
}

lbm_status lbm_mix_alloc_buffers(lbm_mix_t h) {
  if (!h) return LBM_ERR_ARG;
  void* a = nullptr; void* b = nullptr;
  lbm_status s = h->cuda(cudaMalloc(&a, h->need_pops()), "cudaMalloc(populations)");
  if (s != LBM_OK) return s;
  s = h->cuda(cudaMalloc(&b, h->need_scratch()), "cudaMalloc(scratch)");
  if (s != LBM_OK) { cudaFree(a); return s; }
  if (h->owns_buffers) { cudaFree(h->pops); cudaFree(h->scratch); }
  h->pops = a; h->pops_bytes = h->need_pops(); h->scratch = b; h->scratch_bytes = h->need_scratch();
  h->owns_buffers = true; h->initialized = false;
  return LBM_OK;
}

lbm_status lbm_mix_init_fields(lbm_mix_t h, const double* X, const double* u, const double* T,
                               const double* P, int host_ptrs) {
  if (!h) return LBM_ERR_ARG;
  if (!X || !u || !T || !P) return h->fail(LBM_ERR_ARG, "NULL field");
  lbm_status s = h->ready();
  if (s != LBM_OK) return s;
  const size_t N = (size_t)h->N, M = (size_t)h->M;
  const double *dX = X, *du = u, *dT = T, *dP = P;
  if (host_ptrs) {
    s = h->ensure_stage((M + 5) * N * sizeof(double));
    if (s != LBM_OK) return s;
    double* st = h->d_stage;
    cudaError_t e = cudaMemcpyAsync(st, X, M * N * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(st + M * N, u, 3 * N * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(st + (M + 3) * N, T, N * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(st + (M + 4) * N, P, N * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if ((s = h->cuda(e, "host-to-device copy of the fields")) != LBM_OK) return s;
    dX = st; du = st + M * N; dT = st + (M + 3) * N; dP = st + (M + 4) * N;
  }
  if ((s = h->cuda(cudaMemsetAsync(h->d_err, 0, sizeof(unsigned), h->stream), "clear flag")) != LBM_OK) return s;
  if (!h->fixed_reference && (s = h->reference_from_fields(dX, dT, dP)) != LBM_OK) return s;
  if ((s = h->clear_pending()) != LBM_OK) return s;
  if ((s = h->cuda(h->ks->init(h->ctx(), dX, du, dT, dP), "init kernel")) != LBM_OK) return s;
  h->launches += h->ks->setup_launches;
  h->steps = 0;
  h->initialized = true;
  if (host_ptrs) return h->cuda(cudaStreamSynchronize(h->stream), "synchronize");
  return LBM_OK;
}

lbm_status lbm_mix_step(lbm_mix_t h, int nsteps) {
  if (!h) return LBM_ERR_ARG;
  if (nsteps < 0) return h->fail(LBM_ERR_ARG, "nsteps < 0");
  if (!h->initialized) return h->fail(LBM_ERR_STATE, "step before init_fields/set_populations");
  lbm::LaunchCtx c = h->ctx();
  for (int s = 0; s < nsteps; ++s) {
    if (h->timing) {
      while (h->ev_pool.size() < h->ev_used + 4) {
        cudaEvent_t e;
        lbm_status st = h->cuda(cudaEventCreate(&e), "cudaEventCreate");
        if (st != LBM_OK) return st;
        h->ev_pool.push_back(e);
      }
      c.ev = &h->ev_pool[h->ev_used];
      h->ev_used += 4;
    }
    lbm_status st = h->cuda(h->ks->step(c, (int)(h->steps & 1)), "step kernels");
    if (st != LBM_OK) return st;
    h->steps += 1;
    h->launches += h->ks->launches_per_step + (h->p64.frame ? 4 : 0);
  }
  return LBM_OK;
}

lbm_status lbm_mix_get_moments(lbm_mix_t h, double* out, int host_ptrs) {
  if (!h) return LBM_ERR_ARG;
  if (!out) return h->fail(LBM_ERR_ARG, "NULL output");
  if (!h->initialized) return h->fail(LBM_ERR_STATE, "no state");
  const size_t bytes = (size_t)lbm_mix_num_outputs(h->M) * (size_t)h->N * sizeof(double);
  double* dst = out;
  lbm_status s;
  if (host_ptrs) {
    if ((s = h->ensure_stage(bytes)) != LBM_OK) return s;
    dst = h->d_stage;
  }
  if ((s = h->cuda(h->ks->moments(h->ctx(), (int)(h->steps & 1), dst), "moments kernel")) != LBM_OK) return s;
  h->launches += 1;
  if (host_ptrs) {
    if ((s = h->cuda(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, h->stream), "device-to-host copy")) != LBM_OK)
      return s;
    return h->check_flag();
  }
  return LBM_OK;
}

lbm_status lbm_mix_get_populations(lbm_mix_t h, double* out, int host_ptrs) {
  if (!h) return LBM_ERR_ARG;
  if (!out) return h->fail(LBM_ERR_ARG, "NULL output");
  if (!h->initialized) return h->fail(LBM_ERR_STATE, "no state");
  const size_t bytes = (size_t)(h->M + 2) * 27 * (size_t)h->N * sizeof(double);
  double* dst = out;
  lbm_status s;
  if (host_ptrs) {
    if ((s = h->ensure_stage(bytes)) != LBM_OK) return s;
    dst = h->d_stage;
  }
  if ((s = h->cuda(h->ks->get_pops(h->ctx(), (int)(h->steps & 1), dst), "get_populations kernel")) != LBM_OK) return s;
  h->launches += 1;
  if (host_ptrs) {
    if ((s = h->cuda(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, h->stream), "device-to-host copy")) != LBM_OK)
      return s;
    return h->cuda(cudaStreamSynchronize(h->stream), "synchronize");
  }
  return LBM_OK;
}

lbm_status lbm_mix_set_populations(lbm_mix_t h, const double* in, int host_ptrs) {
  if (!h) return LBM_ERR_ARG;
  if (!in) return h->fail(LBM_ERR_ARG, "NULL input");
  lbm_status s = h->ready();
  if (s != LBM_OK) return s;
  const size_t bytes = (size_t)(h->M + 2) * 27 * (size_t)h->N * sizeof(double);
  const double* src = in;
  if (host_ptrs) {
    if ((s = h->ensure_stage(bytes)) != LBM_OK) return s;
    if ((s = h->cuda(cudaMemcpyAsync(h->d_stage, in, bytes, cudaMemcpyHostToDevice, h->stream), "host-to-device copy")) != LBM_OK)
      return s;
    src = h->d_stage;
  }
  if (!h->has_reference && (s = h->reference_from_pops(src)) != LBM_OK) return s;
  if ((s = h->clear_pending()) != LBM_OK) return s;
  if ((s = h->cuda(h->ks->set_pops(h->ctx(), (int)(h->steps & 1), src), "set_populations kernel")) != LBM_OK) return s;
  h->launches += h->ks->setup_launches;
  h->initialized = true;
  if (host_ptrs) return h->cuda(cudaStreamSynchronize(h->stream), "synchronize");
  return LBM_OK;
}

lbm_status lbm_mix_diagnostics(lbm_mix_t h, double* sums) {
  if (!h) return LBM_ERR_ARG;
  if (!sums) return h->fail(LBM_ERR_ARG, "NULL output");
  if (!h->initialized) return h->fail(LBM_ERR_STATE, "no state");
  lbm_status s;
  if ((s = h->cuda(h->ks->diag(h->ctx(), (int)(h->steps & 1), h->d_sums), "diagnostics kernels")) != LBM_OK) return s;
  h->launches += 2;
  if ((s = h->cuda(cudaMemcpyAsync(sums, h->d_sums, (size_t)(h->M + 5) * sizeof(double), cudaMemcpyDeviceToHost,
                                   h->stream), "device-to-host copy")) != LBM_OK)
    return s;
  s = h->check_flag();
  // the kernels sum deviations from the reference tables; add the tables' sums
  const double Nd = (double)h->N;
  for (int a = 0; a < h->M; ++a) sums[a] += Nd * h->p64.RL[a];
  sums[h->M] += Nd * h->p64.RL[h->M];
  sums[h->M + 4] += Nd * h->p64.RL[h->M + 1];
  return s;
}

lbm_status lbm_mix_set_reference(lbm_mix_t h, const double* Y, double T, double rho) {
  if (!h) return LBM_ERR_ARG;
  if (!Y) return h->fail(LBM_ERR_ARG, "NULL mass fractions");
  double Yn[lbm::MAXM], sum = 0.0;
  for (int a = 0; a < h->M; ++a) {
    if (!(Y[a] >= 0.0) || !std::isfinite(Y[a])) return h->fail(LBM_ERR_ARG, "mass fractions must be >= 0");
    sum += Y[a];
  }
  if (!(sum > 0.0)) return h->fail(LBM_ERR_ARG, "mass fractions sum to zero");
  for (int a = 0; a < h->M; ++a) Yn[a] = Y[a] / sum;
  lbm_status s = h->set_reference(Yn, T, rho);
  if (s != LBM_OK) return s;
  h->fixed_reference = true;
  h->initialized = false;      // a stored state was relative to the previous reference
  return LBM_OK;
}

// The halo of a z slab: every population slot, side field and (16-bit
// storage) equilibrium record of `ghost` planes.
static lbm_status halo_check(lbm_mix_t h, int face, int ghost) {
  if (face != 0 && face != 1) return h->fail(LBM_ERR_ARG, "face must be 0 (-z) or 1 (+z)");
  if (ghost < 1) return h->fail(LBM_ERR_ARG, "ghost must be >= 1");
  if ((long long)h->p64.nz < 3LL * ghost) return h->fail(LBM_ERR_ARG, "nz must be at least 3 * ghost");
  return h->ready();
}

lbm_status lbm_mix_halo_bytes(lbm_mix_t h, int ghost, size_t* bytes) {
  if (!h || !bytes) return LBM_ERR_ARG;
  if (ghost < 1) return h->fail(LBM_ERR_ARG, "ghost must be >= 1");
  const size_t plane = (size_t)h->p64.nx * (size_t)h->p64.ny;
  *bytes = (size_t)ghost * plane * ((size_t)(h->M + 2) * 27 * store_elem_bytes(h->prec) +
                                    (size_t)lbm::NSIDE * side_elem_bytes(h->prec) + 2 * (size_t)h->p64.rec_w * 4);
  return LBM_OK;
}

static lbm_status halo_move(lbm_mix_t h, int face, int ghost, void* buf, int unpack) {
  lbm_status s = halo_check(h, face, ghost);
  if (s != LBM_OK) return s;
  if (!buf) return h->fail(LBM_ERR_ARG, "NULL buffer");
  const long long plane = (long long)h->p64.nx * h->p64.ny, nz = h->p64.nz, N = h->N;
  // pack: the `ghost` interior planes next to the face; unpack: the ghost planes of the face
  const long long z0 = unpack ? (face == 0 ? 0 : nz - ghost) : (face == 0 ? ghost : nz - 2LL * ghost);
  const long long seg = (long long)ghost * plane;
  const size_t es = store_elem_bytes(h->prec), ss = side_elem_bytes(h->prec);
  const long long nf = (long long)(h->M + 2) * 27;
  char* b = (char*)buf;
  cudaError_t e;
  if (es == 8) e = halo_copy<double>(h->pops, b, nf, N, z0 * plane, seg, unpack, h->stream);
  else if (es == 4) e = halo_copy<float>(h->pops, b, nf, N, z0 * plane, seg, unpack, h->stream);
  else e = halo_copy<unsigned short>(h->pops, b, nf, N, z0 * plane, seg, unpack, h->stream);
  b += (size_t)nf * seg * es;
  if (e == cudaSuccess) {
    if (ss == 8) e = halo_copy<double>(h->scratch, b, lbm::NSIDE, N, z0 * plane, seg, unpack, h->stream);
    else e = halo_copy<float>(h->scratch, b, lbm::NSIDE, N, z0 * plane, seg, unpack, h->stream);
  }
  b += (size_t)lbm::NSIDE * seg * ss;
  const long long rw = h->p64.rec_w;
  if (e == cudaSuccess && rw > 0)
    e = halo_copy<float>((float*)h->scratch + lbm::eq_rec_offset(N), b, 2, rw * N, z0 * plane * rw, seg * rw, unpack,
                         h->stream);
  if ((s = h->cuda(e, unpack ? "halo unpack" : "halo pack")) != LBM_OK) return s;
  h->launches += rw > 0 ? 3 : 2;
  return LBM_OK;
}

lbm_status lbm_mix_halo_pack(lbm_mix_t h, int face, int ghost, void* buf) {
  if (!h) return LBM_ERR_ARG;
  return halo_move(h, face, ghost, buf, 0);
}

lbm_status lbm_mix_halo_unpack(lbm_mix_t h, int face, int ghost, const void* buf) {
  if (!h) return LBM_ERR_ARG;
  return halo_move(h, face, ghost, const_cast<void*>(buf), 1);
}

lbm_status lbm_mix_synchronize(lbm_mix_t h) {
  if (!h) return LBM_ERR_ARG;
  return h->check_flag();
}

lbm_status lbm_mix_enable_kernel_timing(lbm_mix_t h, int enable) {
  if (!h) return LBM_ERR_ARG;
  h->timing = enable != 0;
  if (!h->timing) h->ev_used = 0;
  return LBM_OK;
}

int lbm_mix_kernel_times(lbm_mix_t h, double* ms, long long* counts, int nk) {
  if (!h) return -1;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return -1;
  for (int k = 0; k < nk; ++k) { if (ms) ms[k] = 0.0; if (counts) counts[k] = 0; }
  for (size_t b = 0; b + 4 <= h->ev_used; b += 4) {
    for (int k = 0; k < 3 && k < nk; ++k) {
      float t = 0.0f;
      if (cudaEventElapsedTime(&t, h->ev_pool[b + k], h->ev_pool[b + k + 1]) == cudaSuccess) {
        if (ms) ms[k] += t;
        if (counts) counts[k] += 1;
      }
    }
  }
  h->ev_used = 0;
  return 3;
}

long long lbm_mix_step_count(lbm_mix_t h) { return h ? h->steps : -1; }
long long lbm_mix_launch_count(lbm_mix_t h) { return h ? h->launches : -1; }

lbm_status lbm_mix_closure_sizes(int M, int* F, int* O, int* n_weights) {
  const lbm::KernelSet* ks = select_kernels(M, LBM_PREC_FP32);
  if (!ks) { g_create_error = "no kernels built for this species count"; return LBM_ERR_UNSUPPORTED; }
  if (F) *F = ks->mlp_F;
  if (O) *O = ks->mlp_O;
  if (n_weights) *n_weights = ks->mlp_nw;
  return LBM_OK;
}

lbm_status lbm_mix_closure_set_weights(lbm_mix_t h, const float* w, int host_ptr) {
  if (!h) return LBM_ERR_ARG;
  if (!w) return h->fail(LBM_ERR_ARG, "NULL weights");
  const size_t nw = (size_t)h->ks->mlp_nw;
  lbm_status s = h->cuda(cudaMemcpyAsync(h->d_w, w, nw * sizeof(float),
                                         host_ptr ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->stream),
                         "copy weights");
  if (s != LBM_OK) return s;
  if ((s = h->cuda(cudaMemsetAsync(h->d_m, 0, 2 * nw * sizeof(float), h->stream), "reset Adam state")) != LBM_OK)
    return s;
  h->adam_t = 0;
  if ((s = h->repack()) != LBM_OK) return s;
  h->launches += 1;
  if (host_ptr) return h->cuda(cudaStreamSynchronize(h->stream), "synchronize");
  return LBM_OK;
}

lbm_status lbm_mix_closure_get_weights(lbm_mix_t h, float* w, int host_ptr) {
  if (!h) return LBM_ERR_ARG;
  if (!w) return h->fail(LBM_ERR_ARG, "NULL output");
  lbm_status s = h->cuda(cudaMemcpyAsync(w, h->d_w, (size_t)h->ks->mlp_nw * sizeof(float),
                                         host_ptr ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream),
                         "copy weights");
  if (s != LBM_OK || !host_ptr) return s;
  return h->cuda(cudaStreamSynchronize(h->stream), "synchronize");
}

lbm_status lbm_mix_closure_samples(lbm_mix_t h, float* features, float* targets) {
  if (!h) return LBM_ERR_ARG;
  if (!features || !targets) return h->fail(LBM_ERR_ARG, "NULL output");
  if (!h->initialized) return h->fail(LBM_ERR_STATE, "no state");
  lbm_status s = h->cuda(h->ks->samples(h->ctx(), (int)(h->steps & 1), features, targets), "samples kernel");
  if (s == LBM_OK) h->launches += 1;
  return s;
}

lbm_status lbm_mix_closure_forward(lbm_mix_t h, const float* features, float* outputs, long long n) {
  if (!h) return LBM_ERR_ARG;
  if (n < 0 || (n > 0 && (!features || !outputs))) return h->fail(LBM_ERR_ARG, "bad arguments");
  if (n == 0) return LBM_OK;
  lbm_status s = h->cuda(h->ks->mlp_forward(h->ctx(), features, outputs, n), "network kernel");
  if (s == LBM_OK) h->launches += 1;
  return s;
}

lbm_status lbm_mix_closure_loss_grad(lbm_mix_t h, const float* features, const float* targets, long long n,
                                     float* grad, double* loss) {
  if (!h) return LBM_ERR_ARG;
  if (n <= 0 || n > (1LL << 30) || !features || !targets) return h->fail(LBM_ERR_ARG, "bad arguments");
  lbm_status s = h->ensure_train_scratch(n);
  if (s != LBM_OK) return s;
  s = h->cuda(lbm::mlp_train_grad(h->stream, h->mlp_shape(), h->d_w, features, targets, (int)n, h->z,
                                  grad ? grad : h->d_g, h->d_loss), "training kernels");
  if (s != LBM_OK) return s;
  h->launches += 16;
  if (loss) {
    if ((s = h->cuda(cudaMemcpyAsync(loss, h->d_loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                     "copy loss")) != LBM_OK)
      return s;
    return h->cuda(cudaStreamSynchronize(h->stream), "synchronize");
  }
  return LBM_OK;
}

lbm_status lbm_mix_closure_train(lbm_mix_t h, const float* features, const float* targets, long long n, int batch,
                                 int steps, double lr, double* last_loss) {
  if (!h) return LBM_ERR_ARG;
  if (n <= 0 || batch <= 0 || steps < 0 || !(lr > 0.0) || !features || !targets)
    return h->fail(LBM_ERR_ARG, "bad arguments");
  const long long rows_max = batch < n ? batch : n;
  lbm_status s = h->ensure_train_scratch(rows_max);
  if (s != LBM_OK) return s;
  const int F = h->ks->mlp_F, O = h->ks->mlp_O;
  const long long nw = h->ks->mlp_nw;
  long long start = 0;
  for (int it = 0; it < steps; ++it) {
    const long long rows = (n - start) < rows_max ? (n - start) : rows_max;
    s = h->cuda(lbm::mlp_train_grad(h->stream, h->mlp_shape(), h->d_w, features + start * F, targets + start * O,
                                    (int)rows, h->z, h->d_g, h->d_loss), "training kernels");
    if (s != LBM_OK) return s;
    s = h->cuda(lbm::mlp_adam(h->stream, h->d_w, h->d_g, h->d_m, h->d_v, nw, (float)lr, ++h->adam_t), "Adam kernel");
    if (s != LBM_OK) return s;
    h->launches += 17;
    start += rows;
    if (start >= n) start = 0;
  }
  if ((s = h->repack()) != LBM_OK) return s;
  h->launches += 1;
  if (last_loss) {
    *last_loss = 0.0;
    if (steps > 0 &&
        (s = h->cuda(cudaMemcpyAsync(last_loss, h->d_loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                     "copy loss")) != LBM_OK)
      return s;
  }
  return h->cuda(cudaStreamSynchronize(h->stream), "synchronize");
}

lbm_status lbm_mix_closure_stats(lbm_mix_t h, long long* accepted, long long* fallback, int reset) {
  if (!h) return LBM_ERR_ARG;
  unsigned long long c[2] = {0, 0};
  lbm_status s = h->cuda(cudaMemcpyAsync(c, h->d_stats, sizeof(c), cudaMemcpyDeviceToHost, h->stream), "copy counters");
  if (s != LBM_OK) return s;
  if (reset && (s = h->cuda(cudaMemsetAsync(h->d_stats, 0, sizeof(c), h->stream), "reset counters")) != LBM_OK)
    return s;
  if ((s = h->cuda(cudaStreamSynchronize(h->stream), "synchronize")) != LBM_OK) return s;
  if (accepted) *accepted = (long long)c[0];
  if (fallback) *fallback = (long long)c[1];
  return LBM_OK;
}


lbm_status lbm_mix_batch_create(const lbm_mix_params* params, int ndomains, void* cuda_stream,
                                lbm_mix_batch_t* out) {
  auto bad = [&](lbm_status st, const std::string& m) { g_create_error = m; return st; };
  if (!out) return bad(LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!params || ndomains < 1) return bad(LBM_ERR_ARG, "need at least one domain");
  for (int d = 1; d < ndomains; ++d)
    if (params[d].M != params[0].M || params[d].precision != params[0].precision ||
        params[d].coupling != params[0].coupling)
      return bad(LBM_ERR_ARG, "all domains must share M, precision and coupling");
  for (int d = 0; d < ndomains; ++d) {
    if (params[d].closure != LBM_CLOSURE_EXACT) return bad(LBM_ERR_UNSUPPORTED, "batched domains use the exact closure");
    if (params[d].cv_poly) return bad(LBM_ERR_UNSUPPORTED, "batched domains use constant heats");
    for (int s = 0; s < 6; ++s)
      if (params[d].bc[s] != LBM_BC_PERIODIC) return bad(LBM_ERR_UNSUPPORTED, "batched domains are periodic");
  }
  lbm_mix_batch* b = new (std::nothrow) lbm_mix_batch();
  if (!b) return bad(LBM_ERR_ARG, "out of host memory");
  b->nd = ndomains; b->M = params[0].M; b->prec = params[0].precision;
  b->user = (cudaStream_t)cuda_stream;
  auto cleanup = [&](lbm_status st) {
    lbm_mix_batch_destroy(b);
    return st;
  };
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess)
    return cleanup(bad(LBM_ERR_CUDA, "stream/event creation failed"));
  for (int d = 0; d < ndomains; ++d) {
    lbm_mix_t h = nullptr;
    lbm_status st = lbm_mix_create(&params[d], cuda_stream, &h);
    if (st != LBM_OK) {
      g_create_error = "domain " + std::to_string(d) + ": " + g_create_error;
      return cleanup(st);
    }
    b->dom.push_back(h);
  }
  b->ks = b->dom[0]->ks;
  // one allocation each for populations and scratch, 256-byte aligned slices
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  std::vector<size_t> po(ndomains), so(ndomains);
  for (int d = 0; d < ndomains; ++d) {
    po[d] = b->pops_total; b->pops_total += up(b->dom[d]->need_pops());
    so[d] = b->side_total; b->side_total += up(b->dom[d]->need_scratch());
    b->nodes += b->dom[d]->N;
  }
  if (cudaMalloc(&b->pops_all, b->pops_total) != cudaSuccess || cudaMalloc(&b->side_all, b->side_total) != cudaSuccess)
    return cleanup(bad(LBM_ERR_CUDA, "cudaMalloc of the ensemble buffers failed"));
  std::vector<void*> ptrs(2 * ndomains);
  std::vector<lbm::BatchGeom> geom(ndomains);
  for (int d = 0; d < ndomains; ++d) {
    lbm_mix* h = b->dom[d];
    ptrs[d] = (char*)b->pops_all + po[d];
    ptrs[ndomains + d] = (char*)b->side_all + so[d];
    if (lbm_mix_bind_buffers(h, ptrs[d], h->need_pops(), ptrs[ndomains + d], h->need_scratch()) != LBM_OK)
      return cleanup(bad(LBM_ERR_ARG, "binding domain buffers failed"));
    geom[d] = lbm::BatchGeom{h->N, h->p64.nx, h->p64.ny, h->p64.nz};
  }
  // tiles: (domain, first node) for the collide block and for 128/256-thread stencil blocks
  std::vector<int2> tiles;
  auto add_tiles = [&](int bs) {
    int cnt = 0;
    for (int d = 0; d < ndomains; ++d)
      for (long long n0 = 0; n0 < b->dom[d]->N; n0 += bs) { tiles.push_back(make_int2(d, (int)n0)); ++cnt; }
    return cnt;
  };
  b->ntiles_c = add_tiles(b->ks->collide_bs);
  b->ntiles_128 = add_tiles(128);
  b->ntiles_256 = add_tiles(256);
  b->param_bytes = b->prec == LBM_PREC_FP64 ? sizeof(lbm::DevParams<double>) : sizeof(lbm::DevParams<float>);
  cudaError_t e = cudaMalloc(&b->d_params, b->param_bytes * ndomains);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_geom, sizeof(lbm::BatchGeom) * ndomains);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_ptrs, sizeof(void*) * 2 * ndomains);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_tiles, sizeof(int2) * tiles.size());
  if (e == cudaSuccess) e = cudaMalloc(&b->d_err, 256);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_geom, geom.data(), sizeof(lbm::BatchGeom) * ndomains, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_ptrs, ptrs.data(), sizeof(void*) * 2 * ndomains, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, 256);
  if (e == cudaSuccess) e = b->ks->batch_prepare();
  int dev = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cleanup(bad(LBM_ERR_CUDA, std::string("CUDA: ") + cudaGetErrorString(e)));
  b->uploaded.assign(ndomains, -1);
  // default launch shapes (the autotuner may replace them): one block per tile
  b->grid_c = b->ntiles_c;
  b->block_l = 256;
  b->grid_l = b->ntiles_256;
  *out = b;
  return LBM_OK;
}

lbm_status lbm_mix_batch_domain(lbm_mix_batch_t b, int d, lbm_mix_t* h) {
  if (!b || !h) return LBM_ERR_ARG;
  if (d < 0 || d >= b->nd) return b->fail(LBM_ERR_ARG, "domain index out of range");
  *h = b->dom[d];
  return LBM_OK;
}

long long lbm_mix_batch_nodes(lbm_mix_batch_t b) { return b ? b->nodes : -1; }

lbm_status lbm_mix_batch_step(lbm_mix_batch_t b, int nsteps) {
  if (!b) return LBM_ERR_ARG;
  if (nsteps < 0) return b->fail(LBM_ERR_ARG, "nsteps < 0");
  for (lbm_mix* h : b->dom) {
    if (!h->initialized) return b->fail(LBM_ERR_STATE, "every domain needs init_fields or set_populations first");
    if (h->steps != b->steps) return b->fail(LBM_ERR_STATE, "a domain was stepped on its own; its parity differs");
  }
  lbm_status st;
  if ((st = b->cuda(cudaEventRecord(b->ev_in, b->user), "record")) != LBM_OK) return st;
  if ((st = b->cuda(cudaStreamWaitEvent(b->stream, b->ev_in, 0), "wait")) != LBM_OK) return st;
  if ((st = b->upload_params()) != LBM_OK) return st;
  if ((st = b->run(nsteps, b->use_graph)) != LBM_OK) return st;
  if ((st = b->cuda(cudaEventRecord(b->ev_out, b->stream), "record")) != LBM_OK) return st;
  if ((st = b->cuda(cudaStreamWaitEvent(b->user, b->ev_out, 0), "wait")) != LBM_OK) return st;
  b->advance(nsteps);
  return LBM_OK;
}

lbm_status lbm_mix_batch_autotune(lbm_mix_batch_t b, int trial_steps, int* config, double* best_ms) {
  if (!b) return LBM_ERR_ARG;
  if (trial_steps < 1) return b->fail(LBM_ERR_ARG, "trial_steps < 1");
  for (lbm_mix* h : b->dom)
    if (!h->initialized || h->steps != b->steps) return b->fail(LBM_ERR_STATE, "initialise every domain first");
  lbm_status st;
  if ((st = b->cuda(cudaStreamSynchronize(b->user), "synchronize")) != LBM_OK) return st;
  if ((st = b->upload_params()) != LBM_OK) return st;
  // save the state: the trials step it
  void *sp = nullptr, *ss = nullptr;
  if ((st = b->cuda(cudaMalloc(&sp, b->pops_total), "cudaMalloc(autotune)")) != LBM_OK) return st;
  if ((st = b->cuda(cudaMalloc(&ss, b->side_total), "cudaMalloc(autotune)")) != LBM_OK) { cudaFree(sp); return st; }
  cudaMemcpyAsync(sp, b->pops_all, b->pops_total, cudaMemcpyDeviceToDevice, b->stream);
  cudaMemcpyAsync(ss, b->side_all, b->side_total, cudaMemcpyDeviceToDevice, b->stream);
  const long long steps0 = b->steps;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto trial = [&](double& ms) -> lbm_status {
    lbm_status s2 = b->run(2, true);                         // warm-up (captures the graph)
    if (s2 != LBM_OK) return s2;
    b->steps += 2;
    cudaEventRecord(e0, b->stream);
    if ((s2 = b->run(trial_steps, true)) != LBM_OK) return s2;
    cudaEventRecord(e1, b->stream);
    b->steps += trial_steps;
    if ((s2 = b->cuda(cudaEventSynchronize(e1), "synchronize")) != LBM_OK) return s2;
    float t = 0.0f;
    cudaEventElapsedTime(&t, e0, e1);
    ms = (double)t / trial_steps;
    return LBM_OK;
  };
  const int sm = b->sm_count > 0 ? b->sm_count : 1;
  double best = 1e300;
  int bmode = 0, bbr = b->nbranch, bc = b->ntiles_c, bl = 256, bg = b->ntiles_256;
  st = LBM_OK;
  // mode 0: persistent launches over all tiles
  b->mode = 0;
  b->block_l = 256; b->grid_l = b->ntiles_256;
  for (int g : {b->ntiles_c, sm, 2 * sm, 3 * sm, 4 * sm}) {
    if (g > b->ntiles_c || st != LBM_OK) continue;
    b->grid_c = g;
    b->drop_graph();
    double ms;
    if ((st = trial(ms)) == LBM_OK && ms < best) { best = ms; bmode = 0; bc = g; }
  }
  b->grid_c = bc;
  for (int blk : {128, 256}) {
    const int nt = blk == 128 ? b->ntiles_128 : b->ntiles_256;
    for (int g : {nt, 8 * sm, 16 * sm}) {
      if (g > nt || st != LBM_OK) continue;
      b->block_l = blk; b->grid_l = g;
      b->drop_graph();
      double ms;
      if ((st = trial(ms)) == LBM_OK && ms < best) { best = ms; bmode = 0; bl = blk; bg = g; }
    }
  }
  b->block_l = bl; b->grid_l = bg;
  // mode 1: each domain's own kernels on concurrent graph branches
  b->mode = 1;
  for (int nb : {4, 8, 16}) {
    if (st != LBM_OK) break;
    b->nbranch = nb;
    b->drop_graph();
    double ms;
    if ((st = trial(ms)) == LBM_OK && ms < best) { best = ms; bmode = 1; bbr = nb; }
  }
  b->mode = bmode;
  b->nbranch = bbr;
  b->block_l = bl; b->grid_l = bg;
  b->drop_graph();
  // restore the state and the step count
  cudaMemcpyAsync(b->pops_all, sp, b->pops_total, cudaMemcpyDeviceToDevice, b->stream);
  cudaMemcpyAsync(b->side_all, ss, b->side_total, cudaMemcpyDeviceToDevice, b->stream);
  lbm_status s3 = b->cuda(cudaStreamSynchronize(b->stream), "synchronize");
  b->steps = steps0;
  cudaFree(sp);
  cudaFree(ss);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != LBM_OK) return st;
  if (s3 != LBM_OK) return s3;
  if (config) { config[0] = b->grid_c; config[1] = b->block_l; config[2] = b->grid_l; config[3] = b->mode; config[4] = b->nbranch; }
  if (best_ms) *best_ms = best;
  return LBM_OK;
}

lbm_status lbm_mix_batch_set_config(lbm_mix_batch_t b, int grid_collide, int block_stencil, int grid_stencil,
                                    int use_graph) {
  if (!b) return LBM_ERR_ARG;
  if (block_stencil != 128 && block_stencil != 256) return b->fail(LBM_ERR_ARG, "stencil blocks are 128 or 256 threads");
  const int ntl = block_stencil == 128 ? b->ntiles_128 : b->ntiles_256;
  if (grid_collide < 1 || grid_collide > b->ntiles_c || grid_stencil < 1 || grid_stencil > ntl)
    return b->fail(LBM_ERR_ARG, "grid sizes must be in 1..number of tiles");
  b->grid_c = grid_collide; b->block_l = block_stencil; b->grid_l = grid_stencil;
  b->use_graph = use_graph != 0;
  b->drop_graph();
  return LBM_OK;
}

lbm_status lbm_mix_batch_set_mode(lbm_mix_batch_t b, int mode, int branches) {
  if (!b) return LBM_ERR_ARG;
  if ((mode != 0 && mode != 1) || branches < 1 || branches > 64) return b->fail(LBM_ERR_ARG, "mode 0/1, 1..64 branches");
  b->mode = mode;
  b->nbranch = branches;
  b->drop_graph();
  return LBM_OK;
}

lbm_status lbm_mix_batch_config(lbm_mix_batch_t b, int* config) {
  if (!b || !config) return LBM_ERR_ARG;
  config[0] = b->grid_c; config[1] = b->block_l; config[2] = b->grid_l; config[3] = b->use_graph ? 1 : 0;
  config[4] = b->ntiles_c; config[5] = b->ntiles_128; config[6] = b->ntiles_256; config[7] = b->ks->collide_bs;
  config[8] = b->mode; config[9] = b->nbranch;
  return LBM_OK;
}

lbm_status lbm_mix_batch_synchronize(lbm_mix_batch_t b) {
  if (!b) return LBM_ERR_ARG;
  unsigned flag = 0;
  lbm_status st = b->cuda(cudaStreamSynchronize(b->user), "synchronize");
  if (st != LBM_OK) return st;
  if ((st = b->cuda(cudaMemcpy(&flag, b->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost), "read error flag")) != LBM_OK)
    return st;
  if (flag) return b->fail(LBM_ERR_NONFINITE, "a node reached non-positive density or temperature (or NaN)");
  for (int d = 0; d < b->nd; ++d)
    if ((st = b->dom[d]->check_flag()) != LBM_OK) return b->fail(st, "domain " + std::to_string(d) + ": " + b->dom[d]->err);
  return LBM_OK;
}

lbm_status lbm_mix_batch_destroy(lbm_mix_batch_t b) {
  if (!b) return LBM_ERR_ARG;
  if (b->stream) cudaStreamSynchronize(b->stream);
  b->drop_graph();
  for (lbm_mix* h : b->dom) lbm_mix_destroy(h);
  if (b->pops_all) cudaFree(b->pops_all);
  if (b->side_all) cudaFree(b->side_all);
  if (b->d_params) cudaFree(b->d_params);
  if (b->d_geom) cudaFree(b->d_geom);
  if (b->d_ptrs) cudaFree(b->d_ptrs);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_err) cudaFree(b->d_err);
  for (cudaStream_t x : b->branches) cudaStreamDestroy(x);
  for (cudaEvent_t x : b->joins) cudaEventDestroy(x);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return LBM_OK;
}

const char* lbm_mix_batch_last_error(lbm_mix_batch_t b) { return b ? b->err.c_str() : g_create_error.c_str(); }

lbm_status lbm_mix_destroy(lbm_mix_t h) {
  if (!h) return LBM_ERR_ARG;
  cudaStreamSynchronize(h->stream);
  if (h->owns_buffers) { cudaFree(h->pops); cudaFree(h->scratch); }
  if (h->d_stage) cudaFree(h->d_stage);
  cudaFree(h->d_err); cudaFree(h->d_partials); cudaFree(h->d_sums); cudaFree(h->d_base);
  cudaFree(h->d_w); cudaFree(h->d_img); cudaFree(h->d_stats);
  if (h->z_base) cudaFree(h->z_base);
  if (h->d_jet) cudaFree(h->d_jet);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  delete h;
  return LBM_OK;
}

const char* lbm_mix_last_error(lbm_mix_t h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
