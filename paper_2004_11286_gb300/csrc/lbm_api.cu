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
#include "lbm_dispatch.h"

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
  d.omega_is_fixed = s.omega_is_fixed; d.omega1_is_fixed = s.omega1_is_fixed;
  d.omega_fixed = (Real)s.omega_fixed; d.omega1_fixed = (Real)s.omega1_fixed;
  d.R_U = (Real)s.R_U; d.cond_bound = (Real)s.cond_bound;
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
  bool has_reference = false;
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
  bool initialized = false;
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;   // 4 per recorded step
  size_t ev_used = 0;
  std::string err;

  size_t need_pops() const { return (size_t)(M + 2) * 27 * (size_t)N * store_elem_bytes(prec); }
  size_t need_scratch() const { return (size_t)lbm::NSIDE * (size_t)N * side_elem_bytes(prec); }
  lbm::LaunchCtx ctx() {
    lbm::LaunchCtx c;
    c.N = N; c.stream = stream; c.pops = pops; c.side = scratch; c.err = d_err;
    c.partials = d_partials; c.p64 = &p64; c.p32 = &p32; c.base = d_base; c.ev = nullptr;
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
    if (flag) return fail(LBM_ERR_NONFINITE, "a node reached non-positive density or temperature (or NaN)");
    return LBM_OK;
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
    double inv_m = 0.0, Cv = 0.0;
    for (int a = 0; a < M; ++a) { inv_m += Y[a] * d.inv_mass[a]; Cv += Y[a] * d.Cv_a[a]; }
    const double R = d.R_U * inv_m, th = R * T;
    for (int a = 0; a < M; ++a)
      for (int i = 0; i < 27; ++i) base[a * 27 + i] = Y[a] * rho * W(i, d.R_a[a] * T);     // Eq. (27eq) at rest
    for (int i = 0; i < 27; ++i) base[M * 27 + i] = rho * W(i, th);                      // Eq. (feq) at rest
    const double rhoE = rho * Cv * T, P = rho * th, Z = 0.5 * (1.0 - 3.0 * th) * P;
    for (int i = 0; i < 27; ++i) {                                                       // Eq. (gieq) at rest
      const int c2 = lbm::c2_of(i);
      const double E = rhoE - 1.5 * P + 0.5 * c2 * rho;
      const double BZ = c2 == 0 ? 3.0 * Z : (c2 == 1 ? -0.5 * Z : 0.0);
      base[(M + 1) * 27 + i] = W(i, th) * E + BZ;
    }
    for (int L = 0; L < lbm::MAXM + 2; ++L) { d.RL[L] = 0.0; d.scale[L] = 1.0; d.inv_scale[L] = 1.0; }
    for (int L = 0; L < S; ++L) {
      double sum = 0.0;
      for (int i = 0; i < 27; ++i) sum += base[L * 27 + i];
      d.RL[L] = sum;
      if (prec == LBM_PREC_FP16_STORE || prec == LBM_PREC_BF16_STORE) {
        d.scale[L] = 1.0 / std::fabs(sum);
        d.inv_scale[L] = std::fabs(sum);
      }
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
    double Y[lbm::MAXM], Cv = 0.0;
    for (int a = 0; a < M; ++a) { Y[a] = r[a] / tot; Cv += Y[a] * p64.Cv_a[a]; }
    return set_reference(Y, rhoE / (rho * Cv), rho);
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
    if (p->bc[s] != LBM_BC_PERIODIC) { g_create_error = "only periodic boundaries are built"; return LBM_ERR_UNSUPPORTED; }
  if (p->precision < LBM_PREC_FP64 || p->precision > LBM_PREC_BF16_STORE) return bad("unknown precision");
  if (p->coupling != LBM_COUPLE_STRONG && p->coupling != LBM_COUPLE_WEAK) return bad("unknown coupling");
  if (p->closure != LBM_CLOSURE_EXACT) { g_create_error = "only the exact Stefan-Maxwell closure is built"; return LBM_ERR_UNSUPPORTED; }
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

  const lbm::KernelSet* ks = select_kernels(M, p->precision);
  if (!ks) { g_create_error = "no kernels built for this (M, precision)"; return LBM_ERR_UNSUPPORTED; }

  lbm_mix* h = new (std::nothrow) lbm_mix();
  if (!h) return bad("out of host memory");
  h->M = M; h->prec = p->precision; h->ks = ks;
  h->N = (long long)p->nx * p->ny * p->nz;
  h->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&h->device);

  lbm::DevParams<double>& d = h->p64;
  d.N = h->N; d.nx = p->nx; d.ny = p->ny; d.nz = p->nz; d.M = M; d.slaved = slaved;
  d.weak = p->coupling == LBM_COUPLE_WEAK;
  d.omega_is_fixed = p->omega_fixed > 0.0; d.omega1_is_fixed = p->omega1_fixed > 0.0;
  d.omega_fixed = p->omega_fixed; d.omega1_fixed = p->omega1_fixed; d.R_U = p->R_U;
  d.cond_bound = p->fp64_cond_bound > 0.0 ? p->fp64_cond_bound : 1e3;
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
  d.rho_eps = 1e-14;
  fill_params<float>(h->p32, d);
  h->p32.rho_eps = 1e-7f;

  const long long nblocks = (h->N + 255) / 256;
  cudaError_t e = cudaMalloc(&h->d_err, 256);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_partials, (size_t)nblocks * 16 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_base, sizeof(double) * (lbm::MAXM + 2) * 27);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_sums, 16 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, 256, h->stream);
  if (e != cudaSuccess) {
    g_create_error = std::string("CUDA: ") + cudaGetErrorString(e);
    if (h->d_err) cudaFree(h->d_err);
    if (h->d_partials) cudaFree(h->d_partials);
    if (h->d_sums) cudaFree(h->d_sums);
    if (h->d_base) cudaFree(h->d_base);
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
  if ((s = h->reference_from_fields(dX, dT, dP)) != LBM_OK) return s;
  if ((s = h->clear_pending()) != LBM_OK) return s;
  if ((s = h->cuda(h->ks->init(h->ctx(), dX, du, dT, dP), "init kernel")) != LBM_OK) return s;
  h->launches += 1;
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
    h->launches += h->ks->launches_per_step;
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
  h->launches += 1;
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

lbm_status lbm_mix_destroy(lbm_mix_t h) {
  if (!h) return LBM_ERR_ARG;
  cudaStreamSynchronize(h->stream);
  if (h->owns_buffers) { cudaFree(h->pops); cudaFree(h->scratch); }
  if (h->d_stage) cudaFree(h->d_stage);
  cudaFree(h->d_err); cudaFree(h->d_partials); cudaFree(h->d_sums); cudaFree(h->d_base);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  delete h;
  return LBM_OK;
}

const char* lbm_mix_last_error(lbm_mix_t h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
