// lbm_mlp.cuh -- the learned Stefan-Maxwell closure on the 5th-generation
// tensor cores (tcgen05): a network of two hidden layers of width 128 (exact
// GELU) and a linear output layer that maps per-node features to the
// normalised fluxes J_a / s of the M x M system of Eq. (transform12).
//
// Interface (shared by convention with the host packing and the tests):
//   features, F = pad16(4M + M(M-1)/2 + 1):  X_a | r_a,c / s at M + 3a + c |
//     h_ab / (1 + h_ab) for a < b, h_ab = (1/2)(1/tau_ab)(Y_a + Y_b) | 1 | 0...
//   outputs, O = pad16(3M): the correction J_a,c / s - J0_a,c at 3a + c to
//   the one-sweep Jacobi estimate J0_a,c = (r_a,c / s) / A_aa,  s = max |r_a,c|,
//   r_a = j_a - rho_a u  (the right-hand side of the J-form system, matrix A).
//
// One tile is 128 nodes, one per thread and one per TMEM lane (MMA M = 128).
// Operands sit in shared memory as bf16 in the no-swizzle K-major layout of
// 8 x 16-byte core matrices: element (r, k) of an R x K matrix is at byte
//   (r / 8) * 16K + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// so the leading (K) core-matrix stride is 128 bytes and the stride between
// 8-row groups is 16K bytes.  Accumulators are FP32 in TMEM columns [0, 128).
#pragma once

#include <cstdint>

#include <cuda_bf16.h>

#include "lbm_helpers.cuh"

namespace lbm {

constexpr int MLP_H = 128;      // hidden width
constexpr int MLP_TILE = 128;   // nodes per tile = MMA M = TMEM lanes
constexpr int mlp_pad16(int n) { return (n + 15) / 16 * 16; }

template <int M>
struct MlpDims {
  static constexpr int NPAIR = M * (M - 1) / 2;
  static constexpr int F = mlp_pad16(4 * M + NPAIR + 1);
  static constexpr int O = mlp_pad16(3 * M);
  static constexpr int W1_BYTES = MLP_H * F * 2;
  static constexpr int W2_BYTES = MLP_H * MLP_H * 2;
  static constexpr int W3_BYTES = O * MLP_H * 2;
  static constexpr int W_BYTES = W1_BYTES + W2_BYTES + W3_BYTES;
  static constexpr int B_FLOATS = MLP_H + MLP_H + O;            // b1 | b2 | b3, FP32
  static constexpr int IMG_BYTES = W_BYTES + B_FLOATS * 4;       // device weight image
  static constexpr int ACT_BYTES = MLP_TILE * MLP_H * 2;         // one bf16 activation tile
  static constexpr int NW = MLP_H * F + MLP_H + MLP_H * MLP_H + MLP_H + O * MLP_H + O;  // FP32 weights
  static_assert(IMG_BYTES % 16 == 0, "16-byte copies of the weight image");
};

__host__ __device__ constexpr int cm_offset(int r, int k, int K) {
  return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// ---------------------------------------------------------------------------
// tcgen05 / mbarrier primitives (inline PTX).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading byte offset (K
// direction, 128), stride byte offset (8-row groups, 16K), the fixed
// descriptor version bit 46, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, int K) {
  const uint64_t lbo = 128, sbo = (uint64_t)K * 16;
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}
// Instruction descriptor, kind::f16: FP32 accumulate (bits 4-5 = 1), A and B
// bf16 (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int Mt, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(Mt >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {   // one whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {   // one whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// Bounded wait on the phase with the given parity; false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// 16 consecutive FP32 columns of this thread's TMEM lane (the wait is in the
// same statement, so the registers are valid when it returns).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all16() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_all;\n" ::: "memory");
}

// Bulk (TMA engine) copy of `bytes` contiguous bytes global -> shared,
// completing on an mbarrier; both addresses 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gsrc, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(smem_dst)),
               "l"(gsrc), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ float gelu_exact(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}
// Writes 8 consecutive values (k0 multiple of 8) of row r of a K-wide bf16 tile.
__device__ __forceinline__ void store_row8(unsigned char* tile, int r, int k0, int K, const float* v) {
  uint4 q;
  q.x = pack_bf16x2(v[0], v[1]); q.y = pack_bf16x2(v[2], v[3]);
  q.z = pack_bf16x2(v[4], v[5]); q.w = pack_bf16x2(v[6], v[7]);
  *reinterpret_cast<uint4*>(tile + cm_offset(r, k0, K)) = q;
}

// ---------------------------------------------------------------------------
// Per-block state of the network for T tiles of 128 rows (block of 128 T
// threads, thread t on row t % 128 of tile t / 128): weights image (shared by
// the tiles), one activation tile, mbarrier and 128 TMEM columns per tile.
// Shared-memory layout (from `base`, 16-byte aligned):
//   [W1 | W2 | W3 (bf16 core-matrix images) | b1 b2 b3 (FP32)] [act x T] [mbar x T] [TMEM slot]
// ---------------------------------------------------------------------------
template <int M, int T = 1>
constexpr int mlp_smem() {
  return (MlpDims<M>::IMG_BYTES + T * MlpDims<M>::ACT_BYTES + 8 * T + 8 + 15) / 16 * 16;
}

template <int M, int T = 1>
struct MlpBlock {
  using D = MlpDims<M>;
  static_assert(T == 1 || T == 2, "one or two tiles per block");
  unsigned char* base;
  uint32_t tmem;
  uint32_t phase;
  __device__ int tile() const { return (int)threadIdx.x / MLP_TILE; }
  __device__ int row() const { return (int)threadIdx.x % MLP_TILE; }
  __device__ unsigned char* act() const { return base + D::IMG_BYTES + tile() * D::ACT_BYTES; }
  __device__ unsigned char* act_of(int k) const { return base + D::IMG_BYTES + k * D::ACT_BYTES; }
  __device__ const float* bias() const { return reinterpret_cast<const float*>(base + D::W_BYTES); }
  __device__ uint32_t mbar_of(int k) const { return smem_u32(base + D::IMG_BYTES + T * D::ACT_BYTES + 8 * k); }
  __device__ uint32_t* slot() const {
    return reinterpret_cast<uint32_t*>(base + D::IMG_BYTES + T * D::ACT_BYTES + 8 * T);
  }
  // TMEM address of this thread's lane quadrant in its tile's columns.
  __device__ uint32_t lane_addr() const {
    return tmem + (uint32_t)(MLP_TILE * tile()) + ((uint32_t)(row() & ~31) << 16);
  }

  // Every thread: start the weight-image copy (completed by finish_setup).
  __device__ void begin_setup(const unsigned char* __restrict__ img) {
    for (int o = threadIdx.x * 16; o < D::IMG_BYTES; o += blockDim.x * 16) cp_async16(base + o, img + o);
    if (threadIdx.x < 32) tmem_alloc(smem_u32(slot()), MLP_TILE * T);
    if (threadIdx.x == 0)
      for (int k = 0; k < T; ++k) mbar_init(mbar_of(k), 1);
    phase = 0;
  }
  __device__ void finish_setup() {
    cp_async_wait_all16();
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    tmem = *reinterpret_cast<volatile uint32_t*>(slot());
  }
  __device__ void teardown() {
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(tmem, MLP_TILE * T);
  }

  // The first thread of each tile issues act[128 x K] . W[N x K]^T into its
  // tile's TMEM columns; every thread waits for its tile.  Every thread takes
  // the same barriers whatever happens, and the result is block-uniform (a
  // timed-out wait sets bit 4 of *err).
  __device__ bool layer(uint32_t w_saddr, int K, int N, bool run, unsigned* err) {
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    bool ok = run;
    if (run) {
      if (row() == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(act()), idesc = umma_idesc_bf16(MLP_TILE, N);
        const uint32_t d = tmem + (uint32_t)(MLP_TILE * tile());
        for (int kk = 0; kk < K / 16; ++kk)
          umma_bf16(d, umma_desc(a0 + kk * 256, K), umma_desc(w_saddr + kk * 256, K), idesc, kk > 0 ? 1u : 0u);
        umma_commit(mbar_of(tile()));
      }
      ok = mbar_wait(mbar_of(tile()), phase);
      phase ^= 1u;
      tc_fence_after();
    }
    ok = __syncthreads_and(ok) != 0;
    if (run && !ok && threadIdx.x == 0) atomicOr(err, 4u);
    return ok;
  }
  // Hidden-layer epilogue: bias + GELU of this thread's row, back into act as bf16.
  __device__ void hidden_epilogue(const float* b) {
    const uint32_t la = lane_addr();
#pragma unroll 1
    for (int c = 0; c < MLP_H / 16; ++c) {
      float v[16];
      tmem_ld16(la + c * 16, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = gelu_exact(v[i] + b[c * 16 + i]);
      store_row8(act(), row(), c * 16, MLP_H, v);
      store_row8(act(), row(), c * 16 + 8, MLP_H, v + 8);
    }
  }

  // Full network for the rows already written to this thread's tile (K = F
  // layout); this thread's outputs in out[0, O).
  __device__ bool forward(float (&out)[D::O], unsigned* err) {
    const uint32_t w1 = smem_u32(base), w2 = w1 + D::W1_BYTES, w3 = w2 + D::W2_BYTES;
    const float* b = bias();
    bool ok = layer(w1, D::F, MLP_H, true, err);
    if (ok) hidden_epilogue(b);
    ok = layer(w2, MLP_H, MLP_H, ok, err);
    if (ok) hidden_epilogue(b + MLP_H);
    ok = layer(w3, MLP_H, D::O, ok, err);
    const uint32_t la = lane_addr();
#pragma unroll
    for (int c = 0; c < D::O / 16; ++c) {
      float v[16];
      if (ok) tmem_ld16(la + c * 16, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) out[c * 16 + i] = ok ? v[i] + b[2 * MLP_H + c * 16 + i] : 0.0f;
    }
    return ok;
  }
};

// ---------------------------------------------------------------------------
// Features of one node (the interface above) and the residual of the J-form
// system of Eq. (transform12) for a proposed normalised flux.
// ---------------------------------------------------------------------------
template <int M, class Real>
__device__ __forceinline__ void sm_feature_values(const DevParams<Real>& p, const Thermo<M, Real>& th,
                                                  const Real (&itab)[M][M], const Real (&r)[M][3], Real inv_s,
                                                  float (&f)[MlpDims<M>::F]) {
#pragma unroll
  for (int k = 0; k < MlpDims<M>::F; ++k) f[k] = 0.0f;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    f[a] = (float)(th.m * th.Y[a] * p.inv_mass[a]);
#pragma unroll
    for (int c = 0; c < 3; ++c) f[M + 3 * a + c] = (float)(r[a][c] * inv_s);
  }
  int k = 4 * M;
#pragma unroll
  for (int a = 0; a < M; ++a)
#pragma unroll
    for (int b = a + 1; b < M; ++b) {
      const Real h = Real(0.5) * itab[a][b] * (th.Y[a] + th.Y[b]);
      f[k++] = (float)(h / (Real(1) + h));
    }
  f[k] = 1.0f;
}

// Diagonal of the J-form matrix A of Eq. (transform12): 1 + (1/2) sum_{b!=a} (1/tau_ab) Y_b.
template <int M, class Real>
__device__ __forceinline__ void sm_diagonal(const Thermo<M, Real>& th, const Real (&itab)[M][M], Real (&d)[M]) {
#pragma unroll
  for (int a = 0; a < M; ++a) {
    d[a] = Real(1);
#pragma unroll
    for (int b = 0; b < M; ++b)
      if (b != a) d[a] += Real(0.5) * itab[a][b] * th.Y[b];
  }
}

// max_{a,c} |(A J~)_a,c - r~_a,c| for the J-form matrix A of Eq. (transform12).
template <int M, class Real>
__device__ __forceinline__ Real sm_residual(const Thermo<M, Real>& th, const Real (&itab)[M][M], const Real (&diag)[M],
                                            const Real (&rn)[M][3], const Real (&Jn)[M][3]) {
  Real res = Real(0);
#pragma unroll
  for (int a = 0; a < M; ++a) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Real s = diag[a] * Jn[a][c] - rn[a][c];
#pragma unroll
      for (int b = 0; b < M; ++b)
        if (b != a) s -= Real(0.5) * itab[a][b] * th.Y[a] * Jn[b][c];
      res = fmax(res, fabs(s));
    }
  }
  return res;
}

// ---------------------------------------------------------------------------
// Kernels: FP32 weights -> bf16 image, and the network on given features.
// ---------------------------------------------------------------------------
template <int M>
__global__ void mlp_pack_kernel(const float* __restrict__ w, unsigned char* __restrict__ img) {
  using D = MlpDims<M>;
  const long long e = gtid();
  if (e >= D::NW) return;
  __nv_bfloat16* wb = reinterpret_cast<__nv_bfloat16*>(img);
  float* bi = reinterpret_cast<float*>(img + D::W_BYTES);
  long long k = e;
  if (k < (long long)MLP_H * D::F) {                       // W1 [H][F]
    const int r = (int)(k / D::F), c = (int)(k % D::F);
    wb[cm_offset(r, c, D::F) / 2] = __float2bfloat16_rn(w[e]);
    return;
  }
  k -= (long long)MLP_H * D::F;
  if (k < MLP_H) { bi[k] = w[e]; return; }                 // b1
  k -= MLP_H;
  if (k < (long long)MLP_H * MLP_H) {                      // W2 [H][H]
    const int r = (int)(k / MLP_H), c = (int)(k % MLP_H);
    wb[(D::W1_BYTES + cm_offset(r, c, MLP_H)) / 2] = __float2bfloat16_rn(w[e]);
    return;
  }
  k -= (long long)MLP_H * MLP_H;
  if (k < MLP_H) { bi[MLP_H + k] = w[e]; return; }         // b2
  k -= MLP_H;
  if (k < (long long)D::O * MLP_H) {                       // W3 [O][H]
    const int r = (int)(k / MLP_H), c = (int)(k % MLP_H);
    wb[(D::W1_BYTES + D::W2_BYTES + cm_offset(r, c, MLP_H)) / 2] = __float2bfloat16_rn(w[e]);
    return;
  }
  k -= (long long)D::O * MLP_H;
  bi[2 * MLP_H + k] = w[e];                                // b3
}

// out[n][O] = network(feat[n][F]) with bf16 operands on the tensor cores.
template <int M>
__global__ void __launch_bounds__(MLP_TILE, 1)
mlp_forward_kernel(const unsigned char* __restrict__ img, const float* __restrict__ feat, float* __restrict__ out,
                   long long n, unsigned* __restrict__ err) {
  using D = MlpDims<M>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  MlpBlock<M, 1> mlp{smem_raw, 0u, 0u};
  mlp.begin_setup(img);
  const long long row = (long long)blockIdx.x * MLP_TILE + threadIdx.x;
  float f[D::F];
#pragma unroll
  for (int k = 0; k < D::F; ++k) f[k] = row < n ? feat[row * D::F + k] : 0.0f;
#pragma unroll
  for (int k0 = 0; k0 < D::F; k0 += 8) store_row8(mlp.act(), threadIdx.x, k0, D::F, f + k0);
  mlp.finish_setup();
  float o[D::O];
  mlp.forward(o, err);
  if (row < n) {
#pragma unroll
    for (int k = 0; k < D::O; ++k) out[row * D::O + k] = o[k];
  }
  mlp.teardown();
}

}  // namespace lbm
