/*
 * lbm_mix.h -- C ABI of the GB300 multicomponent lattice Boltzmann library.
 *
 * One fused stream-and-collide step of the Stefan-Maxwell + compressible
 * two-population model of Sawant, Dorschner & Karlin (arXiv 2004.11286) on
 * the D3Q27 lattice: M species lattices (Sec. 2.5.3, Eqs. SMlbm, fstar1,
 * transform12), the momentum lattice f with the D3Q27 third-moment
 * correction (Sec. 3.4.2, Eqs. feq, fwithcorrection, Xalpha, Ai) and the
 * energy lattice g (Sec. 3.2, Eq. g; Sec. 3.4.1, Eqs. gansatz-gistar),
 * coupled as in Sec. 3.5 (weak or strong coupling).
 *
 * Conventions shared by every call:
 *   - Units: lattice units, dt = dx = 1, constant specific heats with T0 = 0
 *     (Sec. 4.1).
 *   - Node order: x fastest, then y, then z; N = nx*ny*nz nodes.
 *   - Velocity index: i = (cx+1) + 3*(cy+1) + 9*(cz+1), c in {-1,0,1}^3
 *     (Eq. d3q27vel); rest velocity i = 13; opposite of i is 26 - i.
 *   - Lattice index L: 0..M-1 species, M momentum lattice f, M+1 energy
 *     lattice g; S = M + 2 lattices are stored.
 *   - Host/device arguments: a `host_ptrs` flag of 1 means the pointer is a
 *     host address (pinned or pageable); 0 means a device address on the
 *     handle's device.  Arrays are float64, caller-owned, and are only read
 *     or written during the call (host copies are synchronous with respect
 *     to the caller; device-pointer calls are ordered on the handle's
 *     stream and return before the GPU work completes).
 *   - Errors: every call returns an lbm_status; lbm_mix_last_error() gives
 *     a one-line message.  Kernels latch device-side conditions (a node with
 *     non-positive density or temperature, or a non-finite value) into a flag
 *     word; the next call that synchronises (lbm_mix_synchronize,
 *     lbm_mix_diagnostics, host-pointer copies) reports LBM_ERR_NONFINITE.
 *   - Memory: the library owns the handle and a small internal block
 *     (error flag, reduction partials, host staging).  The population and
 *     scratch buffers are either bound by the caller (lbm_mix_bind_buffers;
 *     the caller frees them after lbm_mix_destroy) or allocated by the
 *     library (lbm_mix_alloc_buffers; freed by lbm_mix_destroy).
 *   - Threading: a handle may be used by one host thread at a time.
 */
#ifndef LBM_MIX_H
#define LBM_MIX_H

#include <stddef.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = 1,          /* invalid argument (message says which) */
  LBM_ERR_UNSUPPORTED = 2,  /* valid request the library does not implement */
  LBM_ERR_CUDA = 3,         /* a CUDA runtime call failed */
  LBM_ERR_NONFINITE = 4,    /* a node reached rho <= 0, T <= 0 or NaN */
  LBM_ERR_TIMEOUT = 5,      /* a bounded device wait gave up */
  LBM_ERR_STATE = 6         /* call out of order (e.g. step before init) */
} lbm_status;

/* Boundary types of the six faces (lbm_mix_params.bc).  LBM_BC_JET and
 * LBM_BC_OUTLET make the opposed-jets boundary set of Sec. 4.3; see bc. */
enum { LBM_BC_PERIODIC = 0, LBM_BC_BOUNCEBACK = 1, LBM_BC_JET = 2, LBM_BC_OUTLET = 3 };
/* Precision of the populations in memory and of the arithmetic:
 *   FP64, FP32: stored as deviations from one reference rest state, arithmetic
 *     in the same type;
 *   FP16_STORE, BF16_STORE: FP32 arithmetic; each population stored in 16 bits
 *     as its deviation from the local equilibrium of the node that wrote it
 *     (f - f^eq of Eqs. 27eq, feq, gieq, the node's lattice weights at its
 *     velocity and temperature times its density), scaled per lattice.  Each
 *     collision also writes a per-node FP32 record of the quantities its
 *     equilibria are built from, which the receivers of its populations read
 *     (in the scratch buffer, see lbm_mix_required_bytes). */
enum { LBM_PREC_FP64 = 0, LBM_PREC_FP32 = 1, LBM_PREC_FP16_STORE = 2, LBM_PREC_BF16_STORE = 3 };
enum { LBM_COUPLE_STRONG = 0, LBM_COUPLE_WEAK = 1 };
enum { LBM_CLOSURE_EXACT = 0, LBM_CLOSURE_MLP = 1 };

/* Problem statement as the paper poses it (Secs. 2.1, 2.3, 3.1, 3.3, 3.5). */
typedef struct {
  int M;                      /* number of species, 1..8 */
  const double* molar_mass;   /* [M] m_a > 0; R_a = R_U / m_a (Eq. Ra) */
  const double* cv_molar;     /* [M] C-bar_{a,v} / R_U > 0 (Sec. 3.1, constant heats) */
  const double* D;            /* [M*M] row-major, symmetric binary diffusivities
                                 D_ab > 0 (Eq. smDiffusionCoefficients2).  A
                                 diagonal entry <= 0 selects the default
                                 self-diffusivity: the geometric mean of the
                                 row's off-diagonal entries (M = 1 needs D_11 > 0). */
  const double* mu;           /* [M] species dynamic viscosities mu_a > 0 for the
                                 Wilke rule (Eqs. viscosityMixture, wilkePhi);
                                 may be NULL when omega_fixed > 0 */
  const double* lambda;       /* [M] species conductivities lambda_a > 0 for the
                                 Mathur rule (Eq. conductivityMixture); may be
                                 NULL when omega1_fixed > 0 */
  double omega_fixed;         /* > 0: constant omega instead of Eq. (omega) */
  double omega1_fixed;        /* > 0: constant omega_1 instead of Eq. (omega1) */
  double R_U;                 /* universal gas constant in lattice units (> 0) */
  int nx, ny, nz;             /* grid, each >= 1, fewer than 2^31 nodes */
  int bc[6];                  /* -x,+x,-y,+y,-z,+z: all LBM_BC_PERIODIC, or
                                 LBM_BC_BOUNCEBACK on both x faces with y and z
                                 periodic (the closed tube of Sec. 4.2: halfway
                                 bounce-back of every lattice; gradients mirror
                                 the field across the wall, odd for Phi_x), or
                                 LBM_BC_JET on both x faces, LBM_BC_OUTLET on both
                                 y faces and z periodic: the opposed jets of
                                 Sec. 4.3.  Then the outermost x and y layers of
                                 the grid are a frame of outside nodes that take
                                 no collision: after every collision they hold
                                 the post-collision populations that stream into
                                 the domain.  On the x faces, rows jet_y0 <= y <
                                 jet_y1 are nozzles (the complete equilibrium of
                                 the inlet state, Eqs. 27eq, feq, gieq), the other
                                 rows free-slip walls (the boundary node's mirror
                                 image, x velocity reflected); on the y faces a
                                 copy of the boundary node (zero normal
                                 derivative); a corner takes the x-face rule of
                                 its nearest boundary row.  Gradients read a
                                 frame node as its nearest boundary node, with
                                 Phi_x negated beyond a free-slip wall.  Frame
                                 nodes carry no state of their own (their
                                 observables and conservation sums are not
                                 meaningful).  FP64 and FP32 storage, exact
                                 closure, constant heats only.
                                 Other combinations: LBM_ERR_UNSUPPORTED; walls
                                 or jets with LBM_CLOSURE_MLP or in a batch likewise. */
  int slaved_species;         /* strong coupling: slaved index, -1 -> M-1 (Sec. 3.5.2) */
  int precision;              /* LBM_PREC_* */
  int coupling;               /* LBM_COUPLE_* */
  int closure;                /* LBM_CLOSURE_EXACT, or LBM_CLOSURE_MLP: the learned
                                 network proposes the fluxes of Eq. (transform12)
                                 and the exact solve runs where its residual
                                 exceeds closure_residual_bound (FP32-arithmetic
                                 precisions with M >= 2 only) */
  double fp64_cond_bound;     /* FP32 paths: solve the M x M system of Eq. (transform12)
                                 in FP64 where its 1-norm condition bound exceeds this
                                 (<= 0 -> 1e3) */
  double closure_residual_bound; /* LBM_CLOSURE_MLP: largest accepted
                                 max_{a,c} |(A J~ - r/s)_{a,c}| of the J-form system
                                 in units of s = max|r| (<= 0 -> 1e-2) */
  const double* cv_poly;      /* NULL: constant heats cv_molar.  Else [M][cv_terms]
                                 row-major, temperature-dependent heats (Sec. 3.1):
                                 C-bar_{a,v}(T) / R_U = sum_k cv_poly[a][k] T^k, T0 = 0;
                                 U_a, H_a are their integrals (Eqs. specUa,
                                 specHa) and T solves Eq. (temperature) per node.
                                 C-bar_{a,v} must stay > 0 over the temperatures
                                 reached.  FP64 and FP32 storage; not with walls,
                                 LBM_CLOSURE_MLP or in a batch (LBM_ERR_UNSUPPORTED). */
  int cv_terms;               /* 1..3 coefficients per species with cv_poly */
  /* LBM_BC_JET: the two nozzles, index 0 on the x = 0 face, 1 on x = nx - 1. */
  const double* jet_X;        /* [2][M] inlet mole fractions (each row sums to 1) */
  double jet_u[2];            /* inlet x velocities (into the domain: [0] > 0, [1] < 0) */
  double jet_T[2], jet_P[2];  /* inlet temperatures and pressures (> 0) */
  int jet_y0, jet_y1;         /* nozzle rows [jet_y0, jet_y1), 1 <= jet_y0 <= jet_y1 <= ny - 1 */
} lbm_mix_params;

typedef struct lbm_mix* lbm_mix_t;

/* Validates `p`, derives the constant tables (Wilke phi_ab, 1/(D_ab m_a m_b),
 * C_{a,v}, C_{a,p}) and creates a handle on the current CUDA device.
 * `cuda_stream` is a cudaStream_t (NULL = legacy default stream) on which
 * every later call is ordered.  Allocates only the small internal block. */
LBM_API lbm_status lbm_mix_create(const lbm_mix_params* p, void* cuda_stream, lbm_mix_t* out);

/* Bytes the caller must provide for the populations (S*27*N elements of the
 * storage type) and the scratch side fields (20*N reals, FP64 in FP64 mode,
 * FP32 otherwise: Phi_alpha, 1/omega-1/2, C_p, the q^corr scale and theta
 * written by each collision; G_alpha, K_alpha and the sender's theta; X_alpha
 * of Eq. Xalpha; with temperature-dependent heats the mixture enthalpy's
 * polynomial coefficients and T).  The scratch also carries the previous step's non-local
 * terms, which the next step applies to the arriving populations.  With
 * 16-bit storage the scratch holds, after the side fields (rounded up to 256
 * bytes), two buffers of per-node equilibrium records of
 * 4 * (8 + 4*ceil((M+1)/4) + (weak coupling ? 4 : 0)) bytes each. */
LBM_API lbm_status lbm_mix_required_bytes(lbm_mix_t h, size_t* pops_bytes, size_t* scratch_bytes);

/* Binds caller-owned device buffers (at least the required sizes, 256-byte
 * aligned).  The library never frees bound buffers. */
LBM_API lbm_status lbm_mix_bind_buffers(lbm_mix_t h, void* pops, size_t pops_bytes,
                                void* scratch, size_t scratch_bytes);

/* Allocates the population and scratch buffers with cudaMalloc (freed by
 * lbm_mix_destroy).  For callers without their own allocator. */
LBM_API lbm_status lbm_mix_alloc_buffers(lbm_mix_t h);

/* Equilibrium initial state (Eqs. 27eq, fixed, feq, gieq) from mole fractions
 * X [M][N] (each node summing to 1), velocity u [3][N], temperature T [N] > 0
 * and pressure P [N] > 0.  Resets the step counter to 0. */
LBM_API lbm_status lbm_mix_init_fields(lbm_mix_t h, const double* X, const double* u,
                               const double* T, const double* P, int host_ptrs);

/* Advances nsteps >= 0 time steps (stream + collide of every lattice, Eqs.
 * SMlbm, fwithcorrection, g) in place on the handle's stream (AA pattern:
 * one read and one write of every population per step).  Asynchronous. */
LBM_API lbm_status lbm_mix_step(lbm_mix_t h, int nsteps);

/* Number of outputs of lbm_mix_get_moments for M species: 6 + 5*M. */
LBM_API int lbm_mix_num_outputs(int M);

/* Observables of the current state, [6+5M][N] float64:
 * rho, u_x, u_y, u_z, T, P (Sec. 2.1, Eq. temperature2), X_1..X_M, Y_1..Y_M,
 * then V_a (x,y,z) for a = 1..M, the diffusion velocities of Eq. (transform12)
 * (species velocity u + V_a, Sec. 2.5.3). */
LBM_API lbm_status lbm_mix_get_moments(lbm_mix_t h, double* out, int host_ptrs);

/* Post-streaming populations of the current time level in natural layout
 * [S][27][N] float64 (decoded from the storage precision).  With
 * lbm_mix_set_populations this is the checkpoint / restart interface; set
 * keeps the step counter (the in-place layout depends on its parity). */
LBM_API lbm_status lbm_mix_get_populations(lbm_mix_t h, double* out, int host_ptrs);
LBM_API lbm_status lbm_mix_set_populations(lbm_mix_t h, const double* in, int host_ptrs);

/* Grid sums in float64, deterministic order, written to host sums[M+5]:
 * sum rho_a of each stored species lattice (a = 1..M), sum rho, sum j (3)
 * of the momentum lattice and sum rho*E of the energy lattice.
 * Synchronises the stream and reports latched device errors. */
LBM_API lbm_status lbm_mix_diagnostics(lbm_mix_t h, double* sums);

/* Waits for the handle's stream; reports latched device errors. */
LBM_API lbm_status lbm_mix_synchronize(lbm_mix_t h);

/* Fixes the reference rest state (mass fractions Y[M], normalised here,
 * temperature T > 0, density rho > 0) that every population is stored
 * relative to; init_fields then keeps it instead of deriving one from the
 * fields' means.  Handles whose states are exchanged (z slabs) must share
 * one reference.  The stored state, if any, is invalidated (init again). */
LBM_API lbm_status lbm_mix_set_reference(lbm_mix_t h, const double* Y, double T, double rho);

/* z-slab decomposition of a periodic (or x-walled) grid.  A slab is a handle
 * whose grid is its nz_local planes of the global grid plus `ghost` planes
 * below and above (nz = nz_local + 2 ghost, nz >= 3 ghost), periodic in z
 * within itself.  After every step, each ghost region is refreshed with the
 * `ghost` planes of the neighbouring slab that it mirrors: every population
 * slot (the in-place layout of the current parity), every side field and,
 * with 16-bit storage, both equilibrium-record buffers.  One step reads
 * across at most three planes (the collision's neighbours, then the two
 * stencil passes of the non-local terms of Eq. Xalpha), so with ghost >= 3
 * the interior evolves exactly as the same planes of the undivided grid.
 *   lbm_mix_halo_bytes:  bytes of one face's buffer;
 *   lbm_mix_halo_pack:   copies the `ghost` interior planes next to face
 *                        0 (-z: planes ghost..2 ghost-1) or 1 (+z: planes
 *                        nz-2 ghost..nz-ghost-1) into the device buffer;
 *   lbm_mix_halo_unpack: copies a buffer into the ghost planes of face 0
 *                        (0..ghost-1) or 1 (nz-ghost..nz-1).
 * Slab k's face-1 pack fills slab k+1's face 0, and its face-0 pack slab
 * k-1's face 1 (slab indices periodic).  The buffer is caller-owned device
 * memory, on this device or reachable from it (another GPU's buffer through
 * peer access, or a receive buffer of a collective); ordered on the handle's
 * stream.  LBM_ERR_ARG for a bad face, ghost or grid. */
LBM_API lbm_status lbm_mix_halo_bytes(lbm_mix_t h, int ghost, size_t* bytes);
LBM_API lbm_status lbm_mix_halo_pack(lbm_mix_t h, int face, int ghost, void* buf);
LBM_API lbm_status lbm_mix_halo_unpack(lbm_mix_t h, int face, int ghost, const void* buf);

/* Time steps taken since the last init_fields. */
LBM_API long long lbm_mix_step_count(lbm_mix_t h);

/* Kernel launches issued by this handle since creation (instrumentation). */
LBM_API long long lbm_mix_launch_count(lbm_mix_t h);

/* Instrumentation.  With timing enabled, every step records CUDA events on
 * the handle's stream around each of its kernels (index 0: collide + stream,
 * 1: G_alpha and K_alpha stencil, 2: X_alpha stencil).  lbm_mix_kernel_times synchronises, adds
 * the elapsed times (ms) of all steps recorded since the previous query into
 * ms[0..nk-1], writes the number of launches per kernel into counts, and
 * forgets them.  Returns the number of kernels per step (3). */
LBM_API lbm_status lbm_mix_enable_kernel_timing(lbm_mix_t h, int enable);
LBM_API int lbm_mix_kernel_times(lbm_mix_t h, double* ms, long long* counts, int nk);

/* Conservation sums that allocate nothing (the paper has no counterpart: this
 * is a service of the library).  For callers that cannot call cudaMalloc where
 * they need the sums -- code whose device memory is owned by a pool or arena,
 * plugins that are only handed device pointers, or loops in which an
 * allocation and its implicit synchronisation are not allowed.
 *   pops   device, natural-layout full populations [M+2][27][N] float64
 *          (as written by lbm_mix_get_populations to a device buffer)
 *   sums   device, [M+5] float64 output, same order as lbm_mix_diagnostics
 *   stream cudaStream_t (NULL = legacy default stream); asynchronous
 * The reduction's scratch is a file-scope __device__ array of 2^18 doubles
 * (2 MiB, held by every GPU that loads the library until exit); grids whose
 * per-block partials do not fit (about 5.1e6 nodes at M = 8, 8.4e6 at M = 3)
 * are rejected with LBM_ERR_ARG.  The first call on a device takes the
 * array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture.  Every call shares the one array: calls that overlap on
 * the GPU (different streams, or other host threads) race and must be
 * serialised by the caller.  Errors are reported by lbm_mix_last_error(NULL). */
LBM_API lbm_status lbm_mix_conserved_sums_noalloc(const double* pops, int M, int nx, int ny, int nz,
                                                  double* sums, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Learned Stefan-Maxwell closure.  A network (two hidden layers of width 128
 * with the exact GELU, a linear output layer) stands in for the per-node
 * solve of Eq. (transform12) written for the fluxes J_a = rho_a V_a:
 *   J_a + (1/2) sum_{b!=a} (1/tau_ab)(Y_b J_a - Y_a J_b) = r_a = j_a - rho_a u.
 * Interface (per node, FP32, row-major [rows][F] / [rows][O]):
 *   s = max_{a,c} |r_a,c|;
 *   features, F = pad16(4M + M(M-1)/2 + 1): X_a (a < M); r_a,c / s at
 *     M + 3a + c; h_ab / (1 + h_ab) for a < b in lexicographic order with
 *     h_ab = (1/2)(1/tau_ab)(Y_a + Y_b); the constant 1; zeros;
 *   outputs, O = pad16(3M): J_a,c / s - J0_a,c at 3a + c (the rest unused),
 *     the correction to the one-sweep Jacobi estimate J0_a,c = (r_a,c / s) / A_aa
 *     with A the matrix of the system above; the accepted fluxes are
 *     s (J0 + output).
 * Weights (FP32, packed): W1 [128][F], b1 [128], W2 [128][128], b2 [128],
 * W3 [O][128], b3 [O].  The handle owns an FP32 master copy (trained by the
 * training kernels) and a bf16 image that the tensor-core inference uses
 * (tcgen05, FP32 accumulation), in lbm_mix_closure_forward and, with
 * LBM_CLOSURE_MLP, fused into every step.  A new handle starts with zero
 * weights: the closure is then the Jacobi estimate alone, accepted only
 * where it meets the bound.  All pointers below are device pointers unless
 * stated.
 * ------------------------------------------------------------------------ */

/* F, O and the packed weight count for M species; LBM_ERR_UNSUPPORTED for a
 * species count without kernels. */
LBM_API lbm_status lbm_mix_closure_sizes(int M, int* F, int* O, int* n_weights);

/* Replace the FP32 master weights (host_ptr != 0: `w` is host memory,
 * synchronous) and rebuild the bf16 image; resets the Adam state. */
LBM_API lbm_status lbm_mix_closure_set_weights(lbm_mix_t h, const float* w, int host_ptr);

/* Copy the FP32 master weights out (host_ptr != 0: host memory, synchronous). */
LBM_API lbm_status lbm_mix_closure_get_weights(lbm_mix_t h, float* w, int host_ptr);

/* Training pairs at every node of the current state: features [N][F] and
 * the exact outputs [N][O] (the J-form system solved in FP64, minus the
 * Jacobi estimate), in the node order of the fields.  Stream-ordered. */
LBM_API lbm_status lbm_mix_closure_samples(lbm_mix_t h, float* features, float* targets);

/* Network outputs [n][O] for features [n][F] on the tensor cores with the
 * bf16 image (the arithmetic of the fused inference).  Stream-ordered. */
LBM_API lbm_status lbm_mix_closure_forward(lbm_mix_t h, const float* features, float* outputs, long long n);

/* Mean-squared loss over the n samples and the 3M valid outputs, and its
 * gradient with respect to the FP32 master weights (packed like them) from
 * the FP32 training kernels.  `grad` may be NULL; *loss (host) is written
 * after a synchronisation. */
LBM_API lbm_status lbm_mix_closure_loss_grad(lbm_mix_t h, const float* features, const float* targets,
                                             long long n, float* grad, double* loss);

/* `steps` Adam updates (Kingma & Ba 2015; beta 0.9/0.999, eps 1e-8, rate lr)
 * of the master weights on consecutive mini-batches of `batch` samples taken
 * in order (cyclically) from the n pairs; rebuilds the bf16 image.  The caller
 * shuffles the pairs.  *last_loss (host, may be NULL) is the loss of the last
 * mini-batch, before its update; the call synchronises. */
LBM_API lbm_status lbm_mix_closure_train(lbm_mix_t h, const float* features, const float* targets, long long n,
                                         int batch, int steps, double lr, double* last_loss);

/* Nodes whose network fluxes passed the residual check and nodes that took
 * the exact solve, summed over the steps since the last reset (host values;
 * synchronises).  reset != 0 zeroes the counters after reading. */
LBM_API lbm_status lbm_mix_closure_stats(lbm_mix_t h, long long* accepted, long long* fallback, int reset);

/* ------------------------------------------------------------------------
 * Batched ensemble: many independent periodic domains (uneven grids, each
 * with its own species constants, diffusivities and initial state) stepped
 * together, one launch per kernel for all of them.  Persistent blocks walk a
 * list of tiles (domain, first node); the launch shapes come from
 * lbm_mix_batch_autotune (or lbm_mix_batch_set_config), and pairs of steps
 * (both AA parities) replay as one captured CUDA graph.  Per node the work
 * is exactly that of lbm_mix_step.
 * ------------------------------------------------------------------------ */
typedef struct lbm_mix_batch* lbm_mix_batch_t;

/* `ndomains` parameter blocks (all with the same M, precision and coupling,
 * the exact closure).  The library allocates one population and one scratch
 * buffer for all domains and a non-blocking internal stream; every call is
 * ordered after the work on `cuda_stream`, and the caller's stream waits for
 * the batched step.  Errors: lbm_mix_last_error(NULL). */
LBM_API lbm_status lbm_mix_batch_create(const lbm_mix_params* params, int ndomains, void* cuda_stream,
                                        lbm_mix_batch_t* out);

/* Borrowed handle of domain d for init_fields / set_populations,
 * get_moments, get_populations and diagnostics (not for step, bind or
 * destroy: the batch owns it). */
LBM_API lbm_status lbm_mix_batch_domain(lbm_mix_batch_t b, int d, lbm_mix_t* h);

/* Total nodes over the domains (-1 for NULL). */
LBM_API long long lbm_mix_batch_nodes(lbm_mix_batch_t b);

/* nsteps steps of every domain (all must be initialised and at the same
 * step count).  Asynchronous on the caller's stream. */
LBM_API lbm_status lbm_mix_batch_step(lbm_mix_batch_t b, int nsteps);

/* Times the candidate execution plans on `trial_steps` steps each (graph
 * replays), keeps the fastest and restores the state it started from:
 *   mode 0, persistent launches over the tiles of all domains (collide grid:
 *     one block per tile or 1-4 blocks per SM; stencil blocks of 128 or 256
 *     threads, one per tile or 8/16 per SM);
 *   mode 1, each domain's own kernels (its parameter block by value) on 4, 8
 *     or 16 concurrent branches of the step graph.
 * config (may be NULL) receives [collide grid, stencil block, stencil grid,
 * mode, branches]; *best_ms the step time. */
LBM_API lbm_status lbm_mix_batch_autotune(lbm_mix_batch_t b, int trial_steps, int* config, double* best_ms);

/* Sets the launch shapes by hand; use_graph = 0 launches every step. */
LBM_API lbm_status lbm_mix_batch_set_config(lbm_mix_batch_t b, int grid_collide, int block_stencil,
                                            int grid_stencil, int use_graph);

/* Chooses the execution plan by hand (mode 0 or 1 as in
 * lbm_mix_batch_autotune, 1..64 graph branches for mode 1). */
LBM_API lbm_status lbm_mix_batch_set_mode(lbm_mix_batch_t b, int mode, int branches);

/* config[10]: collide grid, stencil block, stencil grid, graphs on, collide
 * tiles, 128-thread tiles, 256-thread tiles, nodes per collide tile, mode,
 * branches. */
LBM_API lbm_status lbm_mix_batch_config(lbm_mix_batch_t b, int* config);

/* Waits for the batch and reports a non-physical node (LBM_ERR_NONFINITE). */
LBM_API lbm_status lbm_mix_batch_synchronize(lbm_mix_batch_t b);

/* Releases the domains, the shared buffers and the graph. */
LBM_API lbm_status lbm_mix_batch_destroy(lbm_mix_batch_t b);

/* Message of the last error on `b` (of the last failed create if NULL). */
LBM_API const char* lbm_mix_batch_last_error(lbm_mix_batch_t b);

/* Releases the handle, its internal block and library-allocated buffers. */
LBM_API lbm_status lbm_mix_destroy(lbm_mix_t h);

/* Message of the last error on `h` (or of the last failed create if h is NULL). */
LBM_API const char* lbm_mix_last_error(lbm_mix_t h);

#ifdef __cplusplus
}
#endif
#endif /* LBM_MIX_H */
