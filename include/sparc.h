/*
 * sparc.h - C ABI of the GB300 CheFSI library (libsparc.so).
 *
 * The library computes the Chebyshev-filtered subspace iteration (CheFSI)
 * step of real-space Kohn-Sham DFT as described in SPARC for extended systems
 * (arXiv:1603.04339, Section 3.4 "Electron density calculation"):
 *
 *   H(k) = -1/2 nabla_h^2 + V_eff + V_nl                 (Eqn. EL, Eq. FD:Laplacian,
 *                                                          Eq. NonlocalPS:FD)
 *   U_f  = C_m((H - c)/e) U                              (Eq. ChebFilter)
 *   H~ = U_f^H H U_f,  M~ = U_f^H U_f,  H~ y = lambda M~ y
 *                                                        (Eq. SubspaceGeneralizedEigenproblem)
 *   U    = U_f Y                                         (Eq. OrbitalTransformation)
 *
 * Around the step: the SCF iteration at Gamma or over k-points with forces
 * (sparc_scf_*, Sections 2, 3.4-3.6 and 5), filters batched over k-points and
 * over independent cells in one CUDA graph with a launch-shape autotuner, and a
 * learned initial density (sparc_mlp_*, project-added).
 *
 * Conventions that hold for every entry point:
 *   - Grid: n1 x n2 x n3 nodes, spacings h1,h2,h3 (bohr); node (i,j,k), 0-based,
 *     sits at (-L1/2 + i h1, ...), L_s = n_s h_s; grid index g = i + n1 (j + n2 k).
 *   - Orbitals: a column-major Nd x Ns matrix (Nd = n1 n2 n3) in DEVICE memory,
 *     column n starts at X + n*ld elements, ld >= Nd.  Element type by
 *     sparc_dtype; complex values are interleaved (re, im).
 *   - Bloch-periodic boundary: psi(x + L_s e_s) = exp(i k_s L_s) psi(x).  A real
 *     dtype (F64, F32) is only accepted at k = 0 (Gamma point).
 *   - Energies in Hartree, lengths in bohr, k in bohr^-1 (Cartesian).
 *   - Calls are asynchronous on `stream` (a cudaStream_t, NULL = legacy default
 *     stream) unless stated otherwise.  Argument errors are returned at once;
 *     errors found by kernels (non-positive-definite M~, bounded waits that
 *     ran out, a row index outside its array) are latched in a device status
 *     word that sparc_sync() reads.
 *   - The caller owns every buffer it passes.  The context owns its workspace,
 *     which grows on demand and is reused across calls; calls on one context
 *     must not overlap on different streams.
 *   - Nothing throws or aborts across the ABI; every failure is a status code,
 *     and sparc_last_error() gives a one-line reason.
 */
#ifndef SPARC_H
#define SPARC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPARC_OK = 0,
  SPARC_ERR_INVALID_ARG = 1,   /* a size, pointer or bound is out of range          */
  SPARC_ERR_OOM = 2,           /* device allocation of workspace failed             */
  SPARC_ERR_CUDA = 3,          /* a CUDA runtime call failed (message has details)  */
  SPARC_ERR_NOT_POSDEF = 4,    /* M~ is not numerically positive definite           */
  SPARC_ERR_NO_CONVERGENCE = 5,/* the subspace eigensolver hit its sweep limit      */
  SPARC_ERR_TIMEOUT = 6        /* a bounded device wait gave up                     */
} sparc_status;

typedef enum {
  SPARC_F64 = 0,   /* double                          */
  SPARC_F32 = 1,   /* float                           */
  SPARC_C128 = 2,  /* complex double, (re, im) pairs  */
  SPARC_C64 = 3    /* complex float,  (re, im) pairs  */
} sparc_dtype;

/* Rayleigh-Ritz precision modes. */
typedef enum {
  SPARC_RR_FP64 = 0,  /* Grams, eigensolve and rotation in FP64 (input must be F64/C128)   */
  SPARC_RR_MIXED = 1  /* F32 and C64 input: Grams and rotation on tensor cores with
                         3xTF32 error compensation (see sparc_gram_f32, sparc_gram_c64);
                         FP64 factorisations, FP32 Jacobi eigenvectors, FP64 Ritz values */
} sparc_rr_mode;

/* Finite-difference grid at one Bloch wavevector (Section 3.1). */
typedef struct {
  int n[3];          /* nodes per axis, each >= 2*fd_radius + 1                          */
  double h[3];       /* mesh spacing per axis (bohr), > 0                                 */
  int fd_radius;     /* n_o of Eq. FD:Laplacian, 1..8 (paper: 6, twelfth order)           */
  double k[3];       /* Bloch wavevector, Cartesian (bohr^-1)                             */
} sparc_grid;

/* Kleinman-Bylander projectors on cuboid boxes (Eq. NonlocalPS:FD, Section 3.4).
 * Projector p has real values chi[chi_off[p] + a + nb0*(b + nb1*c)] at the
 * unwrapped box node (box_lo[3p] + a, box_lo[3p+1] + b, box_lo[3p+2] + c);
 * box_lo may be negative or >= n (the node maps to its periodic image, which
 * carries the Bloch phase of the cell it lies in).  Each box_n[3p+s] <= n[s].
 * All pointers are HOST pointers, read once by sparc_ham_create. */
typedef struct {
  int nproj;                 /* number of projectors (may be 0)          */
  const int32_t* box_lo;     /* [3*nproj]                                 */
  const int32_t* box_n;      /* [3*nproj]                                 */
  const int64_t* chi_off;    /* [nproj]                                   */
  const double* chi;         /* [chi_len] packed box values               */
  int64_t chi_len;
  const double* gamma;       /* [nproj] KB energies gamma_Jl (Ha)         */
} sparc_nonlocal;

typedef struct sparc_ctx sparc_ctx;   /* device, workspace, status word    */
typedef struct sparc_ham sparc_ham;   /* H(k): grid, V_eff, projectors     */

/* Create a context on CUDA device `device`.  *ctx is NULL on failure. */
sparc_status sparc_create(sparc_ctx** ctx, int device);
void sparc_destroy(sparc_ctx* ctx);
/* One-line description of the last failure on this context ("" if none). */
const char* sparc_last_error(const sparc_ctx* ctx);
/* Synchronise `stream`, then read and clear the device status word: a bounded
 * wait that gave up -> SPARC_ERR_TIMEOUT; M~ not positive definite ->
 * SPARC_ERR_NOT_POSDEF; a gathered row index outside its array ->
 * SPARC_ERR_INVALID_ARG; the eigensolver's sweep limit -> SPARC_ERR_NO_CONVERGENCE
 * (checked in that order when several are latched). */
sparc_status sparc_sync(sparc_ctx* ctx, void* stream);

/* Build H(k) on the context's device: copies the grid, V_eff (host, Nd doubles)
 * and the projector boxes; precomputes FD weights (Eq. weightsLap) and the
 * projector-to-grid maps with their Bloch phases.  Synchronous. */
sparc_status sparc_ham_create(sparc_ctx* ctx, const sparc_grid* grid, const double* veff_host,
                              const sparc_nonlocal* nl, sparc_ham** H);
/* Replace V_eff (Nd doubles).  `on_device` != 0: veff is a device pointer,
 * copied asynchronously on `stream`; otherwise a host pointer (synchronous). */
sparc_status sparc_ham_set_veff(sparc_ham* H, const double* veff, int on_device, void* stream);
/* Free H.  Uses no state of its context, so it may follow sparc_destroy of that
 * context; calls other than this one need a live context. */
void sparc_ham_destroy(sparc_ham* H);

/* Y = H X (Eqn. EL discretised by Eq. FD:Laplacian and Eq. NonlocalPS:FD).
 * X, Y: device, column-major Nd x ns, leading dimension ld; must not overlap. */
sparc_status sparc_apply_H(sparc_ham* H, sparc_dtype dtype, const void* X, void* Y, int ns,
                           int64_t ld, void* stream);

/* Y = H X like sparc_apply_H, but the call itself allocates no device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory at the point of the call, such as applications
 * whose device memory is owned by another allocator or pool (a framework's
 * caching allocator, a fixed memory budget that must not be exceeded), or
 * latency-bound loops that may not block on cudaMalloc, which can synchronise
 * the device.  Its scratch is one fixed array of SPARC_NOALLOC_SCRATCH_BYTES in
 * the library image, present on every GPU that loads the library until the
 * process exits.
 *   - Limit: 2 * ceil(ns/8)*8*Nd + max(nproj,1)*ceil(ns/8)*8 elements of
 *     `dtype` (each part rounded up to 256 bytes) must fit in the array;
 *     larger problems are rejected with SPARC_ERR_INVALID_ARG and a message.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it for the
 *     life of the process; make that first call before any stream capture.
 *     The kept address is stale after cudaDeviceReset on that device, so the
 *     entry point may not be used after such a reset.
 *   - The projector values of H in `dtype` must already be on the device
 *     (any call of sparc_apply_H with that dtype and H uploads them);
 *     otherwise SPARC_ERR_INVALID_ARG.
 *   - All calls on a device share the array: calls that overlap on the GPU
 *     race and must be serialised by the caller.  Every byte a call reads from
 *     it is written earlier in the same call, so nothing needs clearing.
 * Arguments, layout and errors otherwise as sparc_apply_H. */
#define SPARC_NOALLOC_SCRATCH_BYTES (32u << 20)
sparc_status sparc_apply_H_noalloc(sparc_ham* H, sparc_dtype dtype, const void* X, void* Y,
                                   int ns, int64_t ld, void* stream);

/* Scaled Chebyshev filter of degree m (Eq. ChebFilter with e = (b-a)/2, c = (b+a)/2):
 *   Y = C_m((H - c)/e) X / C_m((a0 - c)/e),
 * computed by the three-term recurrence.  a = filter cutoff lambda_c,
 * b = upper bound of the spectrum, a0 = lower estimate; needs a0 < a < b, m >= 1.
 * X, Y: device, column-major Nd x ns (ld); X is not modified; may not overlap. */
sparc_status sparc_cheb_filter(sparc_ham* H, sparc_dtype dtype, int m, double a, double b,
                               double a0, const void* X, void* Y, int ns, int64_t ld,
                               void* stream);

/* The filter of sparc_cheb_filter for nk Hamiltonians that differ only in the
 * Bloch wavevector k (the k-point sum of the density, Section 2 and Section 4:
 * one filter per k-point), run as one sequence of launches: with SPARC_C64 each
 * launch of the H-pass and of the projection covers the blocks of up to 32
 * k-points at once.
 *   H[nk]: Hamiltonians on one context with equal grids (n, h, fd_radius) and
 *          projector boxes (otherwise SPARC_ERR_INVALID_ARG); V_eff, projector
 *          values and k are taken per k.  nk >= 1.
 *   a[nk], b[nk], a0[nk]: host arrays, the bounds of each k (a0 < a < b).
 *   X, Y: device, nk consecutive column-major Nd x ns blocks of leading
 *         dimension ld (block k starts at element k * ns * ld); X is not
 *         modified; X and Y may not overlap.
 * Result: block k equals sparc_cheb_filter(H[k], dtype, m, a[k], b[k], a0[k],
 * ...) bit for bit.  Other dtypes, Hamiltonians outside the tiled kernel's range
 * (fd_radius != 6), and Hamiltonians on the TMA-fed pass (sparc_filter_kernel) whose
 * projector values differ between k, run one sparc_cheb_filter per k.
 * With SPARC_C64 the call's launches are captured once into a CUDA graph held by
 * the context and replayed, one graph launch per call; a call with the same
 * Hamiltonians, sizes and buffers but new bounds updates that graph in place.  (With
 * kernel timing on, the launches are issued one by one.)  Do not call it from inside
 * a stream capture. */
sparc_status sparc_cheb_filter_batch(sparc_ham* const* H, int nk, sparc_dtype dtype, int m,
                                     const double* a, const double* b, const double* a0,
                                     const void* X, void* Y, int ns, int64_t ld, void* stream);

/* Which H-pass kernel sparc_cheb_filter(H, dtype, ...) runs (the recurrence step of
 * Eq. ChebFilter, the H-apply of Section 3.1):
 *   SPARC_KERNEL_GENERIC (0): the per-node kernel (FP64, complex128, fd_radius != 6);
 *   SPARC_KERNEL_TILED (1): the tiled FP32 / complex64 pass;
 *   SPARC_KERNEL_TMA (2): the TMA-fed pass on x-padded blocks (FP32 at the Gamma
 *     point; complex64 at any k, with the projector slots split by periodic image)
 * (without a tuned tile shape).  Returns SPARC_ERR_INVALID_ARG for a null H or
 * out, an unknown dtype or a real dtype for a complex Hamiltonian. */
#define SPARC_KERNEL_GENERIC 0
#define SPARC_KERNEL_TILED 1
#define SPARC_KERNEL_TMA 2
sparc_status sparc_filter_kernel(const sparc_ham* H, sparc_dtype dtype, int* out);

/* Launch-shape autotuner of the filter.  Times sparc_cheb_filter_batch (degree
 * min(m, 4), arguments as there) for several launch configurations, keeps the
 * fastest in the context (among those within 3% of the fastest, the one with
 * the most blocks per launch) and returns its code in *units (0 if the dtype has
 * a single launch shape) with its time in *ms.  A code is
 *   blocks per launch + SPARC_TUNE_SHAPE * tile shape,
 * blocks of 8 orbitals per launch being fractions and multiples of the number
 * whose two live buffers fit in L2, all blocks of one k, or all blocks of all k;
 * the tile shape (SPARC_F32 only) is 0 for 16 x 16 nodes per CTA of 512 threads,
 * 1 for 16 x 8 nodes per CTA of 256 threads (two CTAs per SM).  Later filter
 * calls on this context with the same dtype, Nd, ns and nk use it (nk = 1 for
 * sparc_cheb_filter).  Tuned: SPARC_F32 with nk = 1 and SPARC_C64 with nk > 1.
 * Synchronises `stream`; overwrites Y.  Make it before capturing filter calls
 * into a CUDA graph. */
#define SPARC_TUNE_SHAPE (1 << 20)
sparc_status sparc_autotune_filter(sparc_ham* const* H, int nk, sparc_dtype dtype, int m,
                                   const double* a, const double* b, const double* a0,
                                   const void* X, void* Y, int ns, int64_t ld, void* stream,
                                   int* units, double* ms);

/* Set (units > 0) or clear (units = 0) the launch configuration code (as
 * sparc_autotune_filter returns it: blocks per launch + SPARC_TUNE_SHAPE * tile
 * shape) that later filter calls on this context use for (dtype, Nd, ns, nk),
 * e.g. a code chosen in an earlier process.  With nothing set the filter takes
 * the grouping of its cost model and the 16 x 16 tile. */
sparc_status sparc_set_filter_units(sparc_ctx* ctx, sparc_dtype dtype, int64_t nd, int ns, int nk,
                                    int units);

/* Filter graph: the filters of ncell independent cells -- each its own
 * Hamiltonian (grid, projectors), ns, ld and degree m -- captured once into one
 * CUDA graph whose branches (up to nbranch concurrent streams, cell i on branch
 * i % nbranch) run at the same time, so that small cells fill the GPU together;
 * one sparc_filter_graph_launch then runs every filter of the batch.  Each cell
 * gets its own workspace, allocated here.  The launch shape of every cell is
 * the one its filter call would take when the graph is captured, including a
 * grouping chosen by sparc_autotune_filter (tune the cells first).
 *   H[ncell]: Hamiltonians on one context; m, a, b, a0, ns, ld: host arrays
 *   [ncell]; X[ncell], Y[ncell]: device pointers per cell (layout as
 *   sparc_cheb_filter).  The buffers must stay valid while the graph exists.
 * Result of a launch: Y[i] equals sparc_cheb_filter(H[i], dtype, m[i], a[i],
 * b[i], a0[i], X[i], Y[i], ns[i], ld[i]) bit for bit.  Synchronous; no stream
 * capture may be active on the calling thread. */
typedef struct sparc_filter_graph sparc_filter_graph;
sparc_status sparc_filter_graph_create(sparc_ham* const* H, int ncell, sparc_dtype dtype,
                                       const int* m, const double* a, const double* b,
                                       const double* a0, const void* const* X, void* const* Y,
                                       const int* ns, const int64_t* ld, int nbranch,
                                       sparc_filter_graph** G);
/* New filter bounds for every cell (host arrays [ncell]): re-captures and
 * updates the executable graph in place.  Synchronous. */
sparc_status sparc_filter_graph_set_bounds(sparc_filter_graph* G, const double* a,
                                           const double* b, const double* a0);
/* Run the graph on `stream` (asynchronous). */
sparc_status sparc_filter_graph_launch(sparc_filter_graph* G, void* stream);
/* Free the graph and its workspaces (synchronises the device).  Uses no state
 * of its context, so it may follow sparc_destroy of that context. */
void sparc_filter_graph_destroy(sparc_filter_graph* G);

/* ---------------------------------------------------------------- learned density
 * Project-added (not in the paper): a network that predicts a correction to the
 * superposition of atomic densities from atom-centred descriptors, trained on
 * densities that sparc_scf_step converged; its output feeds
 * sparc_scf_set_density.  Everything runs in the library's kernels (FP32).
 *
 * Descriptors of grid node x (16 per node, widths s_k > 0 in bohr):
 *   D_k(x) = sum_J sum_{T in {-1,0,1}^3 L} exp(-|x - R_J - T|^2 / s_k^2),
 * nodes at -L/2 + i h (x fastest), the frame of sparc_grid.
 * Network: y = relu(relu(D W1 + b1) W2 + b2) w3 + b3, W1 16x128, W2 128x128
 * (row-major), parameters flat [W1, b1, W2, b2, w3, b3] (SPARC_MLP_NPARAM floats).
 * Loss: mean over the points of (y - t)^2.  Optimiser: Adam (b1 = 0.9,
 * b2 = 0.999, eps = 1e-8) with bias correction. */
#define SPARC_MLP_NFEAT 16
#define SPARC_MLP_NHID 128
#define SPARC_MLP_NPARAM (16 * 128 + 128 + 128 * 128 + 128 + 128 + 1)
typedef struct sparc_mlp sparc_mlp;
/* Create with initial parameters (host, SPARC_MLP_NPARAM floats); Adam state zero. */
sparc_status sparc_mlp_create(sparc_ctx* ctx, const float* theta, sparc_mlp** M);
/* set != 0: replace the parameters (host) and reset Adam; set = 0: read them.
 * Synchronises the device. */
sparc_status sparc_mlp_params(sparc_mlp* M, float* theta, int set);
/* D (device, Nd x 16 floats, row per node) for grid n[3], h[3] and natom atoms
 * R (host, 3*natom), widths (host, 16).  Returns after the descriptors are
 * written (synchronises `stream`). */
sparc_status sparc_mlp_descriptors(sparc_ctx* ctx, const int* n, const double* h, int natom,
                                   const double* R, const double* widths, float* D, void* stream);
/* y[p] (device, np floats) = network(D[p]) for D (device, np x 16). */
sparc_status sparc_mlp_forward(sparc_mlp* M, const float* D, int64_t np, float* y, void* stream);
/* Gradient of the loss over the points idx[0..np) (device int64 row indices into
 * the nrows rows of D and t; NULL: rows 0..np-1, np <= nrows) into grad (device,
 * SPARC_MLP_NPARAM floats; may be NULL); *loss (host, may be NULL; then the call
 * does not synchronise).  An index outside [0, nrows) is not read: the point
 * counts as zero and the next synchronising call (sparc_sync) returns
 * SPARC_ERR_INVALID_ARG.  The per-CTA partial sums are reduced in a fixed order:
 * bit-reproducible. */
sparc_status sparc_mlp_grad(sparc_mlp* M, const float* D, const float* t, int64_t nrows,
                            const int64_t* idx, int64_t np, float* grad, double* loss, void* stream);
/* One Adam step with learning rate lr > 0 on the gradient of sparc_mlp_grad. */
sparc_status sparc_mlp_train_step(sparc_mlp* M, const float* D, const float* t, int64_t nrows,
                                  const int64_t* idx, int64_t np, float lr, double* loss, void* stream);
/* Free (synchronises the device); uses no state of its context. */
void sparc_mlp_destroy(sparc_mlp* M);

/* Extremal-eigenvalue estimates by `ksteps` Lanczos steps with full
 * reorthogonalisation, in FP64 (Section 4: filter bounds by the Lanczos method).
 * v0: device start vector, Nd elements of F64 (k = 0) or C128 (k != 0); it is
 * normalised internally and not modified.  On return (the call synchronises
 * `stream`) *a0 = smallest Ritz value, *b = largest Ritz value + |beta_k|.
 * 2 <= ksteps <= 64. */
sparc_status sparc_lanczos_bounds(sparc_ham* H, int ksteps, const void* v0, double* a0, double* b,
                                  void* stream);

/* Rayleigh-Ritz step (Eqs. SubspaceGeneralizedEigenproblem, OrbitalTransformation):
 * H~ = U^H H U, M~ = U^H U, Cholesky M~ = L L^H, C = L^-1 H~ L^-H, C q = lambda q,
 * U <- U L^-H Q.  U: device, column-major Nd x ns (ld), filtered on entry,
 * rotated (orthonormal columns, U^H U = I) on exit.  eig: device, ns doubles,
 * ascending Ritz values.  mode: sparc_rr_mode (FP64 for F64/C128 data, MIXED for
 * F32/C64 data).  2 <= ns <= 1024.  Non-positive-definite M~ or a Jacobi sweep
 * limit are reported by the return code (the call synchronises `stream`). */
sparc_status sparc_rayleigh_ritz(sparc_ham* H, sparc_dtype dtype, void* U, int ns, int64_t ld,
                                 double* eig, int mode, void* stream);

/* The projections of Eq. SubspaceGeneralizedEigenproblem for FP32 data, as
 * sparc_rayleigh_ritz computes them in MIXED mode: G = A^T B, with A, B device,
 * real FP32, column-major nd x ns (lda, ldb >= nd) and G device, FP64,
 * column-major ns x ns.  (H~ = U^T (H U) and M~ = U^T U are the two calls.)
 * Tensor-core products (tcgen05, kind::tf32) of the TF32 high and low parts of
 * both factors (four products), FP32 accumulation over chunks of 64 grid points
 * (the tensor core's accumulation rounds toward zero: sums of squares come out
 * about 2.5e-7 low) and FP64 across chunks;
 * the result is symmetrised (G is taken as symmetric: tiles below the diagonal
 * are the transposes of those above).  Deterministic.  1 <= ns <= 4096. */
sparc_status sparc_gram_f32(sparc_ctx* ctx, const float* A, int64_t lda, const float* B, int64_t ldb,
                            int64_t nd, int ns, double* G, void* stream);

/* The rotation of Eq. OrbitalTransformation for FP32 data: C = U Yr, with U
 * device FP32 column-major nd x ns (ldu), Yr device FP64 column-major ns x ns
 * (rounded to FP32), C device FP32 column-major nd x ns (ldc); C may not
 * overlap U.  Tensor-core products with 3xTF32 compensation.  1 <= ns <= 4096. */
sparc_status sparc_rotate_f32(sparc_ctx* ctx, const float* U, int64_t ldu, const double* Yr, int64_t nd,
                              int ns, float* C, int64_t ldc, void* stream);

/* The projections of Eq. SubspaceGeneralizedEigenproblem for complex64 data (Bloch
 * orbitals at k != 0, Section 3.3), as sparc_rayleigh_ritz computes them in MIXED mode:
 * G = A^H B, with A, B device, complex64 ((re, im) pairs), column-major nd x ns (lda,
 * ldb >= nd) and G device, complex128, column-major ns x ns.  Computed on the real
 * views of the columns (2 nd FP32 values each): Re G = r(A)^T r(B) and
 * Im G = -r(A)^T r(i B), two calls of the sparc_gram_f32 kernels; G is taken as
 * Hermitian (its real part symmetrised, its imaginary part antisymmetrised).  The
 * workspace holds i B (nd x ns complex64).  Deterministic.  1 <= ns <= 4096. */
sparc_status sparc_gram_c64(sparc_ctx* ctx, const void* A, int64_t lda, const void* B, int64_t ldb,
                            int64_t nd, int ns, void* G, void* stream);

/* The rotation of Eq. OrbitalTransformation for complex64 data: C = U Yr, with U
 * device complex64 column-major nd x ns (ldu), Yr device complex128 column-major
 * ns x ns (rounded to FP32), C device complex64 column-major nd x ns (ldc); C may not
 * overlap U.  One tensor-core rotation of the real views, r(C) = r(U) Re Yr +
 * r(i U) Im Yr, with 3xTF32 compensation.  1 <= ns <= 4096. */
sparc_status sparc_rotate_c64(sparc_ctx* ctx, const void* U, int64_t ldu, const void* Yr, int64_t nd,
                              int ns, void* C, int64_t ldc, void* stream);

/* ---------------------------------------------------------------- SCF iteration
 * One self-consistent-field iteration around the CheFSI step (Section 3.4, Eq. EL;
 * Section 5 names the solvers), for one Bloch wavevector of weight 1:
 *   filter bounds (Lanczos, 10 steps from the start vector v0; the cutoff and lower end
 *   are the largest and smallest Ritz values of the previous iteration, or a Weyl
 *   estimate at the first), scaled Chebyshev filter of degree m, Rayleigh-Ritz (mixed
 *   for FP32 data), Fermi level by Brent's method, density
 *   rho = 2 sum g_n |u_n|^2 / (h1h2h3), Poisson -(1/4pi) lap_h phi = rho + b by
 *   conjugate gradients (periodic, zero-mean phi, warm start), LDA (Slater exchange,
 *   Perdew-Wang 1992 correlation), V_out = phi + V_xc, Anderson extrapolation of V_eff
 *   (relaxation mix_beta, history mix_history), and the free energy of
 *   Eq. FreeEnergy:GroundState:DFT:discrete (E_c = 0).  The next V_eff is written into
 *   H.  All grid arithmetic is FP64 and deterministic.
 * Local pseudopotential of atom I: V_I(r) = -Z_I erf(r/rc_I)/r; its pseudocharge
 * b_I = -(1/4pi) lap_h V_I (Eq. PseudochargeDiscrete) on a cube of half-width
 * ceil(6 rc_I / h_s) nodes (charge error below 1e-8), self energy by Eq. DiscreteEself.  sparc_scf_create sets
 * H's V_eff to V_xc of the starting density rho0 = -b (a superposition of Gaussian
 * atomic densities, neutral with the pseudocharges). */
typedef struct {
  int natom;
  const double* R;       /* [3*natom] positions (bohr), frame of the grid (origin at the centre) */
  const double* Z;       /* [natom] valence charges, > 0; N_e = sum Z */
  const double* rc;      /* [natom] widths of the local pseudopotentials (bohr), > 0 */
  double kT;             /* smearing k_B T (Ha), > 0 (the paper: 0.01) */
  double mix_beta;       /* Anderson relaxation, > 0 (the paper: 0.3) */
  int mix_history;       /* Anderson history, 0..8 (the paper: 7) */
  double poisson_tol;    /* relative residual of the Poisson solve, > 0 */
  const double* v0;      /* Lanczos start vector, host: Nd doubles (k = 0) or Nd (re, im) pairs */
  const int32_t* proj_atom; /* [nproj of H] atom of each projector, for sparc_scf_forces; may be NULL */
  int first_passes;      /* CheFSI passes of the first SCF iteration at the starting potential,
                            0..64 (0 and 1: one; Section 4 repeats CheFSI there) */
} sparc_scf_desc;

typedef struct {
  double free_energy;    /* Ha */
  double fermi;          /* lambda_f (Ha) */
  double vresid;         /* |V_out - V_in| / |V_out| of this iteration */
  double nelec;          /* 2 sum g_n (= N_e) */
  double e_band, e_xc, e_el, e_self, e_entropy;   /* the terms of the free energy */
  int poisson_iters;
  double a0, a, b;       /* filter bounds used */
} sparc_scf_info;

typedef struct sparc_scf sparc_scf;
/* Pseudocharges, self energy and the starting V_eff of H.  S uses H in every call but
 * sparc_scf_destroy, so H must outlive the calls on S. */
sparc_status sparc_scf_create(sparc_ham* H, const sparc_scf_desc* d, sparc_scf** S);
/* The same with the Brillouin-zone sum over nk k-points (Section 2; Eq. EL with the
 * k-point weights): H[k] is H(k) for k-point k (equal grids, stencils and projector
 * boxes, one context), wk[k] > 0 its weight (host; they should sum to 1).  The
 * density is 2 sum_k w_k sum_n g_nk |psi_nk|^2 with one Fermi level for all k;
 * every step updates V_eff of every H[k].  With any k != 0, d->v0 holds Nd complex
 * values (2 Nd doubles). */
sparc_status sparc_scf_create_k(sparc_ham* const* H, int nk, const double* wk, const sparc_scf_desc* d,
                                sparc_scf** S);
/* One iteration on the orbitals U (device, column-major Nd x ns, ld >= Nd, dtype F64, F32,
 * C128 or C64; updated in place to the rotated orbitals); eig: device, ns Ritz values.
 * With nk k-points, U holds nk such blocks (k-point k at element k ns ld) and eig
 * nk ns values; the filter of all k runs batched (sparc_cheb_filter_batch), and
 * info's filter bounds are those of the first k-point.  nk ns <= 4096.
 * 2 ns must exceed N_e.  Synchronises `stream`. */
sparc_status sparc_scf_step(sparc_scf* S, sparc_dtype dtype, int m, void* U, int ns, int64_t ld, double* eig,
                            sparc_scf_info* info, void* stream);
/* Copy one grid field (Nd doubles) to the device buffer dst: which = 0 b, 1 rho (last
 * iteration), 2 phi, 3 V_xc, 4 V_out, 5 the current V_eff of H (the next V_in). */
sparc_status sparc_scf_read(const sparc_scf* S, int which, double* dst, void* stream);
/* Starting density (project-added, not in the paper, which starts from the
 * superposition of atomic densities): rho0 = max(-b + scale * dy, 0) scaled to
 * N_e electrons, where -b is that superposition (the pseudocharges of the
 * Gaussian atoms) and dy a correction (device, Nd floats; NULL: none).  Sets
 * V_in = phi[rho0 + b] + V_xc[rho0] (Poisson and LDA as in sparc_scf_step).
 * Only before the first sparc_scf_step of S. */
sparc_status sparc_scf_set_density(sparc_scf* S, const float* dy, double scale, void* stream);
void sparc_scf_destroy(sparc_scf* S);
/* Atomic forces at the state of the last sparc_scf_step (Section 3.6): U are its
 * rotated orbitals, with its occupations and electrostatic potential: F64 or F32 at
 * the Gamma point (one k-point), or C128 / C64 Bloch orbitals of every k-point of S
 * (nk consecutive ns x ld blocks, as sparc_scf_step takes them).  f_host (host,
 * 9*natom doubles): [0, 3 natom) the forces, then the local (Eq. LocalForce:Discrete)
 * and the nonlocal (Eq. NonlocForce:Discrete, the projector derivative moved onto
 * nabla_h psi; for Bloch orbitals with the image phases of Eq. NonlocalPS:FD, the
 * Bloch-wrapped gradient and the k-point weights) parts, 3 per atom, Ha/bohr; the
 * overlap correction f_c is zero (E_c = 0).  Needs sparc_scf_desc.proj_atom when H
 * has projectors.  Synchronises `stream`. */
sparc_status sparc_scf_forces(sparc_scf* S, sparc_dtype dtype, const void* U, int ns, int64_t ld, double* f_host,
                              void* stream);

/* Kernel timing (instrumentation, not part of the method).  While enabled, every
 * launch of the kernels below is bracketed by CUDA events recorded on the
 * stream it is launched on.  sparc_timing_read() synchronises those events and
 * returns the summed device time (ms) and the launch count since the last
 * enable; it is valid after the launches have completed.  Launches issued while
 * their stream is being captured into a CUDA graph are not timed.
 *   which = 0: the H-apply / Chebyshev-recurrence pass of the generic kernel (k_hpass)
 *   which = 1: the nonlocal projection (k_nl_gather, k_gather_rows, k_gather_rows_f2)
 *   which = 2: the Gram products of Rayleigh-Ritz (and sparc_gram_f32, sparc_gram_c64)
 *   which = 3: the Cholesky + subspace eigensolve of Rayleigh-Ritz
 *   which = 4: the subspace rotation of Rayleigh-Ritz (and sparc_rotate_f32, sparc_rotate_c64)
 *   which = 5: the Jacobi sweeps of the subspace eigensolve (inside which = 3)
 *   which = 6: the FP32 / complex64 filter pass (k_pass_tma, k_pass_f2, k_pass_c2)
 *   which = 7, 8, 9: parts of which = 3 in the mixed mode of FP32 data: the first
 *     orthonormalisation's FP32 factorisation; the second factorisation (series or
 *     FP64) with the reduction of H~; the Ritz pairs after the sweeps (Newton-Schulz
 *     step, Rayleigh quotients, order) */
sparc_status sparc_timing_enable(sparc_ctx* ctx, int on);
sparc_status sparc_timing_read(sparc_ctx* ctx, int which, double* ms_total, int64_t* launches);
/* Number of kernels this context has launched since it was created (kernels run from
 * a CUDA graph included, counted when the graph runs). */
sparc_status sparc_launch_count(const sparc_ctx* ctx, int64_t* launches);
/* Number of CUDA graph launches of this context since it was created: the captured
 * Jacobi sweeps, filter graphs and k-point batch filters (each one host launch). */
sparc_status sparc_graph_launch_count(const sparc_ctx* ctx, int64_t* launches);
/* Jacobi sweeps used by the last Rayleigh-Ritz call on this context. */
sparc_status sparc_last_sweeps(const sparc_ctx* ctx, int* sweeps);
/* max |M~1 - I| of the last mixed-mode FP32 Rayleigh-Ritz call on this context: how far
 * from orthonormal its first (FP32 Cholesky) orthonormalisation left the basis, as
 * measured by the Gram of that basis (Section 3.4; -1 before any such call).  At or
 * below 1e-3 the second factorisation ran as a short series in it, above in FP64. */
sparc_status sparc_last_ortho_err(const sparc_ctx* ctx, double* err);

/* Failure injection, for testing the error paths (not part of the method).  All
 * injections are made on the host; none makes a kernel fault, trap or hang.
 *   SPARC_INJECT_ALLOC_FAIL: the next `value` workspace growths of the context fail
 *     as if the device allocation had failed (the calls return SPARC_ERR_OOM and
 *     leave the context usable).
 *   SPARC_INJECT_WAIT_LIMIT: bounded waits of the TMA-fed filter pass give up after
 *     `value` SM clocks (0: the default, about 2^32 clocks).
 *   SPARC_INJECT_STALL: the next launch of the TMA-fed filter pass stops filling its
 *     shared-memory stages at step `value` of each CTA (-1: off), so that the waits
 *     for that stage run out; no copy is left in flight.  The launch latches the
 *     timeout in the status word: the next synchronising call returns
 *     SPARC_ERR_TIMEOUT, and the outputs of that launch are undefined.
 *   SPARC_INJECT_CG_MAX_ITERS: the Poisson solver of sparc_scf_step stops after
 *     `value` conjugate-gradient iterations (0: the default 4000); short of its
 *     tolerance, the step returns SPARC_ERR_NO_CONVERGENCE.
 *   SPARC_INJECT_FP64_ORTHO: the mixed-mode FP32 Rayleigh-Ritz takes its FP64
 *     fallbacks as if the fast paths had failed: value 1, the second factorisation
 *     (in the orthonormalised basis) in FP64 instead of the series; value 2, also the
 *     first orthonormalisation in FP64 instead of the scaled FP32 Cholesky; 0, off.
 * SPARC_ERR_INVALID_ARG for an unknown `what`. */
typedef enum {
  SPARC_INJECT_ALLOC_FAIL = 1,
  SPARC_INJECT_WAIT_LIMIT = 2,
  SPARC_INJECT_STALL = 3,
  SPARC_INJECT_CG_MAX_ITERS = 4,
  SPARC_INJECT_FP64_ORTHO = 5
} sparc_inject;
sparc_status sparc_debug_inject(sparc_ctx* ctx, int what, int64_t value);

#ifdef __cplusplus
}
#endif

#endif /* SPARC_H */
