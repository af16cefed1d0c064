/*
 * stokes.h -- C ABI of the GB300 double-layer Stokes solver (libstokes.so).
 *
 * The library solves the boundary-integral system of a 2D Stokes flow in a
 * porous pipe (Coulier, Quaife & Darve, "An efficient preconditioner for the
 * fast simulation of a 2D Stokes flow in porous media"): the domain is the
 * region inside an outer wall Gamma_0 and outside M pores (Sec. 2, Eq. 1),
 * the velocity is prescribed on the whole boundary (Eq. 2 for the pipe
 * flow), and the velocity is represented by the double-layer potential of
 * Sec. 2.1, discretised by collocation at trapezoid-rule nodes (Sec. 2.2,
 * Eq. 5-6). The discrete operator applied to a density sigma is, at node i,
 *
 *   (A sigma)_i = -sigma_i / 2
 *              + sum_{j != i} (w_j / pi) (r.n_j)(r.sigma_j) r / rho^4      r = x_i - x_j
 *              + w_i (-kappa_i / (2 pi)) t_i (t_i . sigma_i)            t = (-n_y, n_x)
 *              + sum_{pores k} S(x_i, c_k) lambda_k + R(x_i, c_k) xi_k
 *              + [i on Gamma_0] n_i sum_{j on Gamma_0} w_j n_j . sigma_j
 *
 * with S(x, c) = (1/4pi)(-log rho I + r r^T / rho^2), R(x, c) = (1/4pi) r^perp / rho^2,
 * r = x - c, (a, b)^perp = (b, -a), lambda_k = sum_{j in k} w_j sigma_j and
 * xi_k = sum_{j in k} w_j (x_j - c_k)^perp . sigma_j. The paper states the
 * kernel and that its rank-3-per-component null space "can be removed"
 * (Sec. 2.1); the diagonal entry (the kernel's limit on a smooth curve), the
 * -1/2 jump, the Stokeslet/rotlet completion and the wall term are the
 * standard completed double-layer formulation chosen to remove it.
 *
 * Conventions for every call:
 *  - Nodes are grouped by component, pores and wall in any order given by
 *    `offsets`; vectors on nodes are interleaved (x, y) pairs, so a density or
 *    a right-hand side is 2N doubles [sx_0, sy_0, sx_1, sy_1, ...].
 *  - Normals are unit vectors pointing OUT OF THE FLUID (out of Gamma_0, into
 *    each pore); kappa is the signed curvature with kappa > 0 on a convex
 *    wall and kappa = -1/R on a pore of radius R.
 *  - Array arguments may be HOST or DEVICE pointers (the library checks with
 *    cudaPointerGetAttributes and copies host data through its own device
 *    buffers); the caller keeps ownership of every array it passes. A handle
 *    owns its device copies, preconditioner factors and workspaces.
 *  - All GPU work of a handle runs on the CUDA stream given at creation.
 *    Calls that return scalars (iteration counts, residuals) or write HOST
 *    outputs synchronise that stream; others are asynchronous.
 *  - Every function returns a status (STOKES_OK = 0 or a negative code);
 *    stokes_last_error() returns a thread-local message for the last failure.
 *    No C++ exception crosses the ABI. A handle is not thread-safe.
 */
#ifndef STOKES_H
#define STOKES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum stokes_status {
  STOKES_OK = 0,
  STOKES_EINVAL = -1,     /* bad argument (sizes, offsets, null pointers, values) */
  STOKES_ENOMEM = -2,     /* device allocation failed */
  STOKES_ECUDA = -3,      /* a CUDA call failed; see stokes_last_error() */
  STOKES_ENOTCONV = -4,   /* GMRES hit max_iter; outputs hold the last iterate */
  STOKES_EBREAKDOWN = -5, /* non-finite residual (NaN/Inf) */
  STOKES_ESTATE = -6      /* call order: e.g. precond apply before setup */
};

/* Arithmetic of the discrete operator.
 * STOKES_FP64: native double precision everywhere.
 * STOKES_FP32: single-precision pair sums and completion (positions split
 *   into float hi + lo parts so that differences of nearby nodes keep single
 *   precision relative to their distance), double-precision diagonal terms,
 *   moments and outputs.
 * STOKES_DF64: double-float pair sums (unevaluated sums of two floats with
 *   error-free transformations) giving FP64-class accuracy on the FP32 pipes.
 * STOKES_MIXED_IR (solve only): FP32 inner GMRES inside FP64 iterative
 *   refinement; the outer residual uses the native FP64 operator. */
enum stokes_precision {
  STOKES_FP64 = 0,
  STOKES_FP32 = 1,
  STOKES_DF64 = 2,
  STOKES_MIXED_IR = 3
};

enum stokes_pc_kind {
  STOKES_PC_NONE = 0,
  STOKES_PC_BLOCKDIAG = 1,
  STOKES_PC_TWOGRID = 2,     /* set up by stokes_precond_setup_twogrid* */
  STOKES_PC_BD_LEARNED = 3,  /* block diagonal + learned coarse correction */
  STOKES_PC_BD_COARSE = 4    /* block diagonal + exact Galerkin coarse correction */
};
enum stokes_pc_side { STOKES_PC_RIGHT = 0, STOKES_PC_LEFT = 1 };

typedef struct stokes_geom stokes_geom;
typedef struct stokes_coarse_model stokes_coarse_model;

/* Build a handle from the discrete boundary (Sec. 2.2: nodes are the
 * collocation points, weights the arclength quadrature weights).
 *   nodes     [2N]   node positions, interleaved (x, y)
 *   normals   [2N]   unit normals, out of the fluid
 *   weights   [N]    quadrature weights, > 0
 *   curvature [N]    signed curvature (see conventions)
 *   offsets   [n_comp+1] HOST int64, offsets[0] = 0, strictly increasing by
 *             at least 8 nodes; component c owns nodes [offsets[c], offsets[c+1])
 *   n_comp    number of components (>= 1); outer_comp in [0, n_comp) is Gamma_0
 *   centres   [2 n_comp] HOST, the completion centre c_k of each pore (the
 *             wall's entry is ignored), or NULL for the quadrature centroid
 *             sum w x / sum w of each component
 *   stream    cudaStream_t (NULL = legacy default stream)
 *   out       receives the handle; unchanged on error
 * Errors: STOKES_EINVAL (sizes, offsets, non-finite or non-positive weights,
 * normals off unit length by > 1e-6), STOKES_ENOMEM, STOKES_ECUDA. */
int stokes_geometry_create(const double* nodes, const double* normals, const double* weights,
                           const double* curvature, const int64_t* offsets, int n_comp,
                           int outer_comp, const double* centres, void* stream,
                           stokes_geom** out);

/* Free a handle and everything it owns (NULL is a no-op). */
int stokes_geometry_destroy(stokes_geom* g);

/* Number of nodes N of a handle (unknowns are 2N); -1 for NULL. */
int64_t stokes_geometry_num_nodes(const stokes_geom* g);

/* y = A sigma (the operator above, Eq. 6 for the double-layer system).
 *   sigma [2N] in, y [2N] out (host or device; may not alias)
 *   precision: STOKES_FP64, STOKES_FP32 or STOKES_DF64.
 * Errors: STOKES_EINVAL, STOKES_ECUDA. */
int stokes_matvec(stokes_geom* g, const double* sigma, double* y, int precision);

/* Build the preconditioner (Sec. 4.1 and its footnote): block diagonal with
 * one block per component, the restriction of A to that component
 * (including its own completion or wall term), assembled on the GPU,
 * LU-factorised with partial pivoting in FP64 and inverted exactly.
 *   pc_kind: STOKES_PC_NONE (drops any existing factors),
 *     STOKES_PC_BLOCKDIAG, or the block diagonal with a second, coarse
 *     level (the paper has no counterpart; see the coarse-model calls
 *     below): STOKES_PC_BD_COARSE (exact Galerkin coarse inverse) or
 *     STOKES_PC_BD_LEARNED (coarse inverse predicted by `model`).
 *   model: a trained or loaded coarse model for STOKES_PC_BD_LEARNED,
 *     otherwise ignored (may be NULL).
 * The coarse level: Z (2N x 3M) holds the rigid motions of each pore p on
 * its nodes (e_x, e_y and (x - c_p)^perp / r_p, (a, b)^perp = (b, -a),
 * r_p = L_p / 2 pi with L_p the sum of the pore's weights), W = diag(w),
 * Y = A Z is formed at setup and with a coarse inverse C each apply is
 *   c = C Z^T W r,  z = Z c + B^-1 (r - Y c)
 * (no extra operator application). Exact: C = E^-1, E = Z^T W Y, inverted
 * by Gauss-Jordan elimination with partial pivoting in FP64 (at most 1365
 * pores). Learned: C holds only the blocks C[p][q] of q = p and the 16
 * pores nearest to p. Memory of the coarse level: 16 N M + 72 M^2 bytes.
 * Errors: STOKES_EINVAL, STOKES_ENOMEM, STOKES_ECUDA; a singular block or
 * coarse operator gives STOKES_EBREAKDOWN; STOKES_ESTATE for a model that
 * was never trained or loaded. */
int stokes_precond_setup(stokes_geom* g, int pc_kind, const stokes_coarse_model* model);

/* Two-grid preconditioner (the paper has no counterpart: a GPU-native
 * alternative to its block-diagonal baseline for densely packed pores):
 *   P^-1 r = I Ac^-1 R r + B^-1 (r - I R r)
 * Ac is the operator above on the coarse grid made of every `coarsen`-th
 * node of every component with weights times `coarsen` (the trapezoid rule
 * on a coarser equispaced parameter grid), assembled densely on the GPU and
 * LU-factorised with partial pivoting in single precision; I is the real
 * trigonometric interpolation of each component's coarse samples (Nyquist
 * cosine split evenly), R = (n_coarse / n_fine) I^T; B^-1 are the pores'
 * diagonal blocks (as in stokes_precond_setup) and -2 I on the wall.
 * Requires every component's node count to be a multiple of `coarsen` with
 * at least 8 coarse nodes, and nodes equispaced in the curve's parameter
 * (the trapezoid rule of Sec. 2.2). Replaces any previous preconditioner;
 * stokes_gmres_solve then runs flexible GMRES, right side only.
 * Memory: 16 (N / coarsen)^2 bytes for the coarse factors.
 * Errors: STOKES_EINVAL (sizes), STOKES_ENOMEM, STOKES_EBREAKDOWN (zero
 * pivot), STOKES_ECUDA. */
int stokes_precond_setup_twogrid(stokes_geom* g, int coarsen);

/* The same with a choice of how the coarse operator is applied:
 *   STOKES_TG_COARSE_AUTO     explicit float inverse up to 40960 coarse
 *                             unknowns (2 N / coarsen), LU factors above
 *   STOKES_TG_COARSE_INVERSE  explicit float inverse (2 m^3 more setup
 *                             flops; each apply one dense GEMV of 4 m^2 bytes)
 *   STOKES_TG_COARSE_LU       the float LU factors through persistent
 *                             triangular solves (the same 4 m^2 bytes per
 *                             apply, no inversion)
 * stokes_precond_setup_twogrid(g, q) is the AUTO mode. The coarse LU is
 * blocked and right-looking: from 8192 coarse unknowns on it takes
 * 128-column panels, each factored as two 64-column sub-panels by one
 * cooperative launch apiece (three launches per column below that size),
 * and its trailing updates run on the tensor cores (three TF32 products per
 * term; STOKES_TG_GEMM=simt keeps the CUDA-core GEMM). The environment
 * variable STOKES_TG_PANEL=coop or =launches forces either panel path (same
 * factors bit for bit). */
enum stokes_tg_coarse { STOKES_TG_COARSE_AUTO = 0, STOKES_TG_COARSE_INVERSE = 1, STOKES_TG_COARSE_LU = 2 };
int stokes_precond_setup_twogrid_ex(stokes_geom* g, int coarsen, int coarse_mode);

/* z = P^-1 v with the current preconditioner (for tests and external
 * Krylov codes). v, z [2N]. STOKES_ESTATE if not set up. */
int stokes_precond_apply(stokes_geom* g, const double* v, double* z);

/* The same with a choice of stored operator: STOKES_FP64 (the double LU
 * factors and inverses above) or STOKES_FP32 (float copies of the explicit
 * inverses of every block, the largest ones inverted from float copies of
 * their factors; used by the FP32 and DF64 solves). */
int stokes_precond_apply_prec(stokes_geom* g, const double* v, double* z, int precision);

/* Solve A sigma = f by restarted GMRES (Sec. 4: GMRES of Saad and Schultz,
 * relative-residual tolerance) with the preconditioner of the last
 * stokes_precond_setup* call (none if never set up). With a right
 * preconditioner the solver keeps the preconditioned basis vectors
 * (flexible GMRES), so preconditioners that round to single precision are
 * safe; the stop is always on the true residual.
 *   f       [2N] right-hand side (the boundary data at the nodes)
 *   tol     relative residual tolerance (> 0)
 *   restart Krylov dimension per cycle, 1..8192 (basis of restart+1 vectors of 2N doubles)
 *   max_iter total inner iterations (>= 1)
 *   precision STOKES_FP64, STOKES_FP32, STOKES_DF64 (operator arithmetic;
 *             Arnoldi, Givens and the least-squares update always FP64; the
 *             true residual, recomputed at every restart, is that of the
 *             chosen operator (FP32 stalls near single precision), except
 *             in DF64 solves: a restart starts from the double-float
 *             residual, and convergence is decided only by the native FP64
 *             operator, which recomputes the residual when the double-float
 *             one reaches tol or stops falling (a cycle started from a
 *             double-float residual aims at 0.3 tol); a DF64 cycle that
 *             starts within 1e4 tol of the tolerance runs its Arnoldi steps
 *             on the FP32 operator: it only has to reduce the residual by at
 *             most 1e4, within the FP32 operator's accuracy on a
 *             correction; when the solve converges or reaches max_iter,
 *             true_relres_out is an FP64 residual) or
 *             STOKES_MIXED_IR
 *             (iterative refinement: outer residual with the FP64 operator,
 *             corrections by GMRES on the FP32 operator until its Arnoldi
 *             residual estimate is below max(1e-4, tol / (2 |r| / |f|));
 *             STOKES_TRACE=1 in the environment prints each step; iters_out counts the
 *             inner iterations, both residual outputs are the outer one)
 *   pc_side STOKES_PC_RIGHT (default; stops on the true residual
 *           |f - A sigma| / |f|) or STOKES_PC_LEFT (Sec. 4.1; stops on the
 *           preconditioned residual |P^-1 (f - A sigma)| / |P^-1 f|)
 *   sigma   [2N] in: initial guess; out: solution
 *   iters_out, true_relres_out, pc_relres_out: HOST scalars (may be NULL)
 * Returns STOKES_OK on convergence, STOKES_ENOTCONV at max_iter (sigma holds
 * the last iterate), STOKES_EBREAKDOWN on a non-finite residual. */
int stokes_gmres_solve(stokes_geom* g, const double* f, double tol, int restart, int max_iter,
                       int precision, int pc_side, double* sigma, int* iters_out,
                       double* true_relres_out, double* pc_relres_out);

/* Velocity at points inside the fluid (Sec. 2.2, Eq. 7 with the
 * double-layer kernel): u(x) = sum_j (w_j / pi)(r.n_j)(r.sigma_j) r / rho^4
 * + sum_k S(x, c_k) lambda_k + R(x, c_k) xi_k, r = x - x_j (no jump, no
 * diagonal term, no wall term). Accurate when the target is farther than
 * about the local node spacing from the boundary (Sec. 2.2 footnote).
 *   sigma [2N]; targets [2T]; u [2T]; precision FP64, FP32 or DF64.
 * A target on a node gives a non-finite value for that target. */
int stokes_eval_velocity(stokes_geom* g, const double* sigma, const double* targets,
                         int64_t n_targets, double* u, int precision);

/* Kernel timing. While enabled, the library brackets every launch of each
 * kernel class below with CUDA events on the handle's stream; launches that
 * a converged GMRES cycle skipped are dropped from the record.
 * stokes_profile_enable(g, on) synchronises the stream, clears the record
 * and switches recording on (on != 0) or off. stokes_profile_read
 * synchronises and returns, for one class, the number of recorded launches,
 * their summed device time in ms and their summed algorithmic work:
 *   PAIRS_*    source-target pairs of the pair sum (all N x T pairs)
 *   EPILOGUE   target-pore pairs of the completion
 *   BD_APPLY   bytes: every block inverse / factor read once, v in, z out
 *   ARNOLDI    bytes of one CGS2 step: 4 (j + 1) + 4 vectors of 2N doubles
 *   BD_SETUP   flops: (2/3) m^3 per block, 2 m^3 where the inverse is formed
 *   LU_GEMM    flops 2 M N K of the trailing-update products of the two-grid
 *              coarse LU (and of its explicit inverse)
 *   LU_PANEL   columns factorised by the coarse LU's panel kernels
 *   COARSE_SOLVE bytes of the coarse factors or inverse read per apply (4 m^2)
 * BD_APPLY covers a whole preconditioner apply; for the two-grid
 * preconditioner its units are the bytes of the coarse factors, the
 * transfer matrices and the pore blocks read once, plus v in and z out.
 * Any output pointer may be NULL. */
enum stokes_prof_kind {
  STOKES_PROF_PAIRS_FP64 = 0,
  STOKES_PROF_PAIRS_FP32 = 1,
  STOKES_PROF_PAIRS_DF64 = 2,
  STOKES_PROF_EPILOGUE = 3,
  STOKES_PROF_BD_APPLY = 4,
  STOKES_PROF_ARNOLDI = 5,
  STOKES_PROF_BD_SETUP = 6,
  STOKES_PROF_LU_GEMM = 7,
  STOKES_PROF_LU_PANEL = 8,
  STOKES_PROF_COARSE_SOLVE = 9
};
int stokes_profile_enable(stokes_geom* g, int on);
int stokes_profile_read(stokes_geom* g, int kind, int64_t* launches, double* total_ms,
                        double* total_units);

/* y = A sigma in FP64 without a handle and without allocating GPU memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate, such as code under an allocator that owns the whole
 * device (a framework memory pool, an embedded runtime with a fixed arena)
 * or on paths where an allocation's implicit device synchronisation is not
 * allowed. It computes the same operator as stokes_matvec with STOKES_FP64,
 * reading the boundary arrays directly instead of a handle.
 *   nodes, normals [2N], weights, curvature [N], sigma, y [2N]: DEVICE arrays
 *   of the current device (or managed memory)
 *   offsets [n_comp+1], centres [2 n_comp] (the completion centres; the
 *   wall's entry is ignored): HOST arrays, copied into the scratch array by
 *   cudaMemcpyAsync on `stream`: pageable memory is read before the call
 *   returns, pinned memory when the copy runs, so keep pinned arrays
 *   unchanged until the stream has passed this call;
 *   n_comp, outer_comp as in stokes_geometry_create;
 *   stream: cudaStream_t (NULL = legacy stream).
 * Its scratch (offsets, centres, moments, split partial sums) lives in one
 * 32 MiB file-scope device array that every GPU loading the library keeps
 * until exit; problems that need more (about 2 million nodes and up) are
 * rejected with STOKES_EINVAL before anything runs, as are host arrays or
 * another device's arrays for the device arguments and the offsets errors
 * of stokes_geometry_create. All calls on a device share that array and
 * leave their contents in it; every call writes all it reads, so nothing
 * needs clearing, but two calls that overlap on the GPU race and give wrong
 * results. The first call on a device looks up the array's address
 * (cudaGetSymbolAddress) with that device current and keeps it for the
 * life of the process (cudaDeviceReset between calls is not supported);
 * make that first call before any stream capture. Asynchronous on
 * `stream`; returns STOKES_OK, STOKES_EINVAL or STOKES_ECUDA and sets no
 * stokes_last_error() message. */
int stokes_matvec_noalloc(const double* nodes, const double* normals, const double* weights,
                          const double* curvature, const int64_t* offsets, int n_comp,
                          int outer_comp, const double* centres, const double* sigma, double* y,
                          void* stream);

/* Launch-shape autotuner of the pair kernels (the paper has no
 * counterpart: its matvec is an FMM on a CPU; here the direct pair sum's
 * best CTA shape depends on the problem size and the arithmetic).
 *
 * Each pair kernel (precision STOKES_FP64, STOKES_FP32 or STOKES_DF64) is
 * compiled in a few shape variants: threads per CTA, targets accumulated
 * per thread, sources per shared-memory tile. Variant 0 is the built-in
 * default. The source range is split so that the grid holds about
 * `ctas_per_sm` CTAs per SM (152 SMs). A handle uses, in this order: the
 * shape set on it (stokes_set_pair_shape or stokes_autotune), the
 * process-wide cache entry of its size class (precision, ceil(log2 N),
 * ceil(log2 T); N sources, T targets), the default (variant 0, 4 CTAs/SM).
 * Every shape computes the same sums in the same order within a thread; the
 * results differ between shapes only through the source splitting
 * (rounding of the partial sums). */

/* Number of compiled shape variants of a precision's pair kernel, or
 * STOKES_EINVAL for an unknown precision. */
int stokes_pair_shape_count(int precision);

/* Threads per CTA, targets per thread and sources per tile of a variant
 * (outputs may be NULL). STOKES_EINVAL for unknown precision or variant. */
int stokes_pair_shape_info(int precision, int variant, int* threads, int* targets_per_thread, int* tile);

/* Fix the shape of a precision's pair kernel on a handle; variant < 0 clears
 * it (back to the cache or the default). ctas_per_sm in [1, 64]. */
int stokes_set_pair_shape(stokes_geom* g, int precision, int variant, int ctas_per_sm);

/* The shape a handle would use for n_targets targets (>= 1). */
int stokes_get_pair_shape(stokes_geom* g, int precision, int64_t n_targets, int* variant, int* ctas_per_sm);

/* Time every (variant, ctas_per_sm in {2, 4, 8}) of the pair kernel alone on
 * the handle's nodes as targets: one warm-up launch and `reps` (1..100) timed
 * launches each, CUDA events on the handle's stream. The fastest is set on
 * the handle and stored in the cache under the handle's size class (T = N).
 * Outputs (may be NULL): the chosen variant and ctas_per_sm and its time per
 * launch in ms. Synchronises the stream. Errors: STOKES_EINVAL, STOKES_ECUDA. */
int stokes_autotune(stokes_geom* g, int precision, int reps, int* variant, int* ctas_per_sm, double* best_ms);

/* The process-wide cache (host only; these calls need no GPU).
 * insert: set the entry of a size class (validated against this build's
 *   variants); lookup: *variant = -1 when there is no entry;
 * save: write all entries to `path` as JSON lines (written to path.tmp, then
 *   renamed), each with precision, log2_sources, log2_targets, variant,
 *   threads, targets_per_thread, tile, ctas_per_sm, ms;
 * load: merge the entries of such a file; lines that do not parse, or whose
 *   variant index or shape does not match this build, are skipped;
 *   *n_loaded (may be NULL) counts the entries taken. A missing file is
 *   STOKES_EINVAL. */
int stokes_tune_cache_insert(int precision, int64_t n_sources, int64_t n_targets, int variant, int ctas_per_sm,
                             double ms);
int stokes_tune_cache_lookup(int precision, int64_t n_sources, int64_t n_targets, int* variant, int* ctas_per_sm,
                             double* ms);
int stokes_tune_cache_clear(void);
int stokes_tune_cache_save(const char* path);
int stokes_tune_cache_load(const char* path, int* n_loaded);

/* Batched operator over many geometries and right-hand sides (the paper
 * has no counterpart; it treats one geometry and one right-hand side at a
 * time). For geometries k < n_geoms and right-hand sides r < n_rhs (1..4),
 * system s = k n_rhs + r:
 *   y[s] = A_k sigma[s]   (the operator of stokes_matvec)
 * sigma[s], y[s]: DEVICE arrays of 2 N_k doubles; the pointer arrays
 * themselves are host memory. The pair sums of all systems run in ONE
 * persistent launch whose CTAs take work items (geometry, block of targets,
 * range of sources) from an atomic counter; the n_rhs densities of a
 * geometry share each pair's geometry (r, 1/rho^2, r.a). precision:
 * STOKES_FP32 or STOKES_DF64 (the arithmetic of stokes_matvec's operator of
 * that precision; results differ from it only in the order of the partial
 * sums). All handles must share one CUDA stream; the call synchronises it.
 * At most 1024 systems. Errors: STOKES_EINVAL, STOKES_ENOMEM, STOKES_ECUDA. */
int stokes_batch_matvec(stokes_geom* const* geoms, int n_geoms, int n_rhs, const double* const* sigma,
                        double* const* y, int precision);

/* Solve A_k sigma[s] = f[s] for every system s = k n_rhs + r (layout as in
 * stokes_batch_matvec) by right-preconditioned flexible GMRES(restart)
 * (Sec. 4) run on all systems in lockstep: each step applies every system's
 * preconditioner (the geometry's last stokes_precond_setup* in float
 * copies; none if never set up), the batched operator and a classical
 * Gram-Schmidt step repeated once, all systems' reductions and Givens
 * rotations in shared launches. A restart cycle is captured once as a CUDA
 * graph and replayed; converged systems' kernels return at once. True
 * residuals |f - A sigma| / |f| are taken with the native FP64 operator at
 * every restart.
 *   precision STOKES_DF64 (double-float operator in the cycles) or
 *             STOKES_MIXED_IR (FP64 residuals per system, corrections by
 *             lockstep FP32 cycles to max(1e-4, tol / (2 relres)), as in
 *             stokes_gmres_solve)
 *   restart 1..1000; max_iter >= 1 (per system, inner iterations for IR)
 *   sigma[s] in: initial guess (DEVICE); out: solution
 *   iters, relres, status: HOST arrays of n_geoms n_rhs entries (may be
 *   NULL): iterations, true relative residual and STOKES_OK,
 *   STOKES_ENOTCONV or STOKES_EBREAKDOWN of each system.
 * A geometry whose two-grid coarse solve runs on its LU factors
 * (STOKES_TG_COARSE_LU, or AUTO above 40960 coarse unknowns) is rejected
 * with STOKES_EINVAL: the captured cycle holds ordinary launches only.
 * The call returns STOKES_OK when it ran (per-system outcomes are in
 * status), else STOKES_EINVAL, STOKES_ENOMEM or STOKES_ECUDA. */
int stokes_batch_solve(stokes_geom* const* geoms, int n_geoms, int n_rhs, const double* const* f, double tol,
                       int restart, int max_iter, int precision, double* const* sigma, int* iters,
                       double* relres, int* status);

/* ---- Learned coarse correction (the paper has no counterpart) ----
 *
 * A network predicts the coarse level's inverse C (see stokes_precond_setup)
 * pore by pore: for pore p, the 3 x 3 blocks C[p][q] for q = p and its 16
 * nearest pores (by centre distance, nearest first, ties to the smaller pore
 * number), in the scaled form L_p L_q C[p][q], from 35 features:
 *   x = [c_x / a, c_y / b, r_p, (c_q - c_p) for the 16 nearest q (zeros where
 *        fewer pores exist)],  a, b = half the wall's extent in x and y.
 * Output o = 9 j + 3 al + be is entry (al, be) of block j (j = 0: q = p).
 * Network: y = relu(relu(x W1 + b1) W2 + b2) W3 + b3, 35 -> 256 -> 256 -> 153,
 * bfloat16 weights and activations on the tensor cores with float
 * accumulation; float master parameters updated by Adam (b1 = 0.9,
 * b2 = 0.999, eps = 1e-8). Parameters: a flat float array W1 [35 x 256], b1,
 * W2 [256 x 256], b2, W3 [256 x 153], b3, matrices row-major.
 * Training: each stokes_coarse_model_add_geometry call computes, on the
 * GPU, the geometry's exact E^-1 (as STOKES_PC_BD_COARSE does) and appends
 * one sample per pore (features, scaled target blocks, a mask of present
 * blocks); stokes_coarse_model_train standardises features and targets with
 * the training set's column means and spreads (population; spreads below
 * 1e-12 count as 1) and takes full-batch Adam steps on the masked mean
 * squared error. Arrays may be host or device memory unless stated; calls
 * synchronise the model's stream. */

/* Number of network parameters (114,329). */
int64_t stokes_coarse_model_num_params(void);

/* A model with initial parameters `params` (n_params floats; the caller
 * draws them) and zero Adam moments; its GPU work runs on `stream`.
 * Errors: STOKES_EINVAL, STOKES_ENOMEM, STOKES_ECUDA. */
int stokes_coarse_model_create(const float* params, int64_t n_params, void* stream, stokes_coarse_model** out);
int stokes_coarse_model_destroy(stokes_coarse_model* model);

/* Append the training samples of a geometry (one per pore; its coarse
 * level is computed on the handle's stream and then dropped). */
int stokes_coarse_model_add_geometry(stokes_coarse_model* model, stokes_geom* g);
/* Number of training samples (-1 for NULL). */
int64_t stokes_coarse_model_num_samples(const stokes_coarse_model* model);

/* `steps` full-batch Adam steps with learning rate lr (> 0); *loss_out
 * (may be NULL) receives the loss of the last step's forward pass.
 * STOKES_ESTATE without samples. */
int stokes_coarse_model_train(stokes_coarse_model* model, int steps, double lr, double* loss_out);

/* Parameters (n_params floats) and standardisation (2 * 35 + 2 * 153
 * floats: feature means, feature spreads, target means, target spreads;
 * may be NULL when saving) out of / into a model (the caller stores them). */
int stokes_coarse_model_save(const stokes_coarse_model* model, float* params, float* stats);
int stokes_coarse_model_load(stokes_coarse_model* model, const float* params, const float* stats);

/* The raw network (no standardisation): y [rows x 153] = net(x [rows x 35]). */
int stokes_coarse_model_forward(stokes_coarse_model* model, const float* x, int64_t rows, float* y);

/* Masked mean squared error L = sum mask (net(x) - t)^2 / sum mask of the
 * raw network and its gradient with respect to the flat parameters
 * (backpropagation through the bfloat16 activations; the output and hidden
 * gradients are rounded to bfloat16 before each product).
 *   x [rows x 35], t, mask [rows x 153]; loss: one double (may be NULL);
 *   grad: n_params floats. */
int stokes_coarse_model_loss_grad(stokes_coarse_model* model, const float* x, const float* t, const float* mask,
                                  int64_t rows, double* loss, float* grad);

/* One Adam step of the parameters with the given gradient (n_params floats). */
int stokes_coarse_model_adam_step(stokes_coarse_model* model, const float* grad, double lr);

/* The coarse-level inputs of a geometry, for checking: features x [M x 35]
 * and neighbour pore numbers nbr [M x 16] (-1 where absent) of its M pores
 * in component order; Y = A Z (2N x 3M, column-major) and E = Z^T W Y
 * (3M x 3M, row-major); outputs may be NULL (stokes_coarse_operator) and
 * host or device memory. Errors: STOKES_EINVAL (no pore, more than 1365). */
int stokes_coarse_features(stokes_geom* g, float* x, int* nbr);
int stokes_coarse_operator(stokes_geom* g, double* y, double* e);

/* Number of library kernels that have started on the current device since
 * the library was loaded (each kernel counts itself once when it begins;
 * kernels that return early because a solve already converged count too).
 * Synchronises the device; -1 on error. */
int64_t stokes_kernel_launches(void);

/* y[i] = 1 / x[i] as the FP64 pair kernel computes it (the paper has no
 * counterpart; exposed so that tests can check it against IEEE division):
 * the hardware's approximate reciprocal (PTX rcp.approx.ftz.f64) refined
 * by two Newton-Raphson steps y <- y + y (1 - x y): within about one ulp
 * for normal positive x; non-finite for x = 0. x, y: DEVICE arrays of n doubles
 * (may alias). Asynchronous on `stream` (NULL = legacy stream).
 * Errors: STOKES_EINVAL, STOKES_ECUDA. */
int stokes_rcp_f64(const double* x, double* y, int64_t n, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* stokes_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* STOKES_H */
