/*
 * vps.h -- C ABI of the GB300 vertex-patch multigrid library.
 *
 * The library solves the Poisson problem -Laplace u = f on (0,1)^d,
 * u = 0 on the boundary (d = 2, 3; Section 2, Eq. 2.1), discretised with
 * continuous Q_k Lagrange elements on Gauss-Lobatto support points on the
 * uniform mesh with 2^level cells per direction (Section 2, Eq. 2.2-2.4).
 * Its hot path is the geometric multigrid V-cycle (Algorithm 1) with a
 * vertex-patch Schwarz smoother (Section 2.2, Algorithm 3) whose local
 * solves use fast diagonalisation (Section 2.4, Eq. 2.13-2.15), the
 * matrix-free operator (Section 2.3) and the grid transfers (Section 2.1),
 * inside a preconditioned conjugate-gradient solver.
 *
 * Conventions shared by every call
 * --------------------------------
 * Return value: VPS_OK (0) or a negative VPS_E* code; no call aborts the
 *   process.  vps_last_error() returns a message for the last failure.
 * Handle: created by vps_create, owns the level hierarchy, the 1D tables
 *   and all workspaces (device memory allocated at creation).  A handle is
 *   used by one host thread at a time; all its work is issued on the CUDA
 *   stream given to vps_create, asynchronously unless stated otherwise.
 * Device vectors: every vector argument is a caller-owned DEVICE pointer
 *   (e.g. a PyTorch tensor's data_ptr()), valid for the stream of the
 *   handle.  They must not alias each other unless a call says so.
 * Working precision: VPS_FP64 handles store level vectors as double,
 *   VPS_FP32 handles as float ("void*" arguments below are of that type).
 *   vps_solve always takes double vectors: with VPS_FP32 the V-cycle runs
 *   in float inside a double-precision CG (mixed precision, Section 4.2).
 * Level layout: a vector of level l holds all n1 = k 2^l + 1 nodes per
 *   direction including the boundary, lexicographic with dimension 0
 *   fastest, rows padded to `row_pitch` elements (vps_level_layout); entry
 *   (i0,i1[,i2]) sits at i0 + row_pitch*(i1 + n1*i2).  Boundary nodes and
 *   padding are ignored on input and written as 0 on output.
 * Compact layout: interior nodes only, (n1-2)^d entries, lexicographic with
 *   dimension 0 fastest.  This is the ordering of the paper's DoF layout
 *   (Section 3.1.2) with the Dirichlet nodes eliminated.
 */
#ifndef VPS_H
#define VPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vps_context* vps_handle;

/* status codes */
#define VPS_OK          0
#define VPS_EINVAL     -1  /* bad argument (dimension, degree, level, pointer, damping, ...) */
#define VPS_ENOMEM     -2  /* device allocation failed */
#define VPS_ECUDA      -3  /* a CUDA runtime call or kernel launch failed */
#define VPS_ENOCONV    -4  /* CG reached max_it without meeting the tolerance */
#define VPS_EBREAKDOWN -5  /* CG breakdown: p^T A p <= 0 or a non-finite scalar */
#define VPS_ETIMEOUT   -6  /* a bounded device-side wait expired */

/* precision */
#define VPS_FP64 0         /* everything in double */
#define VPS_FP32 1         /* float level vectors and V-cycle; double outer CG */

/* smoother */
#define VPS_MULTIPLICATIVE 0  /* 2^d-colour multiplicative Schwarz, Algorithm 3 */
#define VPS_ADDITIVE       1  /* damped additive Schwarz over the same patches */

#define VPS_MAX_DEGREE 7

/*
 * vps_create -- build the hierarchy for Q_degree on 2^level cells per direction.
 *   dim 2 or 3; degree 1..7; level >= 1 with at most 2^31 nodes per level
 *   vector; precision VPS_FP64 or VPS_FP32; smoother VPS_MULTIPLICATIVE or
 *   VPS_ADDITIVE; damping > 0 (used by the additive smoother; the
 *   multiplicative one is undamped as in Algorithm 3); n_pre, n_post >= 0
 *   smoothing steps per level in the V-cycle (Algorithm 1 uses 1 and 1).
 *   cuda_stream: a cudaStream_t (NULL = legacy default stream; CUDA graphs
 *   are only used on non-default streams).  On success *out receives the
 *   handle.  Allocates all device memory; synchronous.
 *   Errors: VPS_EINVAL (checked before any CUDA call), VPS_ENOMEM, VPS_ECUDA.
 */
int vps_create(int dim, int degree, int level, int precision, int smoother,
               double damping, int n_pre, int n_post, void* cuda_stream,
               vps_handle* out);

/* vps_destroy -- synchronise the stream and free everything. NULL is a no-op. */
int vps_destroy(vps_handle h);

/*
 * vps_sizes -- problem sizes of the finest level: interior DoFs, number of
 * vertex patches (2^level - 1)^d, and device bytes held by the handle.
 * Any output pointer may be NULL.
 */
int vps_sizes(vps_handle h, int64_t* n_interior, int64_t* n_patches,
              size_t* device_bytes);

/* vps_level_layout -- n1 (nodes per direction), row pitch and total
 * elements of a level-layout vector of `level` (1..finest). */
int vps_level_layout(vps_handle h, int level, int64_t* n1, int64_t* row_pitch,
                     int64_t* total_elems);

/* vps_pack / vps_unpack -- compact <-> level layout of `level`, working
 * precision.  pack writes 0 to boundary and padding entries. */
int vps_pack(vps_handle h, int level, const void* compact, void* level_vec);
int vps_unpack(vps_handle h, int level, const void* level_vec, void* compact);

/*
 * vps_smooth -- n_steps smoothing steps S_l(x, b) on `level` (level layout,
 * working precision), in place on x.  Multiplicative: one step visits the
 * 2^d colours in increasing order; with the default kernel structure every
 * colour is one kernel that gathers each patch's closure, forms the local
 * residual r_j = R_j b - Abar_j Rbar_j x (Section 2.2) and adds
 * A_j^{-1} r_j by fast diagonalisation (Eq. 2.13/2.14) -- the fused kernel,
 * or (default variant) the Boundary kernel of Section 3.2, the same update
 * without reading the interior of x (vps_set_smooth_variant,
 * vps_set_smoother_kernel).  Additive: x += damping *
 * sum_j R_j^T A_j^{-1} R_j (b - A x).  Requires level >= 2 (level 1 holds a
 * single patch: use vps_vcycle).  b and x must not alias.
 */
int vps_smooth(vps_handle h, int level, const void* b, void* x, int n_steps);

/* vps_smooth_colour -- one multiplicative colour pass (0 <= colour < 2^d) on
 * `level` (>= 1), in place on x, with the handle's variant and kernel
 * structure.  Used to test and time single launches. */
int vps_smooth_colour(vps_handle h, int level, int colour, const void* b, void* x);

/* vps_apply -- y = A_level x (Eq. 2.3, matrix-free), working precision,
 * level layout.  x and y must not alias. */
int vps_apply(vps_handle h, int level, const void* x, void* y);

/* vps_restrict -- r_coarse = (I^up)^T r_fine from level `fine_level` to
 * fine_level-1 (Section 2.1: restriction is the transpose of prolongation). */
int vps_restrict(vps_handle h, int fine_level, const void* r_fine, void* r_coarse);

/* vps_prolongate_add -- x_fine += I^up x_coarse (interpolation of the coarse
 * finite element function at the fine support points, Section 2.1). */
int vps_prolongate_add(vps_handle h, int fine_level, const void* x_coarse, void* x_fine);

/*
 * vps_vcycle -- x = Vcycle_L(A_L, 0, b) on the finest level (Algorithm 1),
 * level layout, working precision.  n_pre / n_post smoothing steps per
 * level; the multiplicative post-smoother visits the colours in reverse
 * order so that the cycle is a symmetric preconditioner; the coarsest level
 * (vps_set_coarse_level) is solved exactly.
 */
int vps_vcycle(vps_handle h, const void* b, void* x);

/*
 * vps_solve -- CG on the finest level, preconditioned by one V-cycle per
 * iteration, x0 = 0 (beta in the flexible Polak-Ribiere form).  When the
 * recursive residual reaches rtol ||b||_2, the residual r = b - A x is
 * evaluated in FP64; the solve ends if ||r||_2 <= rtol ||b||_2, else CG
 * restarts from r.  Once a restart fails to halve ||r||, the solve ends:
 * with VPS_OK if ||r||_2 <= gamma || |A| |x| ||_2, gamma = (6k+6) 2^-53,
 * the rounding bound of the FP64 evaluation of r itself (rtol below what
 * FP64 can resolve: the terms of A x cancel by about k^2 h^-2 for smooth
 * solutions, so e.g. 2D meshes of 2^10 cells per direction cannot show
 * 1e-10; |A| is the operator with the absolute values of its 1D band
 * coefficients), with VPS_ENOCONV otherwise.
 * b, x: compact DOUBLE device vectors.  iters / rel_res (host pointers, may
 * be NULL) receive the iteration count and the final FP64 relative
 * residual ||r||/||b||.  The first iteration is issued from the host; on a
 * handle with CUDA graphs enabled (a stream was given, see vps_set_graphs)
 * the later iterations run on the device as one graph whose conditional
 * while-node repeats the iteration until r.r <= (rtol ||b||)^2, max_it or a
 * breakdown (no host round trip per iteration); without graphs the host
 * issues every iteration and synchronises once per iteration to read r.r.
 * The host synchronises again for each FP64 residual check.  Errors:
 * VPS_ENOCONV, VPS_EBREAKDOWN, ...
 */
int vps_solve(vps_handle h, const double* b, double* x, double rtol, int max_it,
              int* iters, double* rel_res);

/*
 * vps_gmres -- the paper's outer solver (Section 4): flexible GMRES on the
 * finest level, right-preconditioned by one V-cycle of Algorithm 1 as
 * printed (the same colour order before and after the coarse correction,
 * i.e. not symmetric), x0 = 0, restarted every `restart` (1..512) products
 * A z.  FP64 Krylov vectors; the V-cycle in the handle's precision and A
 * by the outer operator (vps_set_outer_operator).  Each cycle ends when
 * the least-squares residual reaches rtol ||b||; the residual is then
 * evaluated in FP64 and checked as in vps_solve (rtol, or the rounding
 * bound of its own evaluation), else the next cycle starts from it.
 *   b, x: compact DOUBLE device vectors; iters / rel_res (host, may be
 *   NULL): products A z and the final FP64 relative residual.  Allocates
 *   2 restart + 1 vectors of the finest level on first use.  Synchronises
 *   once per iteration.  Errors: VPS_EINVAL, VPS_ENOCONV, VPS_EBREAKDOWN.
 */
int vps_gmres(vps_handle h, const double* b, double* x, double rtol, int restart, int max_it,
              int* iters, double* rel_res);

/*
 * vps_solve_host -- as vps_solve, but b and x are HOST pointers (compact,
 * double).  Copies b to the device, solves, copies x back; synchronous.
 */
int vps_solve_host(vps_handle h, const double* b_host, double* x_host, double rtol,
                   int max_it, int* iters, double* rel_res);

/*
 * vps_assemble_rhs_sines -- load vector b_i = int f phi_i (Eq. 2.4) on the
 * finest level for f(x) = sum_m coef[m] prod_t sin(pi freq[m*dim+t] x_t)
 * (a frequency 0 stands for the constant 1 in that direction; negative
 * frequencies are rejected),
 * with (k+2)-point Gauss quadrature per cell and direction.  coef, freq:
 * HOST arrays of n_modes (n_modes*dim) entries; b: compact DOUBLE device
 * vector.
 */
int vps_assemble_rhs_sines(vps_handle h, int n_modes, const double* coef,
                           const int* freq, double* b);

/*
 * vps_fmg -- full multigrid (Algorithm 2) as a standalone solver on the
 * handle's hierarchy, for f(x) = sum_m coef[m] prod_t g(freq[m*dim+t], x_t)
 * with g(0, s) = 1 and g(f, s) = sin(pi f s): the load vector of f is
 * assembled on every level (as vps_assemble_rhs_sines); the coarsest level
 * (vps_set_coarse_level) is solved exactly; every finer level starts from
 * the prolongated coarser solution and takes one V-cycle; then V-cycles on
 * the finest level repeat until ||b - A x||_2 <= tol ||b||_2 (norms and
 * residuals in FP64; the V-cycle in the handle's precision, applied as the
 * correction x += V(0, b - A x), equal to V(x, b) since Algorithm 1 is
 * affine in x).  The V-cycle is the one Algorithm 1 prints: the same colour
 * order before and after the coarse correction.  If the residual stops
 * falling at the rounding bound of its own FP64 evaluation (see vps_solve),
 * the solve ends there with VPS_OK.
 *   x: compact DOUBLE device output; iters (host, may be NULL): V-cycles of
 *   the final loop (the count the paper's Tables 1 and 2 report); rel_res:
 *   the final ||b - A x|| / ||b||.  Synchronous.
 *   Errors: VPS_EINVAL, VPS_ENOCONV (not within max_it V-cycles), ...
 */
int vps_fmg(vps_handle h, int n_modes, const double* coef, const int* freq, double tol,
            int max_it, double* x, int* iters, double* rel_res);

/*
 * vps_l2_error_sine -- ||u_h - u||_{L2} for u = prod_t sin(pi x_t) and the
 * finite element function u_h with compact DOUBLE device coefficients x,
 * by (k+2)^d Gauss points per cell.  *err (host) receives the value.
 * Synchronous.
 */
int vps_l2_error_sine(vps_handle h, const double* x, double* err);

/*
 * vps_set_coarse_level -- choose the coarsest level of the V-cycle, solved
 * exactly (Algorithm 1's coarse grid solver).  On the uniform Cartesian mesh
 * the operator of a whole level is a Kronecker sum of 1D stiffness and mass
 * matrices (Eq. 2.11/2.12), so the exact solve is a global fast
 * diagonalisation (Eq. 2.13-2.15 with the level's 1D eigenpairs).
 * level: 1..finest (level 1 holds a single vertex patch; the finest level
 * makes the V-cycle an exact solver), or 0 for the default chosen at
 * creation: the finest level below the top with at most 32 interior nodes
 * per direction.  At most 255 interior nodes per direction.  Synchronises
 * the stream and allocates the level's tables.  Errors: VPS_EINVAL.
 */
int vps_set_coarse_level(vps_handle h, int level);
int vps_get_coarse_level(vps_handle h, int* level);

/*
 * vps_set_coarse_solver / vps_get_coarse_solver -- how the exact coarse
 * solve (the 2d passes of the global fast diagonalisation: S^T along each
 * direction, the last of them scaled by 1/(sum of eigenvalues), then S along
 * each) is launched; solver is a combination of
 *   VPS_COARSE_COOPERATIVE: one cooperative launch, every block resident,
 *     with a grid barrier between the passes (without: one kernel per pass,
 *     VPS_COARSE_PASSES).  Each barrier wait polls a bounded number of times
 *     (about a second at the least); an expiry is reported like a sweep's
 *     (VPS_ETIMEOUT, see vps_set_colour_schedule);
 *   VPS_COARSE_WIDE_TILES: thread blocks of 16 lines x 64 outputs (4 outputs
 *     per thread) instead of 16 x 32 (2 per thread, twice the blocks).
 * Every output is the same dot product in the same order in every form
 * (bit-identical results); chosen per coarse level by vps_autotune, the
 * default is VPS_COARSE_COOPERATIVE where the device supports cooperative
 * launches.  Errors: VPS_EINVAL (unknown value, or cooperative launches
 * unsupported).
 */
#define VPS_COARSE_PASSES      0
#define VPS_COARSE_COOPERATIVE 1
#define VPS_COARSE_WIDE_TILES  2
int vps_set_coarse_solver(vps_handle h, int solver);
int vps_get_coarse_solver(vps_handle h, int* solver);

/*
 * vps_autotune -- choose, by timed trials on this handle's own buffers, the
 * smoother variant of every level (patches per thread block, the tuning
 * axis of Section 3.1.2) together with the colour schedule
 * (vps_set_colour_schedule: for each schedule the fastest variant of every
 * level; then the schedule whose fastest steps on the levels above the
 * chosen coarsest level add up to the least time, the coarsest level being
 * timed once more if that changes the schedule), the operator tile
 * structure of every level (vps_set_operator_variant), and the coarsest
 * level (vps_set_coarse_level) that gives the fastest CG solve, each
 * candidate with its faster coarse solver form (vps_set_coarse_solver).  cache_path (may be NULL): a JSON file keyed by
 * (dim, degree, precision, smoother, level, smoothing steps) with the
 * smoother variant and operator tile structure of every level, the colour
 * schedule and the coarsest level; an entry found
 * there is applied without timing (*from_cache = 1), otherwise the result is
 * written to it.  Synchronous; runs solves on the handle's stream.
 */
int vps_autotune(vps_handle h, const char* cache_path, int* from_cache);

/* vps_set_smooth_variant / vps_get_smooth_variant -- the smoother kernel
 * variant of `level` (0: every level), and its patches per thread block.
 * Variant 3 * kind + shape, shape 0, 1, 2 the block shape: shape 0 has G1
 * groups of 1 patch per thread, shape 1 G1 groups of 2 patches per thread,
 * shape 2 G2 groups of 1 (G1, G2 per dimension and degree, chosen so that
 * the lines of every contraction stage nearly fill whole warps; the patches
 * per block are returned in *patches_per_block);
 *   kind 0 (variants 0-2): the fused kernel (Algorithm 3);
 *   kind 1 (3-5): the Boundary kernel of Section 3.2:
 *            x_I = A_j^-1 (b_I - A^IB x_B), which equals the fused update
 *            for the exact local solver without reading x_I
 *            (VPS_MULTIPLICATIVE handles only);
 *   kind 2 (6-8): the Boundary kernel in blocks of one warp, each stage in
 *            several rounds of 32 lines (degrees 1..3 only);
 *   kind 3 (9-11) / kind 4 (12-14): the fused / the Boundary kernel in
 *            blocks of the fewest warps that take every stage after the
 *            first in one round (the first, whose lines are the most, in
 *            two): fewer threads per block, so more resident blocks and
 *            patches per SM (VPS_MULTIPLICATIVE handles only; a shape whose
 *            automatic block is already that small has no kind 3 or 4);
 *   kind 5 (variant 15): the colour pass with one thread per patch, 256
 *            patches per block -- degree 1 as point Gauss-Seidel (a Q1 patch
 *            has one interior DoF); 2D degrees 2 and 3 (3: FP32 only) with
 *            the whole patch in registers (VPS_MULTIPLICATIVE handles only).
 * A variant whose shared memory exceeds the GPU's limit for the handle's
 * (dim, degree, precision) is unavailable.  Errors: VPS_EINVAL. */
int vps_set_smooth_variant(vps_handle h, int level, int variant);
int vps_get_smooth_variant(vps_handle h, int level, int* variant, int* patches_per_block);

/* vps_set_operator_variant / vps_get_operator_variant -- tile structure of
 * the level's operator A_l x (Section 2.3's Kronecker sum on the Cartesian
 * mesh) in the V-cycle's residuals: 0 the default; 1 the alternative where
 * one exists (*n_variants = 2: 3D FP32 handles of degree <= 4, whose default
 * takes the z contraction one cell of planes at a time; the alternative
 * takes it plane by plane).  Both compute the same operator.  Chosen per
 * level by vps_autotune.  Errors: VPS_EINVAL (level, unavailable variant). */
int vps_set_operator_variant(vps_handle h, int level, int variant);
int vps_get_operator_variant(vps_handle h, int level, int* variant, int* n_variants);

/* vps_set_colour_schedule / vps_get_colour_schedule -- how the colour
 * passes of a multiplicative smoothing step (Algorithm 3, colour by colour)
 * are scheduled on the GPU; chosen by vps_autotune:
 *   VPS_SCHEDULE_PLAIN: one ordinary launch per colour;
 *   VPS_SCHEDULE_PDL (default): one programmatic dependent launch per
 *     colour (a pass is scheduled while the previous one drains and waits
 *     for it before reading b or x);
 *   VPS_SCHEDULE_SWEEP: the whole step as one dataflow launch of one block
 *     per tile of every colour.  Blocks take tiles in the colours' order,
 *     and a tile starts once the patches of earlier colours that overlap
 *     its patches (vertices at most one apart in every direction) are done,
 *     so the passes overlap where the patches do not.  The result equals the
 *     colour-by-colour passes bit for bit.  Each dependency wait polls a
 *     flag a bounded number of times (about a second at the least); on
 *     expiry the sweep records it and finishes without waiting (its values
 *     are then undefined), and the next vps_solve (at its FP64 residual
 *     check), vps_gmres, vps_fmg or vps_check_waits returns VPS_ETIMEOUT.
 *     Fused kernel structure only (VPS_KERNEL_FUSED, smoother variants
 *     0-5); otherwise, and for vps_smooth_colour, the passes are launched
 *     as with VPS_SCHEDULE_PDL.
 * The same arithmetic in every schedule.  Errors: VPS_EINVAL. */
#define VPS_SCHEDULE_PLAIN 0
#define VPS_SCHEDULE_PDL   1
#define VPS_SCHEDULE_SWEEP 2
int vps_set_colour_schedule(vps_handle h, int schedule);
int vps_get_colour_schedule(vps_handle h, int* schedule);

/* vps_check_waits -- synchronises the handle's stream; VPS_ETIMEOUT if a
 * dependency wait of a VPS_SCHEDULE_SWEEP smoothing step or a grid barrier
 * of a VPS_COARSE_COOPERATIVE coarse solve of this handle expired since the
 * last check (the record is then cleared), else VPS_OK. */
int vps_check_waits(vps_handle h);

/* vps_skip_sweep_tiles -- fault injection for tests: the next dataflow
 * sweep on `level` starts taking tiles at index `tiles` (in the order of the
 * sweep), so the first `tiles` tiles are never run and the tiles that depend
 * on them wait until their poll limit (VPS_ETIMEOUT afterwards).  The sweep
 * after that one runs normally.  Synchronous.  Errors: VPS_EINVAL. */
int vps_skip_sweep_tiles(vps_handle h, int level, int64_t tiles);

/* vps_kernel_launches -- number of kernels the handle has launched since
 * creation (direct launches plus, for every replay of a captured graph, the
 * kernels the graph holds).  Instrumentation for benchmarks. */
int vps_kernel_launches(vps_handle h, int64_t* count);

/*
 * vps_set_outer_operator -- the operator the outer CG (Section 4.1, with
 * the FP64 outer iteration of Section 4.2) applies to its search direction:
 *   VPS_OUTER_FP64 (0): FP64 arithmetic (default for VPS_FP64 handles);
 *   VPS_OUTER_DOUBLE_FLOAT (1): the same sum-factorised operator evaluated
 *     in double-float arithmetic -- each value a pair of floats, products
 *     with FMA-exact rounding errors, sums by TwoSum -- about 48 significant
 *     bits at a fraction of the FP64 cost on this GPU (default for VPS_FP32
 *     handles).  Its rounding can let the recursive CG residual drift from
 *     the true one, so convergence is confirmed on r = b - A x evaluated in
 *     FP64, and CG restarts from that residual if it is still above rtol;
 *     *rel_res of vps_solve is then that FP64 residual.
 * The first switch to mode 1 allocates two float vectors of the finest
 * level.  Errors: VPS_EINVAL (unknown mode), VPS_ENOMEM.
 */
#define VPS_OUTER_FP64 0
#define VPS_OUTER_DOUBLE_FLOAT 1
int vps_set_outer_operator(vps_handle h, int mode);
int vps_get_outer_operator(vps_handle h, int* mode);

/*
 * vps_set_smoother_kernel / vps_get_smoother_kernel -- the kernel structure
 * of the multiplicative smoother's colour passes (Section 3.1, its table of
 * smoother versions), for comparisons; the smoothing itself is the same:
 *   VPS_KERNEL_FUSED (0, default): one kernel per colour (the smoother
 *     variants of vps_set_smooth_variant);
 *   VPS_KERNEL_SEPARATE (1): a local-residual kernel writes b_I - Abar_j x
 *     of every patch to the level's residual vector, a second kernel solves;
 *   VPS_KERNEL_GLOBAL (2): the residual of the whole level by the operator,
 *     then the local solve kernel;
 *   VPS_KERNEL_GLOBAL_INVERSE (3): as 2 with the local solve by the dense
 *     precomputed A_j^-1 instead of fast diagonalisation (the "inverse
 *     matrix" local solver; m^d <= 1024 rows, i.e. k <= 5 in 3D; built on
 *     the host in FP64 on first selection).
 * Kinds 1-3 take the block shape of the level's variant.  Errors:
 * VPS_EINVAL (unknown kind, additive handle, inverse too large). */
#define VPS_KERNEL_FUSED 0
#define VPS_KERNEL_SEPARATE 1
#define VPS_KERNEL_GLOBAL 2
#define VPS_KERNEL_GLOBAL_INVERSE 3
int vps_set_smoother_kernel(vps_handle h, int kind);
int vps_get_smoother_kernel(vps_handle h, int* kind);

/* vps_get_solve_info -- of the handle's last solve: the number of CG
 * restarts from the FP64 residual, and 1 if it ended at the rounding bound
 * of that residual rather than at rtol (see vps_solve).  Host outputs, may
 * be NULL. */
int vps_get_solve_info(vps_handle h, int* restarts, int* at_rounding_bound);

/*
 * vps_apply_outer -- y = A x on the finest level with the handle's outer
 * operator (vps_set_outer_operator): the product the CG forms with its
 * search direction.  x, y: distinct DOUBLE device vectors in the finest
 * level's layout, whatever the handle's precision; boundary entries of y
 * are written 0, padding entries are not written.  Uses the handle's split buffers in mode 1.
 * Asynchronous on the handle's stream.  Errors: VPS_EINVAL.
 */
int vps_apply_outer(vps_handle h, const double* x, double* y);

/* vps_set_graphs -- 1: capture the V-cycle in a CUDA graph on first use and
 * replay it (default on non-default streams); 0: launch kernels directly. */
int vps_set_graphs(vps_handle h, int enable);

/*
 * vps_smooth_additive_static -- one additive smoothing step on `level`
 * (2..), in place on x, WITHOUT a handle and without allocating memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc -- e.g. an application whose framework reserves
 * nearly all device memory for its own pool at start-up, a latency-bound
 * loop that cannot afford the synchronisation of cudaMalloc/cudaFree, or a
 * deployment with a fixed, audited device-memory budget.
 *   Computes x += damping * sum_j R_j^T A_j^{-1} R_j (b - A x), the step of
 *   vps_smooth on a VPS_ADDITIVE handle with the same damping.
 *   dim, degree, level, precision, damping: as for vps_create; b, x: device
 *   vectors in the level layout of `level` (float for VPS_FP32, double for
 *   VPS_FP64), caller-owned, distinct.  cuda_stream: the stream to run on.
 *   Scratch: the residual lives in a static device array of 32 MiB inside
 *   the library, and the tables of 1/(sum of eigenvalues) in a second static
 *   array of 66,048 bytes (one slot per dimension, degree and precision).
 *   A level whose residual needs more than 32 MiB (for example 3D Q4 on
 *   more than 2^5 cells per direction) is rejected with VPS_EINVAL and a
 *   message before any CUDA call; the size is computed in floating point,
 *   so levels whose element count would overflow an integer are rejected
 *   too.  Both arrays stay allocated on every GPU that loaded the library
 *   until the process exits.
 *   Set-up: the first call on a device (with that device current) looks up
 *   both arrays' device addresses; the first call of each (dim, degree,
 *   precision) on a device also uploads that degree's constant tables and
 *   fills its eigenvalue-table slot with synchronous copies.  Make those
 *   first calls before any stream capture begins.  Later calls of a shape
 *   issue kernels only, on cuda_stream.
 *   Every call shares the residual array and overwrites it (nothing in it
 *   has to start at zero): calls whose work overlaps on one GPU race, so
 *   issue them in one stream or order them.  Errors: VPS_EINVAL, VPS_ECUDA;
 *   message via vps_last_error(NULL).
 */
int vps_smooth_additive_static(int dim, int degree, int level, int precision, double damping,
                               const void* b, void* x, void* cuda_stream);

/*
 * Serving: continuous batching of Poisson solve requests (no counterpart in
 * the paper).  A server owns an engine thread on the device current at
 * creation.  Requests wait in a queue and are admitted as solver slots
 * (at most max_active at a time) and device memory (memory_budget bytes)
 * become free; a slot is a handle whose level hierarchy stays resident for
 * later requests of the same (dim, degree, level); idle slots are evicted
 * least recently used first.  Admitted requests of one (dim, degree) form a
 * cohort on one CUDA stream: each runs vps_solve's CG as an asynchronous
 * state machine, and whenever none of the cohort's work is in flight the
 * engine runs the V-cycles of all members that wait for one together --
 * the colour passes, restrictions and prolongations of all their levels as
 * persistent kernels that take tiles from a device-side queue, one launch
 * per smoothing colour or transfer step -- and then the rest of each
 * member's iteration.  Requests join their cohort between these steps;
 * cohorts run concurrently.  The engine thread never waits for the GPU or
 * for an allocation: hierarchies are built (and evicted ones destroyed) by
 * a provisioning thread, and results are copied into the callers' buffers
 * by a completion thread.  precision: VPS_FP32 (FP32 V-cycle, FP64 CG)
 * or VPS_FP64.  A request's result depends only on its own data: every
 * level of it goes through the operations of its own V-cycle in the same
 * order, so it is the same alone and in a mix.  Besides the budget, each
 * cohort holds 4 MiB of device memory (and 4 MiB of pinned host memory)
 * for its queues.
 */
typedef struct vps_server_ctx* vps_server;

#define VPS_REQ_QUEUED  0
#define VPS_REQ_RUNNING 1
#define VPS_REQ_DONE    2
#define VPS_REQ_FAILED  3

int vps_server_create(size_t memory_budget, int max_active, int precision, double rtol,
                      int max_it, vps_server* out);
/* Queue a solve of -Laplace u = f, f = sum_m coef[m] prod_t sin(pi freq[m*dim+t] x_t)
 * (load vector as vps_assemble_rhs_sines).  x_out: HOST buffer of (k 2^level - 1)^dim
 * doubles (compact layout) that receives the solution; it must stay valid
 * until the request is done.  coef/freq are copied.  *id receives the id. */
int vps_server_submit(vps_server s, int dim, int degree, int level, int n_modes,
                      const double* coef, const int* freq, double* x_out, int64_t* id);
/* State (VPS_REQ_*), solver status, CG iterations, relative residual, time
 * queued and time from submission to result (seconds; -1 if not yet). */
int vps_server_query(vps_server s, int64_t id, int* state, int* status, int* iters,
                     double* rel_res, double* queue_s, double* latency_s);
/* Wait (host side, at most timeout_s) for request id, or for all requests
 * submitted so far when id == 0.  VPS_ETIMEOUT if the time ran out. */
int vps_server_wait(vps_server s, int64_t id, double timeout_s);
int vps_server_stats(vps_server s, int64_t* submitted, int64_t* done, int* active, int* queued);
const char* vps_server_last_error(vps_server s);
/* vps_server_batch_stats -- batching counters since creation: cohort V-cycle
 * steps (ticks), batched launches, and the largest number of requests whose
 * tiles one batched launch processed (max_requests_per_launch) or one tick
 * served (max_requests_per_tick).  Host pointers, each may be NULL.
 * Errors: VPS_EINVAL (s NULL). */
int vps_server_batch_stats(vps_server s, int64_t* ticks, int64_t* batched_launches,
                           int* max_requests_per_launch, int* max_requests_per_tick);
/* vps_server_host_times -- host seconds spent since creation by the engine
 * thread in admission (seconds[0]), cohort V-cycle steps (seconds[1]) and
 * polling (seconds[2]), and by the helper threads in building and
 * destroying hierarchies (seconds[3]) and copying results into the callers'
 * buffers (seconds[4]).  seconds: host array of 5.  Errors: VPS_EINVAL. */
int vps_server_host_times(vps_server s, double* seconds);
/* Stops the engine thread (requests still running are abandoned) and frees
 * every slot. */
int vps_server_destroy(vps_server s);

/*
 * vps_fma_peak -- measured multiply-add throughput of the GPU's FP32 or FP64
 * pipe, the denominator of the smoother's fraction of arithmetic peak (the
 * paper quotes its kernels as a fraction of the CUDA-core peak, Section 4.3).
 * Not part of the method.  Runs a kernel of independent multiply-add chains
 * on every SM (8 blocks of 256 threads per SM) twice after one warm-up
 * launch on cuda_stream, timed with CUDA events; synchronises the stream.
 * precision: VPS_FP32 or VPS_FP64.  flops_per_s (host, required) receives
 * 2 x multiply-adds / seconds of the faster timed launch; seconds and
 * sm_count (host, may be NULL) its duration and the device's multiprocessor
 * count.  Allocates nothing.  Errors: VPS_EINVAL, VPS_ECUDA.
 */
int vps_fma_peak(int precision, double* flops_per_s, double* seconds, int* sm_count,
                 void* cuda_stream);

/* vps_last_error -- message of the last failure on h (h = NULL: the last
 * failure of vps_create or vps_smooth_additive_static on this thread).
 * Valid until the next call. */
const char* vps_last_error(vps_handle h);

/* vps_status_string -- name of a status code. */
const char* vps_status_string(int status);

/*
 * vps_check_fp_conversions -- diagnostic of the library's own conversions
 * between float and double, which the vector kernels of the mixed-precision
 * CG use instead of the hardware conversions (those are FP64 instructions,
 * which issue at about 1/64 of the FP32 rate on this GPU).  For each of the
 * n 64-bit patterns in the DEVICE array `patterns` (caller-owned, read only;
 * may be NULL when n is 0):
 *   mismatches[0] counts patterns whose low 32 bits, as a float, convert to
 *     a double that differs from the cast (float -> double, exact);
 *   mismatches[1] counts patterns that, as a double, round to a float that
 *     differs from the cast (round to nearest, ties to even; NaNs compare
 *     equal);
 *   mismatches[2] counts patterns whose double-float split hi + lo breaks
 *     its contract: hi = the value truncated to 24 bits, lo = the next bits
 *     truncated, both of the value's sign, remainder below 2^-47 of the
 *     value, for binary64 exponents in [-73, 127]; zeros give signed zeros;
 *     outside that range hi = fl(v), lo = fl(v - hi).
 * Runs on cuda_stream and synchronises it; allocates 24 bytes from the
 * stream-ordered pool.  Errors: VPS_EINVAL, VPS_ECUDA (message via
 * vps_last_error(NULL)).
 */
int vps_check_fp_conversions(const void* patterns, int64_t n, int64_t* mismatches,
                             void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* VPS_H */
