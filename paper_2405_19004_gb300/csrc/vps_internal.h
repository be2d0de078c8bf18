// Internal declarations shared by the translation units of libvps.
//
// Host-side 1D tables (computed once per degree in setup.cpp, FP64), the
// geometry of a level vector, and the per-(dim, degree) kernel entry points
// that every instantiation unit (kernels_dk.cu compiled with VPS_DIM and
// VPS_K) registers at load time.
#pragma once

#include <cstddef>
#include <cstdint>
#include <utility>
#include <vector>
#include <cuda_runtime.h>

struct vps_context;

namespace vps {

constexpr int kMaxK = 7;

// 1D tables of Q_k in reference units (cell size 1), FP64.
//  Ap, Mp : interior rows (1..2k-1) of the stiffness / mass matrices of the
//           two-cell patch closure (2k+1 nodes), row-major m x n
//           (Section 2.4: the patch operator is a Kronecker sum of these).
//  S, lam : generalised eigenpairs of the interior blocks,
//           A_I S = M_I S diag(lam), S^T M_I S = I (Eq. 2.15); S row-major,
//           column j = eigenvector j.
//  Kb, Mb : rows of the global 1D stiffness / mass matrices as bands:
//           node o with q = o mod k couples to o-k+j, j = 0..2k, coefficient
//           Kb[q*(2k+1)+j]  (Section 2.3, Cartesian cells).
//  P1     : interpolation of the k+1 coarse basis functions of one coarse
//           cell at its 2k+1 fine support points, row-major (2k+1) x (k+1)
//           (Section 2.1).
struct HostTables {
  int k = 0;
  int n = 0, m = 0;
  double z[kMaxK + 1];                       // GLL nodes on [0,1]
  double Khat[(kMaxK + 1) * (kMaxK + 1)];    // reference element stiffness
  double Mhat[(kMaxK + 1) * (kMaxK + 1)];    // reference element mass
  double Ap[(2 * kMaxK - 1) * (2 * kMaxK + 1)];
  double Mp[(2 * kMaxK - 1) * (2 * kMaxK + 1)];
  double S[(2 * kMaxK - 1) * (2 * kMaxK - 1)];
  double lam[2 * kMaxK - 1];
  double Kb[kMaxK * (2 * kMaxK + 1)];
  double Mb[kMaxK * (2 * kMaxK + 1)];
  double P1[(2 * kMaxK + 1) * (kMaxK + 1)];
};

// Computes every table for degree k (1..kMaxK). Returns false on failure.
bool build_tables(int k, HostTables* t, char* err, size_t errlen);

// Generalised eigenpairs of the global interior 1D stiffness and mass
// matrices of a whole level (reference cell size 1): K S = M S diag(lam),
// S^T M S = I, S row-major ni x ni (ni = k 2^level - 1 <= kMaxGlobalFd).
// The level operator is a Kronecker sum of these (Eq. 2.11/2.12 for the
// whole mesh), so the same fast diagonalisation inverts it exactly.
constexpr int kMaxGlobalFd = 255;
bool build_global_fd(int k, int level, std::vector<double>* S, std::vector<double>* lam,
                     char* err, size_t errlen);

// Gauss-Legendre rule on [0,1] with q points (q <= 16).
void gauss_rule(int q, double* x, double* w);

// Lagrange basis of the GLL nodes z (k+1 of them) at point x.
void lagrange_eval(int k, const double* z, double x, double* val);

// Geometry of one level vector.
struct LevelGeom {
  int dim = 0, k = 0, level = 0;
  int n1 = 0;          // nodes per direction incl. boundary
  int ncell = 0;       // cells per direction
  int64_t px = 0;      // row pitch (elements)
  int64_t pz = 0;      // plane pitch (elements), 3D; = px * n1
  int64_t total = 0;   // elements in the buffer
  double h = 0.0;
};

// Elements of a level vector (pitched rows, boundary included), computed in
// floating point: finite and exact for every valid (dim, k, level), HUGE_VAL
// for invalid arguments, and never wrapped, so comparing it with a limit
// rejects levels whose size does not fit in 64-bit integers.
double level_elements(int dim, int k, int level);
// Largest level vector the library addresses (every index fits in int64 and
// the products in make_geom cannot overflow).
constexpr double kMaxLevelElements = 4.0e18;

// Geometry of a level.  A level with more than kMaxLevelElements elements
// gets total = INT64_MAX and no other field set: callers reject it.
LevelGeom make_geom(int dim, int k, int level);

// Patches of one colour on one level.
struct ColourGeom {
  int cnt[3] = {1, 1, 1};     // patches per direction
  int par[3] = {0, 0, 0};     // vertex parity per direction
  int64_t npatch = 0;
};

ColourGeom make_colour(const LevelGeom& g, int colour);

// Number of kernels this thread has launched through the library (every
// launch site increments it); used to report launches per call.
int64_t& launch_counter();
#define VPS_COUNT_LAUNCH() (++::vps::launch_counter())

// Programmatic dependent launch: the kernel may be scheduled while the
// previous kernel of the stream drains (its blocks occupy free SM slots and
// run their prologue), and waits with griddepcontrol.wait
// (grid_dependency_wait in kernels_dk.cu) before it reads anything an
// earlier kernel writes.  Only kernels that execute that wait before such
// reads may be launched this way.  The relaxed dependency applies only to a
// previous kernel that requests it (launch_dependents); after a copy or a
// memset the launch is ordered as usual.  Stream capture records the
// dependency as a programmatic graph edge.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Batched launches (serving): one persistent kernel processes the tiles of
// several levels -- of different requests -- taken from a queue in device
// memory.  Item i owns tiles [tile0, next item's tile0); a block takes the
// next tile with one atomic increment of `head` until head >= ntiles.  The
// host fills a queue (head = 0) and copies it to the device before the
// launch, in the launch's stream.
constexpr int kMaxBatch = 32;   // items per queue
struct BatchItem {
  const void* in = nullptr;     // smoother: b; restriction: fine residual; prolongation: coarse x
  void* out = nullptr;          // smoother: x; restriction: coarse b;      prolongation: fine x
  int64_t tile0 = 0;            // first tile of the item in the launch's tile space
  int n1a = 0, n1b = 0;         // nodes per direction: a = the item's level (smoother) or the
  int64_t pxa = 0, pza = 0;     //   coarse level (transfers); b = the fine level (transfers)
  int64_t pxb = 0, pzb = 0;
  ColourGeom cg;                // smoother: the colour's patches
  double bscale = 1.0;          // smoother: scale of b (1/h in 3D)
  int tiles_per_dim = 0;        // transfers: tiles per direction (t^dim tiles)
};
struct BatchQueue {
  unsigned long long head;      // next tile (0 when uploaded)
  int64_t ntiles;
  int nitems;
  int pad_;
  BatchItem items[kMaxBatch];
};

// Dataflow schedule of a multiplicative smoothing step: one launch of one
// block per tile runs every colour.  Blocks claim tiles in the order of the sweep
// (all tiles of the first colour, then of the second, ...), and a tile
// starts once every patch of an earlier colour that overlaps one of its
// patches is done; the result equals the colour-by-colour passes bit for
// bit.  Per level, in device memory, zero-initialised:
struct SweepCounters {
  unsigned long long head;      // next tile of the running sweep (0 between sweeps)
  unsigned int done;            // blocks of the running sweep that have finished
  unsigned int epoch;           // sweeps completed on the level
};
// flags: one per patch of the level, colour by colour (colour c from
// flag_off[c], in the colour's patch order); a patch's flag holds the epoch
// of the sweep that finished it last.
struct SweepGeom {
  ColourGeom cg[8];             // colour geometry by position in the sweep order
  int colour[8] = {};           // colour at each position
  int pos_of[8] = {};           // position of each colour
  int64_t flag_off[8] = {};     // first flag of each colour
  int64_t tile_end[8] = {};     // tiles of positions 0..s together
  int ncol = 0;                 // 2^dim
  int ncell = 0;                // cells per direction
  unsigned int* flags = nullptr;
  SweepCounters* ctr = nullptr;
  int* err = nullptr;           // set to 1 by a wait that reached its poll limit
  unsigned int spin_limit = 0;  // polls of one flag before the wait gives up
};

// Smoother kernel variants the autotuner chooses from: v = 3 * kind + q,
// q = 0, 1, 2 the block shape (q = 0: G1 patch groups of 1 patch per thread,
// q = 1: G1 groups of 2, q = 2: G2 groups of 1, with G1 and G2 per (dim,
// degree) so that the stages' lines fill whole warps; kind 0 the fused kernel,
// kind 1 the Boundary kernel (x_I = A_j^-1 (b_I - A^IB x_B), Section 3.2),
// kind 2 the Boundary kernel in one-warp blocks, kinds 3 and 4 the fused and
// the Boundary kernel in blocks of the fewest warps that run every stage
// after the first in one round, kind 5 (variant 15) the colour pass with
// one thread per patch (degree 1: point Gauss-Seidel; 2D degrees 2, 3: the
// patch in registers).  Kinds 1 to 5
// serve the multiplicative smoother only (smooth_add_v[3..17] stay null).
constexpr int kQVariants = 3;
constexpr int kSmoothKinds = 6;
constexpr int kSmoothVariants = kSmoothKinds * kQVariants;
constexpr int v0_kind(int kind) { return kind * kQVariants; }

template <typename T>
struct KernelFns {
  using SmoothMultFn = cudaError_t (*)(const LevelGeom&, const ColourGeom&, const T* b, T* x,
                                       const T* inv_lam, cudaStream_t);
  using SmoothAddFn = cudaError_t (*)(const LevelGeom&, const ColourGeom&, const T* r, T* x,
                                      const T* inv_lam, T scale, cudaStream_t);
  // one multiplicative colour pass: x += R^T A_j^-1 (R b - Abar Rbar x)
  SmoothMultFn smooth_mult_v[kSmoothVariants] = {};
  // one additive colour pass from a precomputed residual: x += scale R^T A_ref^-1 R r
  SmoothAddFn smooth_add = nullptr;              // default variant (allocation-free entry point)
  SmoothAddFn smooth_add_v[kSmoothVariants] = {};
  int variant_p[kSmoothVariants] = {};           // patches per block of each variant
  // ablation kernels of Section 3.1: the local residual of every patch of a
  // colour written to r (Separate; the three block shapes), and the
  // local solve with the dense inverse (AinvT: A_j^-1 transposed, m^d x m^d)
  cudaError_t (*resid_v[kQVariants])(const LevelGeom&, const ColourGeom&, const T* b,
                                     const T* x, T* r, cudaStream_t) = {};
  cudaError_t (*inverse_solve)(const LevelGeom&, const ColourGeom&, const T* r, T* x,
                               const T* AinvT, cudaStream_t) = nullptr;
  // y = A x  (b == nullptr)  or  y = b - A x  (residual)
  cudaError_t (*apply)(const LevelGeom&, const T* x, const T* b, T* y, cudaStream_t) = nullptr;
  // the same operator with the other tile structure where two exist (3D
  // FP32, k <= 4: per-plane tiles instead of the cell-batched z windows of
  // `apply`); nullptr elsewhere
  cudaError_t (*apply_alt)(const LevelGeom&, const T* x, const T* b, T* y, cudaStream_t) = nullptr;
  // colour passes launched without programmatic dependent launch
  SmoothMultFn smooth_mult_plain_v[kSmoothVariants] = {};
  // a whole multiplicative smoothing step (every colour, in the order of
  // the SweepGeom) as one persistent dataflow kernel; null for the
  // one-warp variants
  cudaError_t (*smooth_sweep_v[kSmoothVariants])(const LevelGeom&, const SweepGeom&, const T* b,
                                                 T* x, const T* inv_lam, cudaStream_t) = {};
  // batched persistent launches over a device-side queue (q: device copy,
  // ntiles: its tile count, known on the host): multiplicative colour
  // passes (variant v), restrictions, prolongations, and the zeroing of the
  // upper faces of every item's `out` vector (nitems items)
  cudaError_t (*smooth_mult_batch_v[kSmoothVariants])(BatchQueue* q, int64_t ntiles,
                                                      const T* inv_lam, cudaStream_t) = {};
  cudaError_t (*restrict_batch)(BatchQueue* q, int64_t ntiles, cudaStream_t) = nullptr;
  cudaError_t (*prolong_batch)(BatchQueue* q, int64_t ntiles, cudaStream_t) = nullptr;
  cudaError_t (*zero_faces_batch)(const BatchQueue* q, int nitems, cudaStream_t) = nullptr;
  // tiles of one colour pass (patches per block) and of one transfer
  // (coarse cells per tile and direction)
  int transfer_cells = 0;
  // x_fine += P x_coarse
  cudaError_t (*prolong_add)(const LevelGeom& fine, const LevelGeom& coarse, const T* xc, T* xf,
                             cudaStream_t) = nullptr;
  // r_coarse = P^T r_fine
  cudaError_t (*restrict_)(const LevelGeom& fine, const LevelGeom& coarse, const T* rf, T* rc,
                           cudaStream_t) = nullptr;
};

struct KernelSet {
  bool present = false;
  // copies the degree's tables into this unit's constant memory on the
  // current device (synchronous)
  cudaError_t (*upload)(const HostTables&) = nullptr;
  KernelFns<float> f;
  KernelFns<double> d;
  // y = A x with x given as FP32 pairs (hi, lo) and double-float arithmetic
  cudaError_t (*apply_df)(const LevelGeom&, const float* xh, const float* xl, double* y,
                          cudaStream_t) = nullptr;
  // y = |A| |x| (absolute band coefficients), FP64: rounding scale of A x
  cudaError_t (*apply_abs)(const LevelGeom&, const double* x, double* y, cudaStream_t) = nullptr;
};

// Registry indexed [dim-2][k-1]; filled by ensure_registered().
KernelSet* kernel_registry(int dim, int k);
void ensure_registered();
void set_thread_error(const char* msg);

// --- generic vector kernels (ops.cu) ------------------------------------
template <typename T>
cudaError_t launch_pack(const LevelGeom& g, const T* compact, T* lev, cudaStream_t s);
template <typename T>
cudaError_t launch_unpack(const LevelGeom& g, const T* lev, T* compact, cudaStream_t s);

// Deterministic dot products over a whole level buffer: partial sums per
// block into `partial` (kDotBlocks doubles per product), then one block
// reduces them in a fixed order into out[0..nprod).
constexpr int kDotBlocks = 608;  // 4 x 152 SMs
cudaError_t launch_dot1(const double* a, const double* b, int64_t n, double* partial,
                        double* out, cudaStream_t s);

// CG scalar updates (all scalars live in device memory, see api.cu).
struct CgScalars {
  double rz;      // r_i . z_i
  double pAp;     // p . A p
  double alpha;
  double rr;      // r . r after the update
  double rzn;     // r_{i+1} . z_{i+1}
  double rzo;     // r_{i+1} . z_i
  double beta;
  int flag;       // 1: breakdown detected on the device
  // device-side iteration loop (a CUDA graph with a conditional node):
  int it;         // iterations done
  int max_it;
  double nb;      // ||b||
  double rtol;
};
// Ends the body of the device-side CG loop: ++it, and clears the loop's
// condition once r.r has reached (rtol ||b||)^2, it == max_it, or the
// breakdown flag is set.
cudaError_t launch_cg_loop_check(cudaGraphConditionalHandle cond, CgScalars* sc, cudaStream_t s);
cudaError_t launch_cg_loop_init(CgScalars* sc, int it, int max_it, double nb, double rtol,
                                cudaStream_t s);
// CG steps (deterministic reductions; partial, partial2: 2 * kDotBlocks doubles each):
//  start : p = z_old = z_new (+ split into ph, pl when given), rzn = r . z_new
//  next_p: beta = (r.z_new - r.z_old) / rz, p = z_new + beta p, z_old = z_new
//  step_xr: alpha = rzn / p.Ap, x += alpha p, r -= alpha Ap, rr = r . r, rz = rzn
// z_new in FP32 (the FP32 V-cycle's output) or FP64.
template <typename TZ>
cudaError_t launch_cg_start(double* p, double* z, const TZ* zn, const double* r, int64_t n,
                            double* partial, CgScalars* sc, cudaStream_t s, float* ph = nullptr,
                            float* pl = nullptr);
template <typename TZ>
cudaError_t launch_cg_next_p(double* p, double* z, const TZ* zn, const double* r, int64_t n,
                             double* partial, CgScalars* sc, cudaStream_t s, float* ph = nullptr,
                             float* pl = nullptr);
cudaError_t launch_cg_step_xr(double* x, double* r, const double* p, const double* Ap, int64_t n,
                              double* partial, double* partial2, CgScalars* sc, cudaStream_t s);
cudaError_t launch_cast_d2f(const double* a, float* b, int64_t n, cudaStream_t s);
// GMRES block operations: out[i] = V_i . w (i < nv; partial: nv * kDotBlocks
// doubles), w += sign * sum_i c[i] V_i (c on the device), y = a x.
cudaError_t launch_multi_dot(const double* V, int64_t ld, int nv, const double* w, int64_t n,
                             double* partial, double* out, cudaStream_t s);
cudaError_t launch_multi_axpy(double* w, const double* V, int64_t ld, int nv, const double* c,
                              double sign, int64_t n, cudaStream_t s);
cudaError_t launch_scale(double* y, const double* x, double a, int64_t n, cudaStream_t s);
// ph = fl32(a), pl = fl32(a - ph)
cudaError_t launch_split_df(const double* a, float* ph, float* pl, int64_t n, cudaStream_t s);
cudaError_t launch_cast_f2d(const float* a, double* b, int64_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_axpy_inplace(T* y, const T* x, T a, int64_t n, cudaStream_t s);

// One pass of the global fast diagonalisation of a level (runtime ni):
// out[L][o] = sum_c W[c*ni + o] in[c][L], MODE 1 then times inv[L*ni+o]
// (W = S applies S^T to each line; W = S^T stored row-major applies S).
// in_lev / out_lev: read / write the interior of a level-layout vector
// instead of a compact tensor.
// Row length of the global fast diagonalisation's work tensors and weight
// matrices: n rounded up to a multiple of 4 elements, so that rows start on
// 16-byte boundaries (the padding holds zeros).
__host__ __device__ inline int fd_pad(int n) { return (n + 3) & ~3; }

// Grid-wide barrier state of a cooperative launch (device words, zero at
// rest) and its bounded wait.
struct GridSync {
  unsigned int* count = nullptr;  // blocks arrived at the current barrier
  unsigned int* gen = nullptr;    // barriers completed
  int* err = nullptr;             // set to 1 by a wait that reached its poll limit
  unsigned int limit = 0;         // polls before a wait gives up
};
// The whole exact coarse solve (the passes of launch_fd_global_pass) in one
// cooperative launch with grid barriers between the passes; x of total
// elements xtotal is zeroed outside the interior.
template <typename T>
cudaError_t launch_fd_global_solve(const T* b, T* x, const T* S, const T* St, const T* inv, T* t1,
                                   T* t2, int ni, int dim, int px, int pz, int64_t xtotal,
                                   const GridSync& gs, bool wide, cudaStream_t s);

// One pass (mode 0: S^T, 1: S^T scaled by inv, 2: S) of the global fast
// diagonalisation, W with rows of fd_pad(ni), work tensors with rows of
// fd_pad(ni^(d-1)); in_lev / out_lev: the input / output in the level layout;
// wide: tiles of 64 outputs instead of 32.
template <typename T>
cudaError_t launch_fd_global_pass(int mode, const T* in, T* out, const T* W, const T* inv, int ni,
                                  int dim, bool in_lev, bool out_lev, int px, int pz, bool wide,
                                  cudaStream_t s);

// b (compact, double) = sum_m coef_m prod_t b1d[m][t][node_t]  with b1d on device
cudaError_t launch_rhs_tensor(const LevelGeom& g, int n_modes, const double* b1d, double* b,
                              cudaStream_t s);
// per-cell squared L2 error contributions of u_h - prod sin(pi x) -> partial sums
cudaError_t launch_l2_error_sine(const LevelGeom& g, const double* xlev, const double* tab,
                                 int q, double* partial, double* out, cudaStream_t s);

// Serving support (api.cpp): a handle on a stream of its own, a device-memory
// estimate for admission, and a CG solve advanced without blocking.
int create_own_stream(int dim, int degree, int level, int precision, vps_context** out);
size_t estimate_device_bytes(int dim, int degree, int level, int precision);
int cg_async_begin(vps_context* h, int n_modes, const double* coef, const int* freq, double rtol,
                   int max_it);
int cg_async_poll(vps_context* h, int* done, int* status, int* iters, double* rel,
                  const double** x_host);
const char* handle_error(vps_context* h);
// Asynchronous CG with external V-cycles (serving cohorts): while
// cg_async_pending_vcycle(h), the caller runs the V-cycle of h (for several
// handles at once with cohort_vcycle) and then calls cg_async_resume(h).
void set_external_vcycle(vps_context* h, bool on);
int cg_async_prepare(vps_context* h, int max_modes);
int cg_async_pending_vcycle(vps_context* h);
int cg_async_resume(vps_context* h);
// One V-cycle (Algorithm 1, symmetric colour order, x = 0) for each of n
// handles with a pending V-cycle that share dimension, degree, precision,
// smoothing steps and stream: level by level from each handle's top
// (levels aligned by their distance from the top), the colour passes,
// restrictions and prolongations of all handles in one persistent batched
// launch each (queues staged in q_host, pinned, copied to q_dev, both
// q_cap bytes; neither may be reused before the stream has passed this
// cycle), the residuals, memsets and coarse solves per handle.  Each
// handle's levels go through exactly the operations, in the order, of its
// own V-cycle, so its result equals that of the handle alone.
// batched_launches / max_items accumulate the launches and the largest
// number of levels in one launch.
int cohort_vcycle(vps_context* const* hs, int n, void* q_host, void* q_dev, size_t q_cap,
                  int64_t* batched_launches, int* max_items);

}  // namespace vps
