// C ABI of libvps: handle lifecycle, the V-cycle driver (Algorithm 1), the
// preconditioned CG driver and the helpers declared in include/vps.h.
//
// Everything numerical runs in the kernels of kernels_dk.cu and ops.cu; this
// file only validates arguments, owns device memory, sequences launches on
// the handle's stream and, on non-default streams, captures the V-cycle
// into a CUDA graph that is replayed on every later call.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "vps.h"
#include "vps_internal.h"

namespace vps {
void register_kernels_d2_k1(KernelSet*);
void register_kernels_d2_k2(KernelSet*);
void register_kernels_d2_k3(KernelSet*);
void register_kernels_d2_k4(KernelSet*);
void register_kernels_d2_k5(KernelSet*);
void register_kernels_d2_k6(KernelSet*);
void register_kernels_d2_k7(KernelSet*);
void register_kernels_d3_k1(KernelSet*);
void register_kernels_d3_k2(KernelSet*);
void register_kernels_d3_k3(KernelSet*);
void register_kernels_d3_k4(KernelSet*);
void register_kernels_d3_k5(KernelSet*);
void register_kernels_d3_k6(KernelSet*);
void register_kernels_d3_k7(KernelSet*);
}  // namespace vps

using namespace vps;

namespace {

constexpr int kMaxLevels = 24;
constexpr int kMaxDevices = 64;

std::mutex g_mutex;
bool g_registered = false;
bool g_uploaded[kMaxDevices][2][kMaxK];
thread_local std::string g_create_error;

void register_all() {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_registered) return;
  register_kernels_d2_k1(kernel_registry(2, 1));
  register_kernels_d2_k2(kernel_registry(2, 2));
  register_kernels_d2_k3(kernel_registry(2, 3));
  register_kernels_d2_k4(kernel_registry(2, 4));
  register_kernels_d2_k5(kernel_registry(2, 5));
  register_kernels_d2_k6(kernel_registry(2, 6));
  register_kernels_d2_k7(kernel_registry(2, 7));
  register_kernels_d3_k1(kernel_registry(3, 1));
  register_kernels_d3_k2(kernel_registry(3, 2));
  register_kernels_d3_k3(kernel_registry(3, 3));
  register_kernels_d3_k4(kernel_registry(3, 4));
  register_kernels_d3_k5(kernel_registry(3, 5));
  register_kernels_d3_k6(kernel_registry(3, 6));
  register_kernels_d3_k7(kernel_registry(3, 7));
  g_registered = true;
}

}  // namespace

namespace vps {
// Fills the kernel registry (idempotent); used by entry points without a handle.
void ensure_registered() { register_all(); }
// Sets the message vps_last_error(NULL) returns on this thread.
void set_thread_error(const char* msg) { g_create_error = msg ? msg : ""; }
}  // namespace vps

struct vps_context {
  int dim = 0, k = 0, L = 0, prec = 0, smoother = 0;
  double damping = 1.0;
  int n_pre = 1, n_post = 1;
  cudaStream_t stream = nullptr;
  int device = 0;
  bool use_graphs = false;
  std::string err;
  HostTables tab;
  KernelSet* ks = nullptr;
  LevelGeom geom[kMaxLevels + 1];
  size_t esz = 8;                       // bytes per working-precision element
  void* bv[kMaxLevels + 1] = {};        // per-level right-hand sides (working precision)
  void* xv[kMaxLevels + 1] = {};        // per-level iterates
  void* rv[kMaxLevels + 1] = {};        // per-level residuals
  void* inv_lam = nullptr;              // 1/(sum of eigenvalues), working precision, m^d
  // CG state, FP64, finest level layout
  double *cb = nullptr, *cx = nullptr, *cr = nullptr, *cp = nullptr, *cz = nullptr,
         *czn = nullptr, *cAp = nullptr;
  // outer operator of the CG: native FP64, or double-float (p split into
  // two float vectors cph + cpl) with a final FP64 check of the residual
  int outer = VPS_OUTER_FP64;
  float *cph = nullptr, *cpl = nullptr;
  // GMRES: Krylov basis V (m + 1 vectors) and preconditioned vectors Z (m),
  // leading dimension gm_ld; Hessenberg column buffers on device and host
  int gm_m = 0;
  int64_t gm_ld = 0;
  double *gmV = nullptr, *gmZ = nullptr, *gm_partial = nullptr, *gm_dev = nullptr;
  double* gm_host = nullptr;            // pinned
  // full multigrid: FP64 right-hand side, iterate and residual of the levels
  // below the finest (the finest uses cb, cx, cr)
  double* fmg_b[kMaxLevels + 1] = {};
  double* fmg_x[kMaxLevels + 1] = {};
  double* fmg_r[kMaxLevels + 1] = {};
  // last solve: restarts from the FP64 residual, and whether it stopped at
  // the rounding level of the residual's own evaluation instead of rtol
  int last_restarts = 0, last_at_floor = 0;
  double* partial = nullptr;            // 2 * kDotBlocks
  double* partial2 = nullptr;           // 2 * kDotBlocks (a second set for fused CG steps)
  double* dots = nullptr;               // scratch scalars for norms
  CgScalars* sc = nullptr;
  CgScalars* host_sc = nullptr;         // pinned
  double* host_dots = nullptr;          // pinned
  double* comp_b = nullptr;             // compact FP64 staging for vps_solve_host
  double* comp_x = nullptr;
  double* rhs_buf = nullptr;            // 1D load vectors for vps_assemble_rhs_sines
  size_t rhs_cap = 0;
  double* rhs_host = nullptr;           // pinned staging of rhs_buf
  size_t rhs_host_cap = 0;
  cudaEvent_t rhs_ev = nullptr;         // after the last copy out of rhs_host
  double* l2_tab = nullptr;             // basis table for the L2 error
  size_t bytes = 0;
  std::vector<void*> allocs;
  // captured V-cycle graphs (input r = cr; output czn, or xv[L] for the
  // symmetric FP32 cycle of the CG)
  cudaGraphExec_t prec_graph = nullptr;
  cudaGraphExec_t prec_graph_ns = nullptr;  // the non-symmetric cycle (GMRES)
  // CG iterations on the device: a while-node whose body is one iteration
  cudaGraphExec_t cg_loop_graph = nullptr;
  int64_t cg_loop_kernels = 0;          // kernels per loop iteration
  bool cg_loop_off = false;             // the loop graph could not be built here
  int64_t graph_kernels_ns = 0;
  bool own_stream = false;              // stream created (and destroyed) by the library
  int64_t graph_kernels = 0;            // kernel nodes in prec_graph
  int64_t kernels = 0;                  // kernels launched by this handle
  int smooth_var[kMaxLevels + 1] = {};  // smoother variant per level (index into the table)
  int op_var[kMaxLevels + 1] = {};      // operator tile structure per level (1: apply_alt)
  // colour schedule of the multiplicative smoothing step: ordinary launches
  // of the colour passes, programmatic dependent launches, or one dataflow
  // sweep kernel per step (VPS_SCHEDULE_*)
  int schedule = VPS_SCHEDULE_PDL;
  // dataflow sweeps: per level one flag per patch and the sweep counters;
  // the wait-expiry word of every sweep of the handle, and whether a sweep
  // ran since it was last read
  unsigned int* sweep_flags[kMaxLevels + 1] = {};
  SweepCounters* sweep_ctr = nullptr;   // kMaxLevels + 1
  int* wait_err = nullptr;
  bool waits_ran = false;
  // exact coarse solve as one cooperative launch (grid barriers between its
  // passes; barrier words in gsync) or as one launch per pass
  bool coarse_coop = false;
  bool coarse_wide = false;             // tiles of 64 outputs instead of 32
  bool coop_ok = false;                 // the device supports cooperative launches
  unsigned int* gsync = nullptr;        // count, generation
  unsigned int spin_limit = 1u << 21;   // polls of one flag (at least 128 ns each)
  int* host_err = nullptr;              // pinned copy of *wait_err
  // kernel structure of the multiplicative smoother (Section 3.1's
  // Fused / Separate / Global, and Global with the dense inverse)
  int kernel_kind = VPS_KERNEL_FUSED;
  void* ainv = nullptr;                 // A_j^-1 (symmetric, m^d x m^d), working precision
  // asynchronous CG (used by the serving loop)
  int as_phase = 0;                     // 0 idle, 1 iteration in flight, 2 result copy in flight
  // the V-cycles of the asynchronous CG are run by the caller (cohort_vcycle,
  // batched with other handles) instead of by the handle itself: the CG then
  // stops before each V-cycle with as_need = 3 (first iteration), 1 (restart
  // from the FP64 residual) or 2 (next iteration), and cg_async_resume issues
  // the rest of the iteration once the caller has run the V-cycle
  bool as_external = false;
  int as_need = 0;
  int as_it = 0, as_maxit = 0, as_status = 0;
  int as_verify = 0;                    // 1: FP64 residual in flight, 2: |A||x| in flight
  double as_true = 0.0;                 // FP64 residual while |A||x| is in flight
  double as_prev_true = 0.0;            // FP64 residual of the previous check
  double as_nb = 0.0, as_rtol = 0.0, as_rel = 0.0;
  double* host_x = nullptr;             // pinned staging of the compact result
  cudaEvent_t as_ev = nullptr;
  // exact coarse solve on level `coarse` by global fast diagonalisation
  int coarse = 1;
  int gni = 0;                          // interior nodes per direction on that level
  void* gS = nullptr;                   // S then S^T (gni x gni each), working precision
  void* ginv = nullptr;                 // h^(2-d) / (sum of eigenvalues), gni^d
  void* gt1 = nullptr;                  // two gni^d work tensors
  void* gt2 = nullptr;
};

namespace {

int fail(vps_context* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  else g_create_error = buf;
  return code;
}

#define VPS_CK(h, expr)                                                                  \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail((h), e_ == cudaErrorMemoryAllocation ? VPS_ENOMEM : VPS_ECUDA, "%s: %s", \
                  #expr, cudaGetErrorString(e_));                                        \
  } while (0)

int dalloc(vps_context* h, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(h, e == cudaErrorMemoryAllocation ? VPS_ENOMEM : VPS_ECUDA,
                "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  h->allocs.push_back(*p);
  h->bytes += bytes;
  e = cudaMemsetAsync(*p, 0, bytes, h->stream);
  if (e != cudaSuccess) return fail(h, VPS_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  return VPS_OK;
}

int set_device(vps_context* h) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != h->device) {
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return fail(h, VPS_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  }
  return VPS_OK;
}

// Drops the captured V-cycle graphs (after a change of level data, variant
// or coarse level); they are captured again on next use.
void drop_graphs(vps_context* h) {
  if (h->prec_graph) cudaGraphExecDestroy(h->prec_graph);
  if (h->prec_graph_ns) cudaGraphExecDestroy(h->prec_graph_ns);
  if (h->cg_loop_graph) cudaGraphExecDestroy(h->cg_loop_graph);
  h->prec_graph = h->prec_graph_ns = h->cg_loop_graph = nullptr;
}

// Adds the kernels launched during an entry point to the handle's tally.
struct LaunchTally {
  vps_context* h;
  int64_t start;
  explicit LaunchTally(vps_context* hh) : h(hh), start(launch_counter()) {}
  ~LaunchTally() { h->kernels += launch_counter() - start; }
};

int check_level(vps_context* h, int level, int lo) {
  if (level < lo || level > h->L)
    return fail(h, VPS_EINVAL, "level %d outside %d..%d", level, lo, h->L);
  return VPS_OK;
}

// ------------------------------------------------------------ smoothing
template <typename T>
const KernelFns<T>& fns(vps_context* h);
template <>
const KernelFns<float>& fns<float>(vps_context* h) { return h->ks->f; }
template <>
const KernelFns<double>& fns<double>(vps_context* h) { return h->ks->d; }

// y = A_l x, or y = b - A_l x, with the level's operator tile structure.
template <typename T>
cudaError_t level_apply(vps_context* h, int l, const T* x, const T* b, T* y) {
  const KernelFns<T>& F = fns<T>(h);
  if (h->op_var[l] && F.apply_alt) return F.apply_alt(h->geom[l], x, b, y, h->stream);
  return F.apply(h->geom[l], x, b, y, h->stream);
}

// One colour pass of the multiplicative smoother with the handle's kernel
// structure (Section 3.1): Fused (one kernel), Separate (local residual
// kernel, then the local solve), Global (global residual by the operator,
// then the local solve), Global with the dense inverse as local solver.
template <typename T>
int colour_pass(vps_context* h, int l, int c, const T* b, T* x) {
  const KernelFns<T>& F = fns<T>(h);
  const LevelGeom& g = h->geom[l];
  const ColourGeom cg = make_colour(g, c);
  const T* il = static_cast<const T*>(h->inv_lam);
  const int v = h->smooth_var[l];
  T* r = static_cast<T*>(h->rv[l]);
  int q = v % kQVariants;
  if (!F.smooth_add_v[q]) q = 0;
  switch (h->kernel_kind) {
    case VPS_KERNEL_SEPARATE:
      if (!F.resid_v[q]) return fail(h, VPS_EINVAL, "Separate kernel unavailable");
      VPS_CK(h, F.resid_v[q](g, cg, b, x, r, h->stream));
      VPS_CK(h, F.smooth_add_v[q](g, cg, r, x, il, T(1), h->stream));
      return VPS_OK;
    case VPS_KERNEL_GLOBAL:
      VPS_CK(h, level_apply<T>(h, l, x, b, r));
      VPS_CK(h, F.smooth_add_v[q](g, cg, r, x, il, T(1), h->stream));
      return VPS_OK;
    case VPS_KERNEL_GLOBAL_INVERSE:
      if (!F.inverse_solve || !h->ainv) return fail(h, VPS_EINVAL, "dense inverse unavailable");
      VPS_CK(h, level_apply<T>(h, l, x, b, r));
      VPS_CK(h, F.inverse_solve(g, cg, r, x, static_cast<const T*>(h->ainv), h->stream));
      return VPS_OK;
    default:
      if (h->schedule != VPS_SCHEDULE_PLAIN || !F.smooth_mult_plain_v[v])
        VPS_CK(h, F.smooth_mult_v[v](g, cg, b, x, il, h->stream));
      else VPS_CK(h, F.smooth_mult_plain_v[v](g, cg, b, x, il, h->stream));
      return VPS_OK;
  }
}

// The dataflow sweep of level l over the colours in forward (0 .. 2^d-1)
// or backward order, for the variant's patches per block.
SweepGeom sweep_geom(vps_context* h, int l, bool forward, int patches_per_block) {
  SweepGeom sg;
  const LevelGeom& g = h->geom[l];
  const int nc = 1 << h->dim;
  sg.ncol = nc;
  sg.ncell = (int)g.ncell;
  ColourGeom byc[8];
  int64_t off = 0;
  for (int c = 0; c < nc; ++c) {
    byc[c] = make_colour(g, c);
    sg.flag_off[c] = off;
    off += byc[c].npatch;
  }
  int64_t tiles = 0;
  for (int s = 0; s < nc; ++s) {
    const int c = forward ? s : nc - 1 - s;
    sg.colour[s] = c;
    sg.pos_of[c] = s;
    sg.cg[s] = byc[c];
    tiles += (byc[c].npatch + patches_per_block - 1) / patches_per_block;
    sg.tile_end[s] = tiles;
  }
  sg.flags = h->sweep_flags[l];
  sg.ctr = h->sweep_ctr + l;
  sg.err = h->wait_err;
  sg.spin_limit = h->spin_limit;
  return sg;
}

template <typename T>
int smooth_step(vps_context* h, int l, const T* b, T* x, bool forward) {
  const LevelGeom& g = h->geom[l];
  const int nc = 1 << h->dim;
  const T* il = static_cast<const T*>(h->inv_lam);
  const int v = h->smooth_var[l];
  if (v < 0 || v >= kSmoothVariants ||
      !(h->smoother == VPS_ADDITIVE ? fns<T>(h).smooth_add_v[v] != nullptr
                                    : fns<T>(h).smooth_mult_v[v] != nullptr))
    return fail(h, VPS_EINVAL, "smoother variant %d unavailable", v);
  if (h->smoother == VPS_ADDITIVE) {
    T* r = static_cast<T*>(h->rv[l]);
    VPS_CK(h, level_apply<T>(h, l, x, b, r));
    for (int c = 0; c < nc; ++c)
      VPS_CK(h, fns<T>(h).smooth_add_v[v](g, make_colour(g, c), r, x, il, (T)h->damping,
                                          h->stream));
  } else if (h->schedule == VPS_SCHEDULE_SWEEP && h->kernel_kind == VPS_KERNEL_FUSED &&
             fns<T>(h).smooth_sweep_v[v]) {
    const SweepGeom sg = sweep_geom(h, l, forward, fns<T>(h).variant_p[v]);
    h->waits_ran = true;
    VPS_CK(h, fns<T>(h).smooth_sweep_v[v](g, sg, b, x, il, h->stream));
  } else {
    for (int i = 0; i < nc; ++i) {
      const int c = forward ? i : nc - 1 - i;
      if (int rc = colour_pass<T>(h, l, c, b, x)) return rc;
    }
  }
  return VPS_OK;
}

// VPS_ETIMEOUT if a wait of a dataflow sweep of this handle expired since
// the last check (synchronises the stream), else VPS_OK; clears the record.
int check_waits(vps_context* h) {
  if (!h->waits_ran || !h->wait_err) return VPS_OK;
  int err = 0;
  VPS_CK(h, cudaStreamSynchronize(h->stream));
  VPS_CK(h, cudaMemcpy(&err, h->wait_err, sizeof(int), cudaMemcpyDeviceToHost));
  h->waits_ran = false;
  if (!err) return VPS_OK;
  VPS_CK(h, cudaMemset(h->wait_err, 0, sizeof(int)));
  return fail(h, VPS_ETIMEOUT, "a dependency wait of a smoothing sweep reached its limit");
}

// x = A_l^{-1} b on the coarse level by global fast diagonalisation: S^T
// along z, y, x (the last pass scaled by 1/(sum of eigenvalues)), then S back.
template <typename T>
int coarse_solve(vps_context* h, const T* b, T* x) {
  const LevelGeom& g = h->geom[h->coarse];
  const int ni = h->gni, d = h->dim, px = (int)g.px, pz = (int)g.pz;
  const T* S = static_cast<const T*>(h->gS);      // W of the S^T passes
  const T* St = S + (size_t)ni * fd_pad(ni);       // W of the S passes
  const T* inv = static_cast<const T*>(h->ginv);
  T* t1 = static_cast<T*>(h->gt1);
  T* t2 = static_cast<T*>(h->gt2);
  cudaStream_t st = h->stream;
  const bool wide = h->coarse_wide;
  if (h->coarse_coop) {
    GridSync gs;
    gs.count = h->gsync;
    gs.gen = h->gsync + 1;
    gs.err = h->wait_err;
    gs.limit = h->spin_limit;
    h->waits_ran = true;
    VPS_CK(h, launch_fd_global_solve<T>(b, x, S, St, inv, t1, t2, ni, d, px, pz, g.total, gs, wide,
                                        st));
    return VPS_OK;
  }
  VPS_CK(h, cudaMemsetAsync(x, 0, g.total * sizeof(T), st));
  if (d == 3) {
    VPS_CK(h, launch_fd_global_pass<T>(0, b, t1, S, inv, ni, d, true, false, px, pz, wide, st));
    VPS_CK(h, launch_fd_global_pass<T>(0, t1, t2, S, inv, ni, d, false, false, px, pz, wide, st));
    VPS_CK(h, launch_fd_global_pass<T>(1, t2, t1, S, inv, ni, d, false, false, px, pz, wide, st));
    VPS_CK(h, launch_fd_global_pass<T>(2, t1, t2, St, inv, ni, d, false, false, px, pz, wide, st));
    VPS_CK(h, launch_fd_global_pass<T>(2, t2, t1, St, inv, ni, d, false, false, px, pz, wide, st));
    VPS_CK(h, launch_fd_global_pass<T>(2, t1, x, St, inv, ni, d, false, true, px, pz, wide, st));
  } else {
    VPS_CK(h, launch_fd_global_pass<T>(0, b, t1, S, inv, ni, d, true, false, px, pz, wide, st));
    VPS_CK(h, launch_fd_global_pass<T>(1, t1, t2, S, inv, ni, d, false, false, px, pz, wide, st));
    VPS_CK(h, launch_fd_global_pass<T>(2, t2, t1, St, inv, ni, d, false, false, px, pz, wide, st));
    VPS_CK(h, launch_fd_global_pass<T>(2, t1, x, St, inv, ni, d, false, true, px, pz, wide, st));
  }
  return VPS_OK;
}

// Automatic coarsest level: the finest level below L with at most 32
// interior nodes per direction (level 1 if none).
int auto_coarse_level(int k, int L) {
  int best = 1;
  for (int l = 1; l < L; ++l)
    if (k * (1 << l) - 1 <= 32) best = l;
  return best;
}

// Builds the global fast-diagonalisation data of level lc (allocates).
int setup_coarse(vps_context* h, int lc) {
  std::vector<double> S, lam;
  char ebuf[256];
  if (!build_global_fd(h->k, lc, &S, &lam, ebuf, sizeof(ebuf)))
    return fail(h, VPS_EINVAL, "coarse level %d: %s", lc, ebuf);
  const int ni = (int)lam.size(), d = h->dim;
  const size_t nd = (size_t)ni * ni * (d == 3 ? ni : 1);
  const double hs = std::pow(h->geom[lc].h, 2 - d);  // A^{-1} = h^(2-d) A_ref^{-1}
  std::vector<double> inv(nd);
  for (size_t a = 0; a < nd; ++a) {
    const size_t i0 = a % ni, i1 = (a / ni) % ni, i2 = a / ((size_t)ni * ni);
    inv[a] = hs / (lam[i0] + lam[i1] + (d == 3 ? lam[i2] : 0.0));
  }
  for (void* p : {h->gS, h->ginv, h->gt1, h->gt2})
    if (p) {
      cudaFree(p);
      for (auto& q : h->allocs)
        if (q == p) q = nullptr;
    }
  h->gS = h->ginv = h->gt1 = h->gt2 = nullptr;
  int rc;
  // gS: S followed by S^T (both row-major, rows of fd_pad(ni) with zeros
  // past ni); work tensors: ni rows of fd_pad(ni^(d-1))
  const int nip = fd_pad(ni);
  const size_t nt = (size_t)ni * fd_pad(d == 3 ? ni * ni : ni);
  std::vector<double> Sp(2 * (size_t)ni * nip, 0.0);
  for (int i = 0; i < ni; ++i)
    for (int j = 0; j < ni; ++j) {
      Sp[(size_t)i * nip + j] = S[(size_t)i * ni + j];
      Sp[(size_t)(ni + i) * nip + j] = S[(size_t)j * ni + i];
    }
  S.swap(Sp);
  if ((rc = dalloc(h, &h->gS, S.size() * h->esz)) || (rc = dalloc(h, &h->ginv, nd * h->esz)) ||
      (rc = dalloc(h, &h->gt1, nt * h->esz)) || (rc = dalloc(h, &h->gt2, nt * h->esz)))
    return rc;
  cudaError_t e;
  // pageable source: the copies are staged before the calls return
  if (h->prec == VPS_FP64) {
    e = cudaMemcpyAsync(h->gS, S.data(), S.size() * sizeof(double), cudaMemcpyHostToDevice,
                        h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->ginv, inv.data(), nd * sizeof(double), cudaMemcpyHostToDevice,
                          h->stream);
  } else {
    std::vector<float> Sf(S.begin(), S.end()), invf(inv.begin(), inv.end());
    e = cudaMemcpyAsync(h->gS, Sf.data(), Sf.size() * sizeof(float), cudaMemcpyHostToDevice,
                        h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->ginv, invf.data(), nd * sizeof(float), cudaMemcpyHostToDevice,
                          h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  if (e != cudaSuccess) return fail(h, VPS_ECUDA, "coarse tables: %s", cudaGetErrorString(e));
  h->coarse = lc;
  h->gni = ni;
  drop_graphs(h);
  return VPS_OK;
}

// x_top = Vcycle_top(A_top, 0, b_top) (Algorithm 1) in working precision T,
// top = 0: the finest level.  symmetric: post-smoothing visits the colours
// in reverse order (an SPD preconditioner for CG); otherwise in the same
// order as pre-smoothing (S_l on both sides, as Algorithm 1 prints it).
template <typename T>
int vcycle_core(vps_context* h, const T* bL, T* xL, int top = 0, bool symmetric = true) {
  const KernelFns<T>& F = fns<T>(h);
  if (top == 0) top = h->L;
  const T* b[kMaxLevels + 1];
  T* x[kMaxLevels + 1];
  for (int l = 1; l <= h->L; ++l) {
    b[l] = static_cast<const T*>(h->bv[l]);
    x[l] = static_cast<T*>(h->xv[l]);
  }
  b[top] = bL;
  x[top] = xL;
  const int lc = h->coarse;
  for (int l = top; l > lc; --l) {
    const LevelGeom& g = h->geom[l];
    VPS_CK(h, cudaMemsetAsync(x[l], 0, g.total * sizeof(T), h->stream));
    for (int s = 0; s < h->n_pre; ++s) {
      int rc = smooth_step<T>(h, l, b[l], x[l], true);
      if (rc) return rc;
    }
    T* r = static_cast<T*>(h->rv[l]);
    VPS_CK(h, level_apply<T>(h, l, x[l], b[l], r));
    VPS_CK(h, F.restrict_(g, h->geom[l - 1], r, static_cast<T*>(h->bv[l - 1]), h->stream));
  }
  // coarsest level: exact solve (Algorithm 1's coarse grid solver)
  {
    int rc = coarse_solve<T>(h, b[lc], x[lc]);
    if (rc) return rc;
  }
  for (int l = lc + 1; l <= top; ++l) {
    VPS_CK(h, F.prolong_add(h->geom[l], h->geom[l - 1], x[l - 1], x[l], h->stream));
    for (int s = 0; s < h->n_post; ++s) {
      int rc = smooth_step<T>(h, l, b[l], x[l], !symmetric);
      if (rc) return rc;
    }
  }
  return VPS_OK;
}

// z_new = B cr: FP64 V-cycle into czn, or cast -> FP32 V-cycle; the
// symmetric cycle (CG) leaves its FP32 output in xv[L], which the CG
// kernels read directly; the non-symmetric one of Algorithm 1 (GMRES)
// converts it into czn.
int precondition_direct(vps_context* h, bool symmetric) {
  const LevelGeom& g = h->geom[h->L];
  if (h->prec == VPS_FP64) return vcycle_core<double>(h, h->cr, h->czn, 0, symmetric);
  VPS_CK(h, launch_cast_d2f(h->cr, static_cast<float*>(h->bv[h->L]), g.total, h->stream));
  int rc = vcycle_core<float>(h, static_cast<const float*>(h->bv[h->L]),
                              static_cast<float*>(h->xv[h->L]), 0, symmetric);
  if (rc) return rc;
  if (!symmetric)
    VPS_CK(h, launch_cast_f2d(static_cast<const float*>(h->xv[h->L]), h->czn, g.total, h->stream));
  return VPS_OK;
}

int precondition(vps_context* h, bool symmetric = true) {
  if (!h->use_graphs) return precondition_direct(h, symmetric);
  cudaGraphExec_t& exec = symmetric ? h->prec_graph : h->prec_graph_ns;
  int64_t& nk = symmetric ? h->graph_kernels : h->graph_kernels_ns;
  if (!exec) {
    cudaGraph_t graph = nullptr;
    VPS_CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    const int64_t before = launch_counter();
    int rc = precondition_direct(h, symmetric);
    nk = launch_counter() - before;
    launch_counter() = before;  // captured, not launched
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return fail(h, VPS_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      exec = nullptr;
      return fail(h, VPS_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
  }
  VPS_CK(h, cudaGraphLaunch(exec, h->stream));
  launch_counter() += nk;
  return VPS_OK;
}

bool outer_df(const vps_context* h) { return h->outer == VPS_OUTER_DOUBLE_FLOAT; }

// p = z_old = z_new (the preconditioned residual: xv[L] in FP32, czn in
// FP64), rzn = r . z_new for the first alpha.
int cg_start_direction(vps_context* h) {
  const int64_t n = h->geom[h->L].total;
  float* ph = outer_df(h) ? h->cph : nullptr;
  if (h->prec == VPS_FP32)
    VPS_CK(h, launch_cg_start<float>(h->cp, h->cz, static_cast<const float*>(h->xv[h->L]), h->cr,
                                     n, h->partial, h->sc, h->stream, ph, h->cpl));
  else
    VPS_CK(h, launch_cg_start<double>(h->cp, h->cz, h->czn, h->cr, n, h->partial, h->sc,
                                      h->stream, ph, h->cpl));
  return VPS_OK;
}

// beta, p = z_new + beta p, z_old = z_new (after precondition(h)).
int cg_next_direction(vps_context* h) {
  const int64_t n = h->geom[h->L].total;
  float* ph = outer_df(h) ? h->cph : nullptr;
  if (h->prec == VPS_FP32)
    VPS_CK(h, launch_cg_next_p<float>(h->cp, h->cz, static_cast<const float*>(h->xv[h->L]), h->cr,
                                      n, h->partial, h->sc, h->stream, ph, h->cpl));
  else
    VPS_CK(h, launch_cg_next_p<double>(h->cp, h->cz, h->czn, h->cr, n, h->partial, h->sc,
                                       h->stream, ph, h->cpl));
  return VPS_OK;
}

// alpha, x and r updates, r . r (after A p).
int cg_step(vps_context* h) {
  const int64_t n = h->geom[h->L].total;
  VPS_CK(h, launch_cg_step_xr(h->cx, h->cr, h->cp, h->cAp, n, h->partial, h->partial2, h->sc,
                              h->stream));
  return VPS_OK;
}

// Ap = A p with the handle's outer operator.
int cg_apply_p(vps_context* h) {
  const LevelGeom& g = h->geom[h->L];
  if (outer_df(h)) VPS_CK(h, h->ks->apply_df(g, h->cph, h->cpl, h->cAp, h->stream));
  else VPS_CK(h, h->ks->d.apply(g, h->cp, nullptr, h->cAp, h->stream));
  return VPS_OK;
}

// r = b - A x with the FP64 operator, r . r into sc->rr (asynchronous).
int cg_true_residual(vps_context* h) {
  const LevelGeom& g = h->geom[h->L];
  VPS_CK(h, h->ks->d.apply(g, h->cx, h->cb, h->cr, h->stream));
  VPS_CK(h, launch_dot1(h->cr, h->cr, g.total, h->partial, &h->sc->rr, h->stream));
  return VPS_OK;
}

// U = |A| |x| into cAp and U . U into sc->pAp (asynchronous).
int cg_residual_scale(vps_context* h) {
  const LevelGeom& g = h->geom[h->L];
  VPS_CK(h, h->ks->apply_abs(g, h->cx, h->cAp, h->stream));
  VPS_CK(h, launch_dot1(h->cAp, h->cAp, g.total, h->partial, &h->sc->pAp, h->stream));
  return VPS_OK;
}

// Relative rounding bound of the FP64 residual evaluation: every entry of
// b - A x is computed with an error below gamma (|A| |x|)_i, gamma the
// first-order bound (chain length) u of the sum-factorised contractions.
double residual_gamma(const vps_context* h) { return (6.0 * h->k + 6.0) * std::ldexp(1.0, -53); }

// Outcome of a convergence check on the FP64 residual.
enum { kCheckConverged = 1, kCheckRestart = 0, kCheckStagnated = -1 };

// A restart from the FP64 residual that did not halve it: the residual has
// stopped falling, and the rounding bound decides (needs_scale).
bool stagnating(double rel_true, double prev_true) {
  return prev_true > 0.0 && !(rel_true < 0.5 * prev_true);
}

// rel_true = ||b - A x|| / ||b||; scale_norm = || |A||x| || (needed only when
// stagnating).  Above rtol the solve first restarts from the FP64 residual;
// the rounding bound (a worst-case bound, so it is only trusted once the
// residual has stopped falling) then ends it with VPS_OK or VPS_ENOCONV.
int classify_check(vps_context* h, double rtol, double nb, double rel_true, double scale_norm,
                   double prev_true) {
  if (rel_true <= rtol) return kCheckConverged;
  if (!stagnating(rel_true, prev_true)) return kCheckRestart;
  if (scale_norm >= 0.0 && rel_true * nb <= residual_gamma(h) * scale_norm) {
    h->last_at_floor = 1;
    return kCheckConverged;
  }
  return kCheckStagnated;
}

// The device-side CG loop: a graph whose conditional while-node repeats one
// iteration (V-cycle, direction, A p, x/r update, r.r and the stopping
// test) without returning to the host; the host takes over to confirm
// convergence on the FP64 residual.  Built on first use; if this driver
// cannot build it, the host loop is used.
int ensure_cg_loop(vps_context* h) {
  if (h->cg_loop_graph || h->cg_loop_off) return VPS_OK;
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle cond;
  cudaGraphNodeParams np = {};
  cudaGraphNode_t node;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  }
  cudaGraph_t body = nullptr;
  if (e == cudaSuccess) {
    body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
  }
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    h->cg_loop_off = true;
    return VPS_OK;
  }
  const int64_t before = launch_counter();
  int rc = precondition_direct(h, true);
  if (!rc) rc = cg_next_direction(h);
  if (!rc) rc = cg_apply_p(h);
  if (!rc) rc = cg_step(h);
  if (!rc) {
    cudaError_t ek = launch_cg_loop_check(cond, h->sc, h->stream);
    if (ek != cudaSuccess) rc = fail(h, VPS_ECUDA, "loop check: %s", cudaGetErrorString(ek));
  }
  h->cg_loop_kernels = launch_counter() - before;
  launch_counter() = before;  // captured, not launched
  e = cudaStreamEndCapture(h->stream, &body);
  if (rc == VPS_OK && e == cudaSuccess) e = cudaGraphInstantiate(&h->cg_loop_graph, g, 0);
  cudaGraphDestroy(g);
  if (rc) return rc;
  if (e != cudaSuccess) {
    h->cg_loop_graph = nullptr;
    cudaGetLastError();
    h->cg_loop_off = true;
  }
  return VPS_OK;
}

// Preconditioned CG (Section 4.1's outer solver) with the flexible
// (Polak-Ribiere) beta.  Convergence is always confirmed on the residual
// r = b - A x evaluated in FP64: the recursive residual can drift from it
// (double-float outer operator: by about 2^-48 of the magnitudes of the
// operator's terms), and on fine meshes rtol can lie below what FP64 can
// resolve at all (the terms of A x cancel by about k^2 h^-2).  The solve
// ends when the FP64 residual is below rtol, or below the rounding bound of
// its own evaluation (gamma || |A||x| ||); otherwise CG restarts from it,
// and a restart that does not halve it ends the solve (VPS_ENOCONV).
int cg_solve(vps_context* h, double rtol, int max_it, int* iters, double* rel_res) {
  const LevelGeom& g = h->geom[h->L];
  const int64_t n = g.total;
  // ||b||
  VPS_CK(h, launch_dot1(h->cb, h->cb, n, h->partial, h->dots, h->stream));
  VPS_CK(h, cudaMemcpyAsync(h->host_dots, h->dots, sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
  VPS_CK(h, cudaStreamSynchronize(h->stream));
  const double nb = std::sqrt(h->host_dots[0]);
  VPS_CK(h, cudaMemsetAsync(h->cx, 0, n * sizeof(double), h->stream));
  h->last_restarts = 0;
  h->last_at_floor = 0;
  if (iters) *iters = 0;
  if (rel_res) *rel_res = 0.0;
  if (!(nb > 0.0)) {
    if (!std::isfinite(nb)) return fail(h, VPS_EBREAKDOWN, "right-hand side is not finite");
    return VPS_OK;
  }
  VPS_CK(h, cudaMemcpyAsync(h->cr, h->cb, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  VPS_CK(h, cudaMemsetAsync(h->sc, 0, sizeof(CgScalars), h->stream));
  int rc = precondition(h);
  if (rc) return rc;
  if ((rc = cg_start_direction(h))) return rc;
  double rel = 1.0, prev_true = 0.0;
  int it = 0;
  bool fresh = false;  // host_sc already holds the scalars of iteration it
  while (true) {
    if (!fresh) {
      if ((rc = cg_apply_p(h))) return rc;
      if ((rc = cg_step(h))) return rc;
      ++it;
      VPS_CK(h, cudaMemcpyAsync(h->host_sc, h->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost,
                                h->stream));
      VPS_CK(h, cudaStreamSynchronize(h->stream));
    }
    fresh = false;
    if (h->host_sc->flag) {
      if (iters) *iters = it;
      return fail(h, VPS_EBREAKDOWN, "CG breakdown at iteration %d (p^T A p = %g)", it,
                  h->host_sc->pAp);
    }
    rel = std::sqrt(h->host_sc->rr) / nb;
    if (iters) *iters = it;
    if (rel_res) *rel_res = rel;
    if (!std::isfinite(rel))
      return fail(h, VPS_EBREAKDOWN, "CG residual not finite at iteration %d", it);
    bool restart = false;
    if (rel <= rtol) {
      if ((rc = cg_true_residual(h))) return rc;
      VPS_CK(h, cudaMemcpyAsync(h->host_sc, h->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost,
                                h->stream));
      const bool read_waits = h->waits_ran;  // the wait-expiry word, in the same synchronisation
      if (read_waits)
        VPS_CK(h, cudaMemcpyAsync(h->host_err, h->wait_err, sizeof(int), cudaMemcpyDeviceToHost,
                                  h->stream));
      VPS_CK(h, cudaStreamSynchronize(h->stream));
      if (read_waits) {
        h->waits_ran = false;
        if (*h->host_err) {
          VPS_CK(h, cudaMemset(h->wait_err, 0, sizeof(int)));
          return fail(h, VPS_ETIMEOUT, "a dependency wait of a smoothing sweep reached its limit");
        }
      }
      rel = std::sqrt(h->host_sc->rr) / nb;
      if (rel_res) *rel_res = rel;
      if (!std::isfinite(rel))
        return fail(h, VPS_EBREAKDOWN, "CG residual not finite at iteration %d", it);
      double unorm = -1.0;
      if (rel > rtol && stagnating(rel, prev_true)) {  // at the rounding level of its evaluation?
        if ((rc = cg_residual_scale(h))) return rc;
        VPS_CK(h, cudaMemcpyAsync(h->host_sc, h->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost,
                                  h->stream));
        VPS_CK(h, cudaStreamSynchronize(h->stream));
        unorm = std::sqrt(h->host_sc->pAp);
      }
      const int cls = classify_check(h, rtol, nb, rel, unorm, prev_true);
      if (cls == kCheckConverged) return VPS_OK;
      if (cls == kCheckStagnated)
        return fail(h, VPS_ENOCONV,
                    "CG stagnated at an FP64 residual of %g (rtol %g, rounding bound %g)", rel, rtol,
                    residual_gamma(h) * unorm / nb);
      prev_true = rel;
      ++h->last_restarts;
      restart = true;
    }
    if (it >= max_it) break;
    if (!restart && h->use_graphs) {
      if ((rc = ensure_cg_loop(h))) return rc;
      if (h->cg_loop_graph) {  // the next iterations on the device
        VPS_CK(h, launch_cg_loop_init(h->sc, it, max_it, nb, rtol, h->stream));
        VPS_CK(h, cudaGraphLaunch(h->cg_loop_graph, h->stream));
        VPS_CK(h, cudaMemcpyAsync(h->host_sc, h->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost,
                                  h->stream));
        VPS_CK(h, cudaStreamSynchronize(h->stream));
        launch_counter() += (int64_t)(h->host_sc->it - it) * h->cg_loop_kernels;
        it = h->host_sc->it;
        fresh = true;
        continue;
      }
    }
    rc = precondition(h);
    if (rc) return rc;
    if (restart) {
      VPS_CK(h, cudaMemsetAsync(h->sc, 0, sizeof(CgScalars), h->stream));
      if ((rc = cg_start_direction(h))) return rc;
    } else if ((rc = cg_next_direction(h))) {
      return rc;
    }
  }
  return fail(h, VPS_ENOCONV, "CG did not reach %g in %d iterations (%g)", rtol, max_it, rel);
}

// GMRES buffers for restart length m (allocated on first use, kept).
int gmres_alloc(vps_context* h, int m) {
  if (h->gm_m == m) return VPS_OK;
  for (double* p : {h->gmV, h->gmZ, h->gm_partial, h->gm_dev})
    if (p) {
      cudaStreamSynchronize(h->stream);
      cudaFree(p);
      for (auto& q : h->allocs)
        if (q == p) q = nullptr;
    }
  h->gmV = h->gmZ = h->gm_partial = h->gm_dev = nullptr;
  if (h->gm_host) cudaFreeHost(h->gm_host);
  h->gm_host = nullptr;
  h->gm_m = 0;
  const int64_t ld = (h->geom[h->L].total + 31) / 32 * 32;
  void* p;
  if (int rc = dalloc(h, &p, (size_t)(m + 1) * ld * sizeof(double))) return rc;
  h->gmV = (double*)p;
  if (int rc = dalloc(h, &p, (size_t)m * ld * sizeof(double))) return rc;
  h->gmZ = (double*)p;
  if (int rc = dalloc(h, &p, (size_t)(m + 1) * kDotBlocks * sizeof(double))) return rc;
  h->gm_partial = (double*)p;
  if (int rc = dalloc(h, &p, (size_t)(3 * m + 8) * sizeof(double))) return rc;
  h->gm_dev = (double*)p;
  VPS_CK(h, cudaMallocHost(&p, (size_t)(3 * m + 8) * sizeof(double)));
  h->gm_host = (double*)p;
  h->gm_ld = ld;
  h->gm_m = m;
  return VPS_OK;
}

// Flexible GMRES on the finest level (the outer solver of Section 4),
// right-preconditioned by the V-cycle of Algorithm 1 (non-symmetric),
// x0 = 0, restarted every m products A z.  Arnoldi by classical
// Gram-Schmidt applied twice (two block reductions per step, deterministic);
// Givens rotations on the host.  A cycle ends when the least-squares
// residual reaches rtol ||b||, then the residual is evaluated in FP64 and
// checked as in cg_solve (rtol, or the rounding bound of its evaluation);
// otherwise the next cycle starts from it.  *iters: products A z.
int gmres_solve(vps_context* h, int m, double rtol, int max_it, int* iters, double* rel_res) {
  const LevelGeom& g = h->geom[h->L];
  const int64_t n = g.total;
  if (int rc = gmres_alloc(h, m)) return rc;
  const int64_t ld = h->gm_ld;
  double* V = h->gmV;
  double* Z = h->gmZ;
  double* hd = h->gm_dev;   // [0, m]: first projection, [m+1, 2m+1]: second, [2m+2]: ||w||^2
  double* hh = h->gm_host;
  h->last_restarts = 0;
  h->last_at_floor = 0;
  if (iters) *iters = 0;
  if (rel_res) *rel_res = 0.0;
  VPS_CK(h, launch_dot1(h->cb, h->cb, n, h->partial, h->dots, h->stream));
  VPS_CK(h, cudaMemcpyAsync(h->host_dots, h->dots, sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
  VPS_CK(h, cudaStreamSynchronize(h->stream));
  const double nb = std::sqrt(h->host_dots[0]);
  VPS_CK(h, cudaMemsetAsync(h->cx, 0, n * sizeof(double), h->stream));
  if (!(nb > 0.0)) {
    if (!std::isfinite(nb)) return fail(h, VPS_EBREAKDOWN, "right-hand side is not finite");
    return VPS_OK;
  }
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
  auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  VPS_CK(h, cudaMemcpyAsync(h->cr, h->cb, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  double beta = nb, prev_true = 0.0;
  int it = 0;
  while (true) {
    VPS_CK(h, launch_scale(V, h->cr, 1.0 / beta, n, h->stream));
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int j = 0;
    double est = beta / nb;
    while (j < m && it < max_it) {
      double* vj = V + (size_t)j * ld;
      double* zj = Z + (size_t)j * ld;
      double* w = V + (size_t)(j + 1) * ld;
      // z_j = B v_j (input cr, output czn), w = A z_j
      VPS_CK(h, cudaMemcpyAsync(h->cr, vj, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
      if (int rc = precondition(h, false)) return rc;
      VPS_CK(h, cudaMemcpyAsync(zj, h->czn, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
      if (outer_df(h)) {
        VPS_CK(h, launch_split_df(zj, h->cph, h->cpl, n, h->stream));
        VPS_CK(h, h->ks->apply_df(g, h->cph, h->cpl, w, h->stream));
      } else {
        VPS_CK(h, h->ks->d.apply(g, zj, nullptr, w, h->stream));
      }
      // w -= V h twice (classical Gram-Schmidt with one reorthogonalisation)
      VPS_CK(h, launch_multi_dot(V, ld, j + 1, w, n, h->gm_partial, hd, h->stream));
      VPS_CK(h, launch_multi_axpy(w, V, ld, j + 1, hd, -1.0, n, h->stream));
      VPS_CK(h, launch_multi_dot(V, ld, j + 1, w, n, h->gm_partial, hd + m + 1, h->stream));
      VPS_CK(h, launch_multi_axpy(w, V, ld, j + 1, hd + m + 1, -1.0, n, h->stream));
      VPS_CK(h, launch_dot1(w, w, n, h->partial, hd + 2 * m + 2, h->stream));
      VPS_CK(h, cudaMemcpyAsync(hh, hd, (size_t)(2 * m + 3) * sizeof(double),
                                cudaMemcpyDeviceToHost, h->stream));
      VPS_CK(h, cudaStreamSynchronize(h->stream));
      for (int i = 0; i <= j; ++i) Hij(i, j) = hh[i] + hh[m + 1 + i];
      const double hn = std::sqrt(hh[2 * m + 2]);
      Hij(j + 1, j) = hn;
      if (!std::isfinite(hn))
        return fail(h, VPS_EBREAKDOWN, "GMRES: non-finite Arnoldi vector at step %d", it + 1);
      if (hn > 0.0) VPS_CK(h, launch_scale(w, w, 1.0 / hn, n, h->stream));
      for (int i = 0; i < j; ++i) {  // previous rotations on the new column
        const double t = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
        Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
        Hij(i, j) = t;
      }
      const double den = std::hypot(Hij(j, j), Hij(j + 1, j));
      if (!(den > 0.0)) return fail(h, VPS_EBREAKDOWN, "GMRES: breakdown at step %d", it + 1);
      cs[j] = Hij(j, j) / den;
      sn[j] = Hij(j + 1, j) / den;
      Hij(j, j) = den;
      Hij(j + 1, j) = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      ++j;
      ++it;
      est = std::fabs(gv[j]) / nb;
      if (iters) *iters = it;
      if (rel_res) *rel_res = est;
      if (est <= rtol || hn == 0.0) break;
    }
    // x += Z y,  H[:j,:j] y = g[:j]
    for (int i = j - 1; i >= 0; --i) {
      double t = gv[i];
      for (int q = i + 1; q < j; ++q) t -= Hij(i, q) * y[q];
      y[i] = t / Hij(i, i);
    }
    for (int i = 0; i < j; ++i) hh[i] = y[i];
    VPS_CK(h, cudaMemcpyAsync(hd, hh, (size_t)j * sizeof(double), cudaMemcpyHostToDevice,
                              h->stream));
    VPS_CK(h, launch_multi_axpy(h->cx, Z, ld, j, hd, 1.0, n, h->stream));
    // FP64 residual
    if (int rc = cg_true_residual(h)) return rc;
    VPS_CK(h, cudaMemcpyAsync(h->host_sc, h->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost,
                              h->stream));
    VPS_CK(h, cudaStreamSynchronize(h->stream));
    const double rel_true = std::sqrt(h->host_sc->rr) / nb;
    if (rel_res) *rel_res = rel_true;
    if (!std::isfinite(rel_true)) return fail(h, VPS_EBREAKDOWN, "GMRES residual not finite");
    if (rel_true <= rtol) return VPS_OK;
    if (est <= rtol) {  // the least-squares residual had converged: drift or rounding
      double unorm = -1.0;
      if (stagnating(rel_true, prev_true)) {
        if (int rc = cg_residual_scale(h)) return rc;
        VPS_CK(h, cudaMemcpyAsync(h->host_sc, h->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost,
                                  h->stream));
        VPS_CK(h, cudaStreamSynchronize(h->stream));
        unorm = std::sqrt(h->host_sc->pAp);
      }
      const int cls = classify_check(h, rtol, nb, rel_true, unorm, prev_true);
      if (cls == kCheckConverged) return VPS_OK;
      if (cls == kCheckStagnated)
        return fail(h, VPS_ENOCONV, "GMRES stagnated at an FP64 residual of %g (rtol %g)",
                    rel_true, rtol);
      prev_true = rel_true;
      ++h->last_restarts;
    }
    if (it >= max_it)
      return fail(h, VPS_ENOCONV, "GMRES did not reach %g in %d iterations (%g)", rtol, max_it,
                  rel_true);
    beta = rel_true * nb;
  }
}

int upload_rhs_sines(vps_context* h, int level, int n_modes, const double* coef, const int* freq,
                     double* b);

// x += V_l(r) for FP64 level vectors: the V-cycle with initial guess x
// (Algorithm 1 is affine in x: V(x, b) = x + V(0, b - A x)), as printed
// (the same colour order before and after the coarse correction), in the
// handle's working precision.  r is clobbered.
int fmg_correct(vps_context* h, int l, double* r, double* x) {
  const LevelGeom& g = h->geom[l];
  if (h->prec == VPS_FP64) {
    double* c = static_cast<double*>(h->xv[l]);
    if (int rc = vcycle_core<double>(h, r, c, l, false)) return rc;
    VPS_CK(h, launch_axpy_inplace<double>(x, c, 1.0, g.total, h->stream));
  } else {
    float* bf = static_cast<float*>(h->bv[l]);
    float* c = static_cast<float*>(h->xv[l]);
    VPS_CK(h, launch_cast_d2f(r, bf, g.total, h->stream));
    if (int rc = vcycle_core<float>(h, bf, c, l, false)) return rc;
    VPS_CK(h, launch_cast_f2d(c, r, g.total, h->stream));
    VPS_CK(h, launch_axpy_inplace<double>(x, r, 1.0, g.total, h->stream));
  }
  return VPS_OK;
}

// Full multigrid (Algorithm 2): exact solve on the coarsest level, then on
// every finer level prolongation of the coarser solution and one V-cycle,
// then V-cycles on the finest level until ||b - A x|| <= tol ||b|| (norms
// and residuals in FP64).  Right-hand sides: the load vector of f on every
// level.  *iters: the V-cycles of the final loop.
int fmg_solve(vps_context* h, int n_modes, const double* coef, const int* freq, double tol,
              int max_it, int* iters, double* rel_res) {
  const int L = h->L, lc = h->coarse;
  h->last_restarts = 0;
  h->last_at_floor = 0;
  for (int l = lc; l < L; ++l)
    if (!h->fmg_b[l]) {
      const size_t bytes = (size_t)h->geom[l].total * sizeof(double);
      void* p;
      if (int rc = dalloc(h, &p, bytes)) return rc;
      h->fmg_b[l] = (double*)p;
      if (int rc = dalloc(h, &p, bytes)) return rc;
      h->fmg_x[l] = (double*)p;
      if (int rc = dalloc(h, &p, bytes)) return rc;
      h->fmg_r[l] = (double*)p;
    }
  double *fb[kMaxLevels + 1], *fx[kMaxLevels + 1], *fr[kMaxLevels + 1];
  for (int l = lc; l < L; ++l) {
    fb[l] = h->fmg_b[l];
    fx[l] = h->fmg_x[l];
    fr[l] = h->fmg_r[l];
  }
  fb[L] = h->cb;
  fx[L] = h->cx;
  fr[L] = h->cr;
  for (int l = lc; l <= L; ++l) {
    if (int rc = upload_rhs_sines(h, l, n_modes, coef, freq, h->comp_b)) return rc;
    VPS_CK(h, launch_pack<double>(h->geom[l], h->comp_b, fb[l], h->stream));
  }
  const LevelGeom& gL = h->geom[L];
  VPS_CK(h, launch_dot1(h->cb, h->cb, gL.total, h->partial, h->dots, h->stream));
  VPS_CK(h, cudaMemcpyAsync(h->host_dots, h->dots, sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
  VPS_CK(h, cudaStreamSynchronize(h->stream));
  const double nb = std::sqrt(h->host_dots[0]);
  if (iters) *iters = 0;
  if (rel_res) *rel_res = 0.0;
  if (!(nb > 0.0)) {
    VPS_CK(h, cudaMemsetAsync(h->cx, 0, gL.total * sizeof(double), h->stream));
    if (!std::isfinite(nb)) return fail(h, VPS_EBREAKDOWN, "right-hand side is not finite");
    return VPS_OK;
  }
  // coarse grid solver
  const LevelGeom& gc = h->geom[lc];
  if (h->prec == VPS_FP64) {
    if (int rc = coarse_solve<double>(h, fb[lc], fx[lc])) return rc;
  } else {
    VPS_CK(h, launch_cast_d2f(fb[lc], static_cast<float*>(h->bv[lc]), gc.total, h->stream));
    if (int rc = coarse_solve<float>(h, static_cast<const float*>(h->bv[lc]),
                                     static_cast<float*>(h->xv[lc])))
      return rc;
    VPS_CK(h, launch_cast_f2d(static_cast<const float*>(h->xv[lc]), fx[lc], gc.total, h->stream));
  }
  // nested iteration: prolongate, one V-cycle per level
  for (int l = lc + 1; l <= L; ++l) {
    const LevelGeom& g = h->geom[l];
    VPS_CK(h, cudaMemsetAsync(fx[l], 0, g.total * sizeof(double), h->stream));
    VPS_CK(h, h->ks->d.prolong_add(g, h->geom[l - 1], fx[l - 1], fx[l], h->stream));
    VPS_CK(h, h->ks->d.apply(g, fx[l], fb[l], fr[l], h->stream));
    if (int rc = fmg_correct(h, l, fr[l], fx[l])) return rc;
  }
  // V-cycles on the finest level until the residual norm has dropped by tol
  VPS_CK(h, h->ks->d.apply(gL, h->cx, h->cb, h->cr, h->stream));
  double delta = nb, prev = nb;
  int it = 0;
  while (delta > tol * nb && it < max_it) {
    if (int rc = fmg_correct(h, L, h->cr, h->cx)) return rc;
    VPS_CK(h, h->ks->d.apply(gL, h->cx, h->cb, h->cr, h->stream));
    VPS_CK(h, launch_dot1(h->cr, h->cr, gL.total, h->partial, h->dots, h->stream));
    VPS_CK(h, cudaMemcpyAsync(h->host_dots, h->dots, sizeof(double), cudaMemcpyDeviceToHost,
                              h->stream));
    VPS_CK(h, cudaStreamSynchronize(h->stream));
    delta = std::sqrt(h->host_dots[0]);
    ++it;
    if (iters) *iters = it;
    if (rel_res) *rel_res = delta / nb;
    if (!std::isfinite(delta)) return fail(h, VPS_EBREAKDOWN, "FMG residual not finite");
    if (delta > tol * nb && !(delta < 0.5 * prev)) {
      // stagnation: is the residual at the rounding level of its evaluation?
      if (int rc = cg_residual_scale(h)) return rc;
      VPS_CK(h, cudaMemcpyAsync(h->host_sc, h->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost,
                                h->stream));
      VPS_CK(h, cudaStreamSynchronize(h->stream));
      if (delta <= residual_gamma(h) * std::sqrt(h->host_sc->pAp)) {
        h->last_at_floor = 1;
        return VPS_OK;
      }
    }
    prev = delta;
  }
  if (delta > tol * nb)
    return fail(h, VPS_ENOCONV, "FMG did not reach %g in %d V-cycles (%g)", tol, max_it,
                delta / nb);
  return VPS_OK;
}

}  // namespace

namespace {

// Load vector of f = sum_m coef_m prod_t g_mt(x_t), g = sin(pi freq x) (the
// constant 1 for freq 0), on `level` into the compact device vector b: 1D
// integrals with (k+2)-point Gauss rules on the host, tensor product on the
// device (asynchronous on the handle's stream).
int upload_rhs_sines(vps_context* h, int level, int n_modes, const double* coef, const int* freq,
                     double* b) {
  const LevelGeom& g = h->geom[level];
  const int k = h->k, ni = g.n1 - 2, q = k + 2;
  double xq[16], wq[16], val[kMaxK + 1];
  gauss_rule(q, xq, wq);
  std::vector<double> b1d((size_t)n_modes * h->dim * ni, 0.0);
  std::vector<double> full(g.n1);
  for (int md = 0; md < n_modes; ++md)
    for (int t = 0; t < h->dim; ++t) {
      const double f = freq[md * h->dim + t];
      std::fill(full.begin(), full.end(), 0.0);
      for (int c = 0; c < g.ncell; ++c)
        for (int qq = 0; qq < q; ++qq) {
          const double x = (c + xq[qq]) * g.h;
          const double fv = (f == 0 ? 1.0 : std::sin(M_PI * f * x)) * wq[qq] * g.h;
          lagrange_eval(k, h->tab.z, xq[qq], val);
          for (int i = 0; i <= k; ++i) full[k * c + i] += fv * val[i];
        }
      const double s = t == 0 ? coef[md] : 1.0;
      for (int j = 0; j < ni; ++j) b1d[((size_t)md * h->dim + t) * ni + j] = s * full[j + 1];
    }
  const size_t need = b1d.size() * sizeof(double);
  if (need > h->rhs_cap) {
    if (h->rhs_buf) {
      cudaStreamSynchronize(h->stream);
      cudaFree(h->rhs_buf);
    }
    h->rhs_buf = nullptr;
    h->rhs_cap = 0;
    cudaError_t e = cudaMalloc(&h->rhs_buf, need);
    if (e != cudaSuccess) return fail(h, VPS_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
    h->rhs_cap = need;
  }
  // through pinned staging, so that the copy is asynchronous (a copy from
  // pageable memory would first wait for all earlier work of the stream);
  // the staging is reused once the previous copy out of it has executed
  if (h->rhs_ev) VPS_CK(h, cudaEventSynchronize(h->rhs_ev));
  else VPS_CK(h, cudaEventCreateWithFlags(&h->rhs_ev, cudaEventDisableTiming));
  if (need > h->rhs_host_cap) {
    if (h->rhs_host) cudaFreeHost(h->rhs_host);
    h->rhs_host = nullptr;
    h->rhs_host_cap = 0;
    VPS_CK(h, cudaMallocHost(reinterpret_cast<void**>(&h->rhs_host), need));
    h->rhs_host_cap = need;
  }
  std::memcpy(h->rhs_host, b1d.data(), need);
  VPS_CK(h, cudaMemcpyAsync(h->rhs_buf, h->rhs_host, need, cudaMemcpyHostToDevice, h->stream));
  VPS_CK(h, cudaEventRecord(h->rhs_ev, h->stream));
  VPS_CK(h, launch_rhs_tensor(g, n_modes, h->rhs_buf, b, h->stream));
  return VPS_OK;
}

// One CG iteration's device work after z_new = B r is known (or, for the
// first iteration, after p = z): A p, alpha, x and r updates, r.r, and the
// asynchronous copy of the scalars to the host.
int cg_async_iteration(vps_context* h, bool first) {
  const LevelGeom& g = h->geom[h->L];
  const int64_t n = g.total;
  (void)n;
  if (first) {
    if (int rc = cg_start_direction(h)) return rc;
  } else if (int rc = cg_next_direction(h)) {
    return rc;
  }
  if (int rc = cg_apply_p(h)) return rc;
  if (int rc = cg_step(h)) return rc;
  VPS_CK(h, cudaMemcpyAsync(h->host_sc, h->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost,
                            h->stream));
  VPS_CK(h, cudaMemcpyAsync(h->host_dots, h->dots, sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
  VPS_CK(h, cudaEventRecord(h->as_ev, h->stream));
  return VPS_OK;
}

int cg_async_finish(vps_context* h, int status) {
  const LevelGeom& g = h->geom[h->L];
  const int64_t ni = g.n1 - 2;
  const size_t nbytes = (size_t)(h->dim == 3 ? ni * ni * ni : ni * ni) * sizeof(double);
  h->as_status = status;
  VPS_CK(h, launch_unpack<double>(g, h->cx, h->comp_x, h->stream));
  VPS_CK(h, cudaMemcpyAsync(h->host_x, h->comp_x, nbytes, cudaMemcpyDeviceToHost, h->stream));
  VPS_CK(h, cudaEventRecord(h->as_ev, h->stream));
  h->as_phase = 2;
  return VPS_OK;
}

}  // namespace

namespace vps {

int create_own_stream(int dim, int degree, int level, int precision, vps_handle* out) {
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    set_thread_error(cudaGetErrorString(e));
    return VPS_ECUDA;
  }
  int rc = vps_create(dim, degree, level, precision, VPS_MULTIPLICATIVE, 1.0, 1, 1, s, out);
  if (rc) {
    cudaStreamDestroy(s);
    return rc;
  }
  (*out)->own_stream = true;
  return VPS_OK;
}

size_t estimate_device_bytes(int dim, int degree, int level, int precision) {
  // in floating point: a level too large to address gives SIZE_MAX (it can
  // never fit a budget) instead of a wrapped product
  const double esz = precision == VPS_FP64 ? 8 : 4;
  double total = 0;
  for (int l = 1; l <= level; ++l) total += 3 * level_elements(dim, degree, l) * esz;
  const double elems = level_elements(dim, degree, level);
  const double ni = (double)degree * std::ldexp(1.0, level) - 1.0;
  total += 7 * elems * 8 + 2 * (dim == 3 ? ni * ni * ni : ni * ni) * 8;
  if (precision == VPS_FP32) total += 2 * elems * 4;  // double-float split of p
  for (int l = 1; l <= level; ++l)                     // flags of the dataflow sweep
    total += std::pow(std::ldexp(1.0, l) - 1.0, dim) * 4;
  total += (double)(4 << 20);                         // tables, coarse-level data, scalars
  return total < 1.8e19 ? (size_t)total : SIZE_MAX;
}

// Starts a CG solve of the sine-mode right-hand side on h without waiting.
int cg_async_begin(vps_handle h, int n_modes, const double* coef, const int* freq, double rtol,
                   int max_it) {
  if (int rc = set_device(h)) return rc;
  LaunchTally tally(h);
  const LevelGeom& g = h->geom[h->L];
  const int64_t n = g.total;
  if (!h->as_ev) VPS_CK(h, cudaEventCreateWithFlags(&h->as_ev, cudaEventDisableTiming));
  if (!h->host_x) {
    const int64_t ni = g.n1 - 2;
    VPS_CK(h, cudaMallocHost(&h->host_x, (size_t)(h->dim == 3 ? ni * ni * ni : ni * ni) *
                                              sizeof(double)));
  }
  h->as_rtol = rtol;
  h->as_maxit = max_it;
  h->as_it = 1;
  h->as_rel = 1.0;
  h->as_status = VPS_OK;
  h->as_verify = 0;
  h->as_prev_true = 0.0;
  h->last_restarts = 0;
  h->last_at_floor = 0;
  if (int rc = upload_rhs_sines(h, h->L, n_modes, coef, freq, h->comp_b)) return rc;
  VPS_CK(h, launch_pack<double>(g, h->comp_b, h->cb, h->stream));
  VPS_CK(h, launch_dot1(h->cb, h->cb, n, h->partial, h->dots, h->stream));
  VPS_CK(h, cudaMemsetAsync(h->cx, 0, n * sizeof(double), h->stream));
  VPS_CK(h, cudaMemcpyAsync(h->cr, h->cb, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  VPS_CK(h, cudaMemsetAsync(h->sc, 0, sizeof(CgScalars), h->stream));
  if (h->as_external) {  // the caller runs the first V-cycle, then cg_async_resume
    h->as_need = 3;
    h->as_phase = 1;
    return VPS_OK;
  }
  if (int rc = precondition(h)) return rc;
  if (int rc = cg_async_iteration(h, true)) return rc;
  h->as_phase = 1;
  return VPS_OK;
}

// After the caller's V-cycle (z = B r in xv[L] or czn): the rest of the
// pending iteration of an asynchronous CG with external V-cycles.
int cg_async_resume(vps_handle h) {
  if (!h->as_external || h->as_need == 0) return fail(h, VPS_EINVAL, "no V-cycle pending");
  if (int rc = set_device(h)) return rc;
  LaunchTally tally(h);
  const int need = h->as_need;
  h->as_need = 0;
  if (need == 1) VPS_CK(h, cudaMemsetAsync(h->sc, 0, sizeof(CgScalars), h->stream));
  if (int rc = cg_async_iteration(h, need != 2)) return rc;
  if (need != 3) ++h->as_it;
  return VPS_OK;
}

int cg_async_pending_vcycle(vps_handle h) { return h->as_external && h->as_need != 0; }

// Allocates what asynchronous solves of up to max_modes sine modes use
// (event, pinned result staging, the right-hand side's 1D tables), so that
// cg_async_begin allocates nothing.
int cg_async_prepare(vps_handle h, int max_modes) {
  if (int rc = set_device(h)) return rc;
  const LevelGeom& g = h->geom[h->L];
  const int64_t ni = g.n1 - 2;
  if (!h->as_ev) VPS_CK(h, cudaEventCreateWithFlags(&h->as_ev, cudaEventDisableTiming));
  if (!h->host_x)
    VPS_CK(h, cudaMallocHost(&h->host_x, (size_t)(h->dim == 3 ? ni * ni * ni : ni * ni) *
                                              sizeof(double)));
  const size_t need = (size_t)max_modes * h->dim * ni * sizeof(double);
  if (need > h->rhs_cap) {
    if (h->rhs_buf) {
      cudaStreamSynchronize(h->stream);
      cudaFree(h->rhs_buf);
    }
    h->rhs_buf = nullptr;
    h->rhs_cap = 0;
    VPS_CK(h, cudaMalloc(&h->rhs_buf, need));
    h->rhs_cap = need;
  }
  if (!h->rhs_ev) VPS_CK(h, cudaEventCreateWithFlags(&h->rhs_ev, cudaEventDisableTiming));
  if (need > h->rhs_host_cap) {
    if (h->rhs_host) cudaFreeHost(h->rhs_host);
    h->rhs_host = nullptr;
    h->rhs_host_cap = 0;
    VPS_CK(h, cudaMallocHost(reinterpret_cast<void**>(&h->rhs_host), need));
    h->rhs_host_cap = need;
  }
  return VPS_OK;
}

void set_external_vcycle(vps_handle h, bool on) { h->as_external = on; }

// Advances an asynchronous solve if its pending GPU work has finished.
// *done = 1 when the solution is in host_x (then *status, *iters, *rel).
int cg_async_poll(vps_handle h, int* done, int* status, int* iters, double* rel,
                  const double** x_host) {
  *done = 0;
  if (h->as_phase == 0) return fail(h, VPS_EINVAL, "no solve in flight");
  if (h->as_need) return VPS_OK;  // waiting for the caller's V-cycle
  const cudaError_t q = cudaEventQuery(h->as_ev);
  if (q == cudaErrorNotReady) return VPS_OK;
  if (q != cudaSuccess) return fail(h, VPS_ECUDA, "solve: %s", cudaGetErrorString(q));
  if (int rc = set_device(h)) return rc;
  LaunchTally tally(h);
  if (h->as_phase == 2) {
    h->as_phase = 0;
    *done = 1;
    *status = h->as_status;
    *iters = h->as_it;
    *rel = h->as_rel;
    *x_host = h->host_x;
    return VPS_OK;
  }
  if (h->as_it == 1) h->as_nb = std::sqrt(h->host_dots[0]);
  if (!(h->as_nb > 0.0)) {  // b = 0: x = 0
    h->as_rel = 0.0;
    return cg_async_finish(h, std::isfinite(h->as_nb) ? VPS_OK : VPS_EBREAKDOWN);
  }
  if (h->host_sc->flag) return cg_async_finish(h, VPS_EBREAKDOWN);
  h->as_rel = std::sqrt(h->host_sc->rr) / h->as_nb;
  if (!std::isfinite(h->as_rel)) return cg_async_finish(h, VPS_EBREAKDOWN);
  // the convergence check of cg_solve, one asynchronous step at a time
  bool restart = false;
  if (h->as_verify == 1 && h->as_rel > h->as_rtol &&
      stagnating(h->as_rel, h->as_prev_true)) {  // FP64 residual stopped falling: scale
    if (int rc = cg_residual_scale(h)) return rc;
    VPS_CK(h, cudaMemcpyAsync(h->host_sc, h->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost,
                              h->stream));
    VPS_CK(h, cudaEventRecord(h->as_ev, h->stream));
    h->as_verify = 2;
    h->as_true = h->as_rel;
    return VPS_OK;
  }
  if (h->as_verify) {
    const double rel_true = h->as_verify == 2 ? h->as_true : h->as_rel;
    const double unorm = h->as_verify == 2 ? std::sqrt(h->host_sc->pAp) : -1.0;
    h->as_rel = rel_true;
    h->as_verify = 0;
    const int cls = classify_check(h, h->as_rtol, h->as_nb, rel_true, unorm, h->as_prev_true);
    if (cls == kCheckConverged) return cg_async_finish(h, VPS_OK);
    if (cls == kCheckStagnated) return cg_async_finish(h, VPS_ENOCONV);
    h->as_prev_true = rel_true;
    ++h->last_restarts;
    restart = true;
  } else if (h->as_rel <= h->as_rtol) {
    // confirm on the FP64 residual r = b - A x (see cg_solve)
    if (int rc = cg_true_residual(h)) return rc;
    VPS_CK(h, cudaMemcpyAsync(h->host_sc, h->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost,
                              h->stream));
    VPS_CK(h, cudaEventRecord(h->as_ev, h->stream));
    h->as_verify = 1;
    return VPS_OK;
  }
  if (h->as_it >= h->as_maxit) return cg_async_finish(h, VPS_ENOCONV);
  if (h->as_external) {  // the caller runs the V-cycle, then cg_async_resume
    h->as_need = restart ? 1 : 2;
    return VPS_OK;
  }
  if (int rc = precondition(h)) return rc;
  if (restart) {  // from the FP64 residual, which is still above the tolerance
    VPS_CK(h, cudaMemsetAsync(h->sc, 0, sizeof(CgScalars), h->stream));
    if (int rc = cg_async_iteration(h, true)) return rc;
  } else if (int rc = cg_async_iteration(h, false)) {
    return rc;
  }
  ++h->as_it;
  return VPS_OK;
}


namespace {

// Host side of one cohort V-cycle's queues: packed one after another in a
// pinned staging buffer, copied to the device in one transfer before the
// launches that read them.
struct QueueWriter {
  unsigned char* host;
  unsigned char* dev;
  size_t cap, used = 0;
  int64_t launches = 0;
  int max_items = 0;
  BatchQueue* open(size_t* off) {
    const size_t sz = sizeof(BatchQueue);
    if (used + sz > cap) return nullptr;
    *off = used;
    BatchQueue* q = reinterpret_cast<BatchQueue*>(host + used);
    q->head = 0;
    q->ntiles = 0;
    q->nitems = 0;
    q->pad_ = 0;
    return q;
  }
  // closes queue q at offset off: only its header and nitems items are kept
  void close(BatchQueue* q, size_t off) {
    const size_t sz = offsetof(BatchQueue, items) + (size_t)q->nitems * sizeof(BatchItem);
    used = off + (sz + 255) / 256 * 256;
    max_items = std::max(max_items, q->nitems);
  }
  BatchQueue* dev_at(size_t off) const { return reinterpret_cast<BatchQueue*>(dev + off); }
};

// One recorded batched launch: kind 0 colour pass (variant v), 1
// restriction (+ zeroed upper faces), 2 prolongation; or a per-member step
// (kind 3 memset of x, 4 residual, 5 coarse solve, 6 FP32 cast) of member m
// on level l.
struct CohortOp {
  int kind, v, m, l;
  size_t off;
  int64_t ntiles;
  int nitems;
};

template <typename T>
int cohort_vcycle_t(vps_context* const* hs, int n, QueueWriter* qw, cudaStream_t st) {
  vps_context* h0 = hs[0];
  const KernelFns<T>& F = fns<T>(h0);
  const int nc = 1 << h0->dim;
  std::vector<const T*> bL(n);
  std::vector<T*> xL(n);
  for (int m = 0; m < n; ++m) {
    vps_context* h = hs[m];
    if (h->prec == VPS_FP64) {
      bL[m] = reinterpret_cast<const T*>(h->cr);
      xL[m] = reinterpret_cast<T*>(h->czn);
    } else {
      bL[m] = static_cast<const T*>(h->bv[h->L]);
      xL[m] = static_cast<T*>(h->xv[h->L]);
    }
  }
  auto bptr = [&](int m, int l) -> const T* {
    return l == hs[m]->L ? bL[m] : static_cast<const T*>(hs[m]->bv[l]);
  };
  auto xptr = [&](int m, int l) -> T* {
    return l == hs[m]->L ? xL[m] : static_cast<T*>(hs[m]->xv[l]);
  };
  int D = 0;
  for (int m = 0; m < n; ++m) D = std::max(D, hs[m]->L - hs[m]->coarse);
  // record the whole cycle first (queues into the staging buffer), then copy
  // the queues and issue the launches in the recorded order
  std::vector<CohortOp> ops;
  auto fail_all = [&](const char* msg) { return fail(h0, VPS_ENOMEM, "%s", msg); };
  auto colour_ops = [&](const std::vector<int>& act, const std::vector<int>& lev, int c) -> int {
    // one launch per smoother variant present among the members
    std::vector<int> vs;
    for (size_t i = 0; i < act.size(); ++i) {
      const int v = hs[act[i]]->smooth_var[lev[i]];
      if (std::find(vs.begin(), vs.end(), v) == vs.end()) vs.push_back(v);
    }
    for (int v : vs) {
      if (v < 0 || v >= kSmoothVariants || !F.smooth_mult_batch_v[v])
        return fail(h0, VPS_EINVAL, "smoother variant %d has no batched kernel", v);
      size_t off;
      BatchQueue* q = qw->open(&off);
      if (!q) return fail_all("cohort queue buffer full");
      const int P = F.variant_p[v];
      for (size_t i = 0; i < act.size(); ++i) {
        const int m = act[i], l = lev[i];
        if (hs[m]->smooth_var[l] != v) continue;
        const LevelGeom& g = hs[m]->geom[l];
        const ColourGeom cg = make_colour(g, c);
        if (cg.npatch == 0) continue;
        if (q->nitems == kMaxBatch) return fail_all("cohort larger than a queue");
        BatchItem& it = q->items[q->nitems++];
        it = BatchItem();
        it.in = bptr(m, l);
        it.out = xptr(m, l);
        it.tile0 = q->ntiles;
        it.n1a = g.n1;
        it.pxa = g.px;
        it.pza = g.pz;
        it.cg = cg;
        it.bscale = h0->dim == 3 ? 1.0 / g.h : 1.0;
        q->ntiles += (cg.npatch + P - 1) / P;
      }
      qw->close(q, off);
      ops.push_back({0, v, -1, c, off, q->ntiles, q->nitems});
    }
    return VPS_OK;
  };
  auto transfer_op = [&](int kind, const std::vector<int>& act, const std::vector<int>& lev) -> int {
    size_t off;
    BatchQueue* q = qw->open(&off);
    if (!q) return fail_all("cohort queue buffer full");
    for (size_t i = 0; i < act.size(); ++i) {
      const int m = act[i], l = lev[i];  // l: the fine level
      const LevelGeom& f = hs[m]->geom[l];
      const LevelGeom& c = hs[m]->geom[l - 1];
      if (q->nitems == kMaxBatch) return fail_all("cohort larger than a queue");
      BatchItem& it = q->items[q->nitems++];
      it = BatchItem();
      if (kind == 1) {
        it.in = hs[m]->rv[l];
        it.out = const_cast<T*>(bptr(m, l - 1));
      } else {
        it.in = xptr(m, l - 1);
        it.out = xptr(m, l);
      }
      it.tile0 = q->ntiles;
      it.n1a = c.n1;
      it.pxa = c.px;
      it.pza = c.pz;
      it.n1b = f.n1;
      it.pxb = f.px;
      it.pzb = f.pz;
      const int t = (c.ncell + F.transfer_cells - 1) / F.transfer_cells;
      it.tiles_per_dim = t;
      q->ntiles += h0->dim == 3 ? (int64_t)t * t * t : (int64_t)t * t;
    }
    qw->close(q, off);
    ops.push_back({kind, 0, -1, 0, off, q->ntiles, q->nitems});
    return VPS_OK;
  };
  // members whose top level is their coarse level: the cycle is the exact solve
  for (int m = 0; m < n; ++m)
    if (hs[m]->L == hs[m]->coarse) ops.push_back({5, 0, m, hs[m]->L, 0, 0, 0});
  for (int s = 0; s < D; ++s) {  // descent
    std::vector<int> act, lev;
    for (int m = 0; m < n; ++m)
      if (hs[m]->L - s > hs[m]->coarse) {
        act.push_back(m);
        lev.push_back(hs[m]->L - s);
      }
    for (size_t i = 0; i < act.size(); ++i) ops.push_back({3, 0, act[i], lev[i], 0, 0, 0});
    for (int p = 0; p < h0->n_pre; ++p)
      for (int c = 0; c < nc; ++c)
        if (int rc = colour_ops(act, lev, c)) return rc;
    for (size_t i = 0; i < act.size(); ++i) ops.push_back({4, 0, act[i], lev[i], 0, 0, 0});
    if (int rc = transfer_op(1, act, lev)) return rc;
    for (size_t i = 0; i < act.size(); ++i)
      if (lev[i] - 1 == hs[act[i]]->coarse) ops.push_back({5, 0, act[i], lev[i] - 1, 0, 0, 0});
  }
  for (int s = D - 1; s >= 0; --s) {  // ascent
    std::vector<int> act, lev;
    for (int m = 0; m < n; ++m)
      if (hs[m]->L - s > hs[m]->coarse) {
        act.push_back(m);
        lev.push_back(hs[m]->L - s);
      }
    if (int rc = transfer_op(2, act, lev)) return rc;
    for (int p = 0; p < h0->n_post; ++p)
      for (int i = 0; i < nc; ++i)  // reverse colour order: the symmetric cycle of the CG
        if (int rc = colour_ops(act, lev, nc - 1 - i)) return rc;
  }
  // issue
  VPS_CK(h0, cudaMemcpyAsync(qw->dev, qw->host, qw->used, cudaMemcpyHostToDevice, st));
  for (int m = 0; m < n; ++m)
    if (hs[m]->prec == VPS_FP32)
      VPS_CK(h0, launch_cast_d2f(hs[m]->cr, static_cast<float*>(hs[m]->bv[hs[m]->L]),
                                 hs[m]->geom[hs[m]->L].total, st));
  const T* il = static_cast<const T*>(h0->inv_lam);
  for (const CohortOp& op : ops) {
    switch (op.kind) {
      case 0:
        VPS_CK(h0, F.smooth_mult_batch_v[op.v](qw->dev_at(op.off), op.ntiles, il, st));
        ++qw->launches;
        break;
      case 1:
        VPS_CK(h0, F.restrict_batch(qw->dev_at(op.off), op.ntiles, st));
        VPS_CK(h0, F.zero_faces_batch(qw->dev_at(op.off), op.nitems, st));
        qw->launches += 2;
        break;
      case 2:
        VPS_CK(h0, F.prolong_batch(qw->dev_at(op.off), op.ntiles, st));
        ++qw->launches;
        break;
      case 3:
        VPS_CK(h0, cudaMemsetAsync(xptr(op.m, op.l), 0, hs[op.m]->geom[op.l].total * sizeof(T), st));
        break;
      case 4: {
        vps_context* h = hs[op.m];
        VPS_CK(h0, level_apply<T>(h, op.l, xptr(op.m, op.l), bptr(op.m, op.l),
                                  static_cast<T*>(h->rv[op.l])));
        break;
      }
      case 5:
        if (int rc = coarse_solve<T>(hs[op.m], bptr(op.m, op.l), xptr(op.m, op.l))) return rc;
        break;
    }
  }
  return VPS_OK;
}

}  // namespace

int cohort_vcycle(vps_context* const* hs, int n, void* q_host, void* q_dev, size_t q_cap,
                  int64_t* batched_launches, int* max_items) {
  if (n <= 0) return VPS_OK;
  vps_context* h0 = hs[0];
  for (int m = 0; m < n; ++m) {
    vps_context* h = hs[m];
    if (h->dim != h0->dim || h->k != h0->k || h->prec != h0->prec || h->stream != h0->stream ||
        h->n_pre != h0->n_pre || h->n_post != h0->n_post || h->smoother != VPS_MULTIPLICATIVE ||
        h->kernel_kind != VPS_KERNEL_FUSED || !h->as_external || h->as_need == 0)
      return fail(h0, VPS_EINVAL, "cohort members must share shape, precision and stream");
  }
  if (n > kMaxBatch) return fail(h0, VPS_EINVAL, "at most %d cohort members", kMaxBatch);
  if (int rc = set_device(h0)) return rc;
  LaunchTally tally(h0);
  QueueWriter qw{static_cast<unsigned char*>(q_host), static_cast<unsigned char*>(q_dev), q_cap};
  const int rc = h0->prec == VPS_FP64 ? cohort_vcycle_t<double>(hs, n, &qw, h0->stream)
                                      : cohort_vcycle_t<float>(hs, n, &qw, h0->stream);
  if (batched_launches) *batched_launches += qw.launches;
  if (max_items) *max_items = std::max(*max_items, qw.max_items);
  return rc;
}

const char* handle_error(vps_handle h) { return h ? h->err.c_str() : ""; }

}  // namespace vps

namespace {

bool variant_ok(vps_context* h, int v) {
  if (v < 0 || v >= kSmoothVariants) return false;
  return h->prec == VPS_FP64 ? (h->smoother == VPS_ADDITIVE ? h->ks->d.smooth_add_v[v] != nullptr
                                                            : h->ks->d.smooth_mult_v[v] != nullptr)
                             : (h->smoother == VPS_ADDITIVE ? h->ks->f.smooth_add_v[v] != nullptr
                                                            : h->ks->f.smooth_mult_v[v] != nullptr);
}

// Mean time (ms) of `reps` calls of fn on the handle's stream.
template <typename F>
int time_ms(vps_context* h, int reps, F fn, float* ms) {
  cudaEvent_t a, b;
  VPS_CK(h, cudaEventCreate(&a));
  VPS_CK(h, cudaEventCreate(&b));
  int rc = fn();  // warm-up
  if (!rc) {
    cudaEventRecord(a, h->stream);
    for (int i = 0; i < reps && !rc; ++i) rc = fn();
    cudaEventRecord(b, h->stream);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(ms, a, b);
    *ms /= reps;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc;
}

std::string tune_key(vps_context* h) {
  char key[96];
  std::snprintf(key, sizeof(key), "d%d_k%d_%s_%s_L%d_pre%d_post%d", h->dim, h->k,
                h->prec == VPS_FP64 ? "fp64" : "fp32",
                h->smoother == VPS_ADDITIVE ? "add" : "mult", h->L, h->n_pre, h->n_post);
  return key;
}

// Cache file: one JSON object, one entry per line:
//   "d3_k4_fp32_mult_L5_pre1_post1": {"coarse": 3, "variants": [1, 1, 2, 0, 1],
//                                     "ops": [0, 0, 1, 1, 0], "schedule": 1,
//                                     "coarse_solver": 1},
// (one line each).  Entries without every field are tuned again.
bool parse_list(const char* p, const char* name, int* out, int nvar) {
  const char* v = std::strstr(p, name);
  if (!v) return false;
  v += std::strlen(name);
  int i = 0;
  while (i < nvar && *v && *v != ']') {
    while (*v == ' ' || *v == ',') ++v;
    if (*v == ']' || !*v) break;
    out[i++] = std::atoi(v);
    while (*v && *v != ',' && *v != ']') ++v;
  }
  return i == nvar;
}

bool cache_lookup(const char* path, const std::string& key, int* coarse, int* var, int* ops,
                  int* schedule, int* coarse_solver, int nvar) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[2048];
  bool found = false;
  const std::string pat = "\"" + key + "\"";
  while (std::fgets(line, sizeof(line), f)) {
    const char* p = std::strstr(line, pat.c_str());
    if (!p) continue;
    const char* c = std::strstr(p, "\"coarse\":");
    const char* d = std::strstr(p, "\"schedule\":");
    const char* cs = std::strstr(p, "\"coarse_solver\":");
    if (!c || !d || !cs) continue;
    *coarse_solver = std::atoi(cs + 16);
    *coarse = std::atoi(c + 9);
    *schedule = std::atoi(d + 11);
    found = parse_list(p, "\"variants\": [", var, nvar) && parse_list(p, "\"ops\": [", ops, nvar);
  }
  std::fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, int coarse, const int* var,
                 const int* ops, int schedule, int coarse_solver, int nvar) {
  std::vector<std::string> keep;
  if (FILE* f = std::fopen(path, "r")) {
    char line[2048];
    const std::string pat = "\"" + key + "\"";
    while (std::fgets(line, sizeof(line), f)) {
      std::string sline(line);
      if (sline.find("\": {\"coarse\":") == std::string::npos) continue;
      if (sline.find(pat) != std::string::npos) continue;
      while (!sline.empty() && (sline.back() == '\n' || sline.back() == ',')) sline.pop_back();
      keep.push_back(sline);
    }
    std::fclose(f);
  }
  std::string entry = "\"" + key + "\": {\"coarse\": " + std::to_string(coarse) + ", \"variants\": [";
  for (int i = 0; i < nvar; ++i) entry += (i ? ", " : "") + std::to_string(var[i]);
  entry += "], \"ops\": [";
  for (int i = 0; i < nvar; ++i) entry += (i ? ", " : "") + std::to_string(ops[i]);
  entry += "], \"schedule\": " + std::to_string(schedule) +
           ", \"coarse_solver\": " + std::to_string(coarse_solver) + "}";
  keep.push_back(entry);
  if (FILE* f = std::fopen(path, "w")) {
    std::fputs("{\n", f);
    for (size_t i = 0; i < keep.size(); ++i)
      std::fprintf(f, "%s%s\n", keep[i].c_str(), i + 1 < keep.size() ? "," : "");
    std::fputs("}\n", f);
    std::fclose(f);
  }
}

// One CG solve of a smooth right-hand side on the handle's buffers (timing
// trials of the autotuner).
int trial_solve(vps_context* h) {
  const LevelGeom& g = h->geom[h->L];
  VPS_CK(h, launch_pack<double>(g, h->comp_b, h->cb, h->stream));
  int it = 0;
  double rel = 0;
  return cg_solve(h, 1e-10, 200, &it, &rel);
}

}  // namespace

extern "C" {

const char* vps_status_string(int s) {
  switch (s) {
    case VPS_OK: return "VPS_OK";
    case VPS_EINVAL: return "VPS_EINVAL";
    case VPS_ENOMEM: return "VPS_ENOMEM";
    case VPS_ECUDA: return "VPS_ECUDA";
    case VPS_ENOCONV: return "VPS_ENOCONV";
    case VPS_EBREAKDOWN: return "VPS_EBREAKDOWN";
    case VPS_ETIMEOUT: return "VPS_ETIMEOUT";
    default: return "unknown status";
  }
}

const char* vps_last_error(vps_handle h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

int vps_create(int dim, int degree, int level, int precision, int smoother, double damping,
               int n_pre, int n_post, void* cuda_stream, vps_handle* out) {
  g_create_error.clear();
  if (!out) return fail(nullptr, VPS_EINVAL, "out is NULL");
  *out = nullptr;
  if (dim != 2 && dim != 3) return fail(nullptr, VPS_EINVAL, "dim must be 2 or 3 (got %d)", dim);
  if (degree < 1 || degree > VPS_MAX_DEGREE)
    return fail(nullptr, VPS_EINVAL, "degree must be 1..%d (got %d)", VPS_MAX_DEGREE, degree);
  if (level < 1 || level > kMaxLevels) return fail(nullptr, VPS_EINVAL, "level must be >= 1");
  if (precision != VPS_FP64 && precision != VPS_FP32)
    return fail(nullptr, VPS_EINVAL, "precision must be VPS_FP64 or VPS_FP32");
  if (smoother != VPS_MULTIPLICATIVE && smoother != VPS_ADDITIVE)
    return fail(nullptr, VPS_EINVAL, "smoother must be VPS_MULTIPLICATIVE or VPS_ADDITIVE");
  if (!(damping > 0.0) || !std::isfinite(damping))
    return fail(nullptr, VPS_EINVAL, "damping must be positive and finite");
  if (n_pre < 0 || n_post < 0 || n_pre > 64 || n_post > 64)
    return fail(nullptr, VPS_EINVAL, "n_pre/n_post must be 0..64");
  {
    const double elems = level_elements(dim, degree, level);
    if (!(elems <= 2147483647.0))
      return fail(nullptr, VPS_EINVAL, "level %d too large: %.4g elements per vector", level,
                  elems);
  }
  register_all();
  vps_context* h = new vps_context();
  h->dim = dim; h->k = degree; h->L = level; h->prec = precision; h->smoother = smoother;
  h->damping = damping; h->n_pre = n_pre; h->n_post = n_post;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->use_graphs = h->stream != nullptr;
  h->esz = precision == VPS_FP64 ? sizeof(double) : sizeof(float);
  char ebuf[256];
  if (!build_tables(degree, &h->tab, ebuf, sizeof(ebuf))) {
    delete h;
    return fail(nullptr, VPS_EINVAL, "%s", ebuf);
  }
  h->ks = kernel_registry(dim, degree);
  if (!h->ks || !h->ks->present) {
    delete h;
    return fail(nullptr, VPS_EINVAL, "no kernels for dim %d degree %d", dim, degree);
  }
  auto bail = [&](int rc) {
    g_create_error = h->err;
    vps_destroy(h);
    return rc;
  };
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    h->err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return bail(VPS_ECUDA);
  }
  if (h->device < 0 || h->device >= kMaxDevices) {
    h->err = "device index out of range";
    return bail(VPS_ECUDA);
  }
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    bool& up = g_uploaded[h->device][dim - 2][degree - 1];
    if (!up) {
      e = h->ks->upload(h->tab);
      if (e != cudaSuccess) {
        h->err = std::string("constant upload: ") + cudaGetErrorString(e);
        return bail(VPS_ECUDA);
      }
      up = true;
    }
  }
  int rc;
  // default variant before tuning: the Boundary kernel of block shape 0 for
  // the multiplicative smoother, else the fused one; shape 0 for the additive
  const int prefer[2][4] = {{3, 4, 0, 1}, {0, 1, 0, 1}};
  int def_var = 0;
  for (int v : prefer[smoother == VPS_ADDITIVE ? 1 : 0])
    if (variant_ok(h, v)) {
      def_var = v;
      break;
    }
  for (int l = 1; l <= level; ++l) {
    h->smooth_var[l] = def_var;
    h->geom[l] = make_geom(dim, degree, l);
    const size_t vb = (size_t)h->geom[l].total * h->esz;
    if ((rc = dalloc(h, &h->bv[l], vb)) || (rc = dalloc(h, &h->xv[l], vb)) ||
        (rc = dalloc(h, &h->rv[l], vb)))
      return bail(rc);
    // one flag per vertex patch of the level for the dataflow sweep
    const int64_t nv = h->geom[l].ncell - 1;
    void* fl = nullptr;
    if ((rc = dalloc(h, &fl, (size_t)(dim == 3 ? nv * nv * nv : nv * nv) * sizeof(unsigned))))
      return bail(rc);
    h->sweep_flags[l] = static_cast<unsigned int*>(fl);
  }
  {
    void* q = nullptr;
    if ((rc = dalloc(h, &q, (kMaxLevels + 1) * sizeof(SweepCounters)))) return bail(rc);
    h->sweep_ctr = static_cast<SweepCounters*>(q);
    if ((rc = dalloc(h, &q, sizeof(int)))) return bail(rc);
    h->wait_err = static_cast<int*>(q);
    if ((rc = dalloc(h, &q, 2 * sizeof(unsigned)))) return bail(rc);
    h->gsync = static_cast<unsigned*>(q);
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device) == cudaSuccess)
      h->coop_ok = h->coarse_coop = coop != 0;
  }
  // 1/(lambda_i + lambda_j [+ lambda_l]) in reference units
  {
    const int m = h->tab.m;
    const int md = dim == 3 ? m * m * m : m * m;
    std::vector<double> il(md);
    for (int a = 0; a < md; ++a) {
      const int i0 = a % m, i1 = (a / m) % m, i2 = a / (m * m);
      double s = h->tab.lam[i0] + h->tab.lam[i1] + (dim == 3 ? h->tab.lam[i2] : 0.0);
      il[a] = 1.0 / s;
    }
    if ((rc = dalloc(h, &h->inv_lam, md * h->esz))) return bail(rc);
    if (precision == VPS_FP64) {
      e = cudaMemcpyAsync(h->inv_lam, il.data(), md * sizeof(double), cudaMemcpyHostToDevice,
                          h->stream);
    } else {
      std::vector<float> f(il.begin(), il.end());
      e = cudaMemcpyAsync(h->inv_lam, f.data(), md * sizeof(float), cudaMemcpyHostToDevice,
                          h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    if (e != cudaSuccess) {
      h->err = std::string("cudaMemcpy: ") + cudaGetErrorString(e);
      return bail(VPS_ECUDA);
    }
  }
  const LevelGeom& gf = h->geom[level];
  const size_t db = (size_t)gf.total * sizeof(double);
  const int64_t ni = gf.n1 - 2;
  const size_t cbytes = (size_t)(dim == 3 ? ni * ni * ni : ni * ni) * sizeof(double);
  void* p;
  if ((rc = dalloc(h, &p, db))) return bail(rc); h->cb = (double*)p;
  if ((rc = dalloc(h, &p, db))) return bail(rc); h->cx = (double*)p;
  if ((rc = dalloc(h, &p, db))) return bail(rc); h->cr = (double*)p;
  if ((rc = dalloc(h, &p, db))) return bail(rc); h->cp = (double*)p;
  if ((rc = dalloc(h, &p, db))) return bail(rc); h->cz = (double*)p;
  if ((rc = dalloc(h, &p, db))) return bail(rc); h->czn = (double*)p;
  if ((rc = dalloc(h, &p, db))) return bail(rc); h->cAp = (double*)p;
  if (precision == VPS_FP32) {
    if ((rc = vps_set_outer_operator(h, VPS_OUTER_DOUBLE_FLOAT))) return bail(rc);
  }
  if ((rc = dalloc(h, &p, cbytes))) return bail(rc); h->comp_b = (double*)p;
  if ((rc = dalloc(h, &p, cbytes))) return bail(rc); h->comp_x = (double*)p;
  if ((rc = dalloc(h, &p, 2 * kDotBlocks * sizeof(double)))) return bail(rc); h->partial = (double*)p;
  if ((rc = dalloc(h, &p, 2 * kDotBlocks * sizeof(double)))) return bail(rc); h->partial2 = (double*)p;
  if ((rc = dalloc(h, &p, 8 * sizeof(double)))) return bail(rc); h->dots = (double*)p;
  if ((rc = dalloc(h, &p, sizeof(CgScalars)))) return bail(rc); h->sc = (CgScalars*)p;
  if ((rc = dalloc(h, &p, 256 * sizeof(double)))) return bail(rc); h->l2_tab = (double*)p;
  if ((rc = setup_coarse(h, auto_coarse_level(degree, level)))) return bail(rc);
  e = cudaMallocHost(&p, sizeof(CgScalars));
  if (e != cudaSuccess) { h->err = "cudaMallocHost failed"; return bail(VPS_ENOMEM); }
  h->host_sc = (CgScalars*)p;
  e = cudaMallocHost(&p, 8 * sizeof(double));
  if (e != cudaSuccess) { h->err = "cudaMallocHost failed"; return bail(VPS_ENOMEM); }
  h->host_dots = (double*)p;
  e = cudaMallocHost(&p, sizeof(int));
  if (e != cudaSuccess) { h->err = "cudaMallocHost failed"; return bail(VPS_ENOMEM); }
  h->host_err = (int*)p;
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    h->err = std::string("create: ") + cudaGetErrorString(e);
    return bail(VPS_ECUDA);
  }
  *out = h;
  return VPS_OK;
}

int vps_destroy(vps_handle h) {
  if (!h) return VPS_OK;
  if (h->device >= 0) cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  drop_graphs(h);
  for (void* p : h->allocs) cudaFree(p);
  if (h->gm_host) cudaFreeHost(h->gm_host);
  if (h->host_sc) cudaFreeHost(h->host_sc);
  if (h->host_dots) cudaFreeHost(h->host_dots);
  if (h->host_err) cudaFreeHost(h->host_err);
  if (h->host_x) cudaFreeHost(h->host_x);
  if (h->as_ev) cudaEventDestroy(h->as_ev);
  if (h->rhs_buf) cudaFree(h->rhs_buf);
  if (h->rhs_host) cudaFreeHost(h->rhs_host);
  if (h->rhs_ev) cudaEventDestroy(h->rhs_ev);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return VPS_OK;
}

int vps_sizes(vps_handle h, int64_t* n_interior, int64_t* n_patches, size_t* device_bytes) {
  if (!h) return VPS_EINVAL;
  const LevelGeom& g = h->geom[h->L];
  const int64_t ni = g.n1 - 2, nv = g.ncell - 1;
  if (n_interior) *n_interior = h->dim == 3 ? ni * ni * ni : ni * ni;
  if (n_patches) *n_patches = h->dim == 3 ? nv * nv * nv : nv * nv;
  if (device_bytes) *device_bytes = h->bytes;
  return VPS_OK;
}

int vps_level_layout(vps_handle h, int level, int64_t* n1, int64_t* row_pitch, int64_t* total) {
  if (!h) return VPS_EINVAL;
  if (int rc = check_level(h, level, 1)) return rc;
  const LevelGeom& g = h->geom[level];
  if (n1) *n1 = g.n1;
  if (row_pitch) *row_pitch = g.px;
  if (total) *total = g.total;
  return VPS_OK;
}

int vps_pack(vps_handle h, int level, const void* compact, void* lev) {
  if (!h || !compact || !lev) return h ? fail(h, VPS_EINVAL, "NULL vector") : VPS_EINVAL;
  if (int rc = check_level(h, level, 1)) return rc;
  if (int rc = set_device(h)) return rc;
  LaunchTally tally(h);
  if (h->prec == VPS_FP64)
    VPS_CK(h, launch_pack<double>(h->geom[level], (const double*)compact, (double*)lev, h->stream));
  else
    VPS_CK(h, launch_pack<float>(h->geom[level], (const float*)compact, (float*)lev, h->stream));
  return VPS_OK;
}

int vps_unpack(vps_handle h, int level, const void* lev, void* compact) {
  if (!h || !compact || !lev) return h ? fail(h, VPS_EINVAL, "NULL vector") : VPS_EINVAL;
  if (int rc = check_level(h, level, 1)) return rc;
  if (int rc = set_device(h)) return rc;
  LaunchTally tally(h);
  if (h->prec == VPS_FP64)
    VPS_CK(h, launch_unpack<double>(h->geom[level], (const double*)lev, (double*)compact, h->stream));
  else
    VPS_CK(h, launch_unpack<float>(h->geom[level], (const float*)lev, (float*)compact, h->stream));
  return VPS_OK;
}

int vps_smooth(vps_handle h, int level, const void* b, void* x, int n_steps) {
  if (!h) return VPS_EINVAL;
  if (!b || !x || b == x) return fail(h, VPS_EINVAL, "b and x must be distinct non-NULL vectors");
  if (n_steps < 0) return fail(h, VPS_EINVAL, "n_steps < 0");
  if (int rc = check_level(h, level, 2)) return rc;
  if (int rc = set_device(h)) return rc;
  LaunchTally tally(h);
  for (int s = 0; s < n_steps; ++s) {
    int rc = h->prec == VPS_FP64
                 ? smooth_step<double>(h, level, (const double*)b, (double*)x, true)
                 : smooth_step<float>(h, level, (const float*)b, (float*)x, true);
    if (rc) return rc;
  }
  return VPS_OK;
}

int vps_smooth_colour(vps_handle h, int level, int colour, const void* b, void* x) {
  if (!h) return VPS_EINVAL;
  if (!b || !x || b == x) return fail(h, VPS_EINVAL, "b and x must be distinct non-NULL vectors");
  if (int rc = check_level(h, level, 1)) return rc;
  if (colour < 0 || colour >= (1 << h->dim)) return fail(h, VPS_EINVAL, "colour out of range");
  if (int rc = set_device(h)) return rc;
  LaunchTally tally(h);
  const int v = h->smooth_var[level];
  if (!variant_ok(h, v)) return fail(h, VPS_EINVAL, "smoother variant %d unavailable", v);
  if (h->prec == VPS_FP64) return colour_pass<double>(h, level, colour, (const double*)b, (double*)x);
  return colour_pass<float>(h, level, colour, (const float*)b, (float*)x);
}

int vps_apply(vps_handle h, int level, const void* x, void* y) {
  if (!h) return VPS_EINVAL;
  if (!x || !y || x == y) return fail(h, VPS_EINVAL, "x and y must be distinct non-NULL vectors");
  if (int rc = check_level(h, level, 1)) return rc;
  if (int rc = set_device(h)) return rc;
  LaunchTally tally(h);
  const LevelGeom& g = h->geom[level];
  if (h->prec == VPS_FP64)
    VPS_CK(h, h->ks->d.apply(g, (const double*)x, nullptr, (double*)y, h->stream));
  else
    VPS_CK(h, h->ks->f.apply(g, (const float*)x, nullptr, (float*)y, h->stream));
  return VPS_OK;
}

int vps_apply_outer(vps_handle h, const double* x, double* y) {
  if (!h) return VPS_EINVAL;
  if (!x || !y || x == y) return fail(h, VPS_EINVAL, "x and y must be distinct non-NULL vectors");
  if (int rc = set_device(h)) return rc;
  LaunchTally tally(h);
  const LevelGeom& g = h->geom[h->L];
  if (!outer_df(h)) {
    VPS_CK(h, h->ks->d.apply(g, x, nullptr, y, h->stream));
    return VPS_OK;
  }
  VPS_CK(h, launch_split_df(x, h->cph, h->cpl, g.total, h->stream));
  VPS_CK(h, h->ks->apply_df(g, h->cph, h->cpl, y, h->stream));
  return VPS_OK;
}

int vps_restrict(vps_handle h, int fine_level, const void* rf, void* rc_) {
  if (!h) return VPS_EINVAL;
  if (!rf || !rc_ || rf == rc_) return fail(h, VPS_EINVAL, "bad vectors");
  if (int rc = check_level(h, fine_level, 2)) return rc;
  if (int rc = set_device(h)) return rc;
  LaunchTally tally(h);
  const LevelGeom &f = h->geom[fine_level], &c = h->geom[fine_level - 1];
  if (h->prec == VPS_FP64)
    VPS_CK(h, h->ks->d.restrict_(f, c, (const double*)rf, (double*)rc_, h->stream));
  else
    VPS_CK(h, h->ks->f.restrict_(f, c, (const float*)rf, (float*)rc_, h->stream));
  return VPS_OK;
}

int vps_prolongate_add(vps_handle h, int fine_level, const void* xc, void* xf) {
  if (!h) return VPS_EINVAL;
  if (!xc || !xf || xc == xf) return fail(h, VPS_EINVAL, "bad vectors");
  if (int rc = check_level(h, fine_level, 2)) return rc;
  if (int rc = set_device(h)) return rc;
  LaunchTally tally(h);
  const LevelGeom &f = h->geom[fine_level], &c = h->geom[fine_level - 1];
  if (h->prec == VPS_FP64)
    VPS_CK(h, h->ks->d.prolong_add(f, c, (const double*)xc, (double*)xf, h->stream));
  else
    VPS_CK(h, h->ks->f.prolong_add(f, c, (const float*)xc, (float*)xf, h->stream));
  return VPS_OK;
}

int vps_vcycle(vps_handle h, const void* b, void* x) {
  if (!h) return VPS_EINVAL;
  if (!b || !x || b == x) return fail(h, VPS_EINVAL, "b and x must be distinct non-NULL vectors");
  if (int rc = set_device(h)) return rc;
  LaunchTally tally(h);
  return h->prec == VPS_FP64 ? vcycle_core<double>(h, (const double*)b, (double*)x)
                             : vcycle_core<float>(h, (const float*)b, (float*)x);
}

int vps_solve(vps_handle h, const double* b, double* x, double rtol, int max_it, int* iters,
              double* rel_res) {
  if (!h) return VPS_EINVAL;
  if (!b || !x) return fail(h, VPS_EINVAL, "NULL vector");
  if (!(rtol > 0.0) || max_it < 1) return fail(h, VPS_EINVAL, "need rtol > 0 and max_it >= 1");
  if (int rc = set_device(h)) return rc;
  LaunchTally tally(h);
  const LevelGeom& g = h->geom[h->L];
  VPS_CK(h, launch_pack<double>(g, b, h->cb, h->stream));
  int rc = cg_solve(h, rtol, max_it, iters, rel_res);
  cudaError_t e = launch_unpack<double>(g, h->cx, x, h->stream);
  if (rc) return rc;
  if (e != cudaSuccess) return fail(h, VPS_ECUDA, "unpack: %s", cudaGetErrorString(e));
  return VPS_OK;
}

int vps_gmres(vps_handle h, const double* b, double* x, double rtol, int restart, int max_it,
              int* iters, double* rel_res) {
  if (!h) return VPS_EINVAL;
  if (!b || !x) return fail(h, VPS_EINVAL, "NULL vector");
  if (!(rtol > 0.0) || max_it < 1) return fail(h, VPS_EINVAL, "need rtol > 0 and max_it >= 1");
  if (restart < 1 || restart > 512) return fail(h, VPS_EINVAL, "restart must be in 1..512");
  if (int rc = set_device(h)) return rc;
  LaunchTally tally(h);
  const LevelGeom& g = h->geom[h->L];
  VPS_CK(h, launch_pack<double>(g, b, h->cb, h->stream));
  int rc = gmres_solve(h, restart, rtol, max_it, iters, rel_res);
  cudaError_t e = launch_unpack<double>(g, h->cx, x, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (rc) return rc;
  if (e != cudaSuccess) return fail(h, VPS_ECUDA, "unpack: %s", cudaGetErrorString(e));
  return check_waits(h);
}

int vps_solve_host(vps_handle h, const double* b_host, double* x_host, double rtol, int max_it,
                   int* iters, double* rel_res) {
  if (!h) return VPS_EINVAL;
  if (!b_host || !x_host) return fail(h, VPS_EINVAL, "NULL vector");
  if (int rc = set_device(h)) return rc;
  const int64_t ni = h->geom[h->L].n1 - 2;
  const size_t nbytes = (size_t)(h->dim == 3 ? ni * ni * ni : ni * ni) * sizeof(double);
  VPS_CK(h, cudaMemcpyAsync(h->comp_b, b_host, nbytes, cudaMemcpyHostToDevice, h->stream));
  int rc = vps_solve(h, h->comp_b, h->comp_x, rtol, max_it, iters, rel_res);
  VPS_CK(h, cudaMemcpyAsync(x_host, h->comp_x, nbytes, cudaMemcpyDeviceToHost, h->stream));
  VPS_CK(h, cudaStreamSynchronize(h->stream));
  return rc;
}

int vps_assemble_rhs_sines(vps_handle h, int n_modes, const double* coef, const int* freq,
                           double* b) {
  if (!h) return VPS_EINVAL;
  if (n_modes < 1 || n_modes > 4096 || !coef || !freq || !b)
    return fail(h, VPS_EINVAL, "bad sine-mode arguments");
  if (int rc = set_device(h)) return rc;
  LaunchTally tally(h);
  for (int i = 0; i < n_modes * h->dim; ++i)
    if (freq[i] < 0) return fail(h, VPS_EINVAL, "negative frequency");
  if (int rc = upload_rhs_sines(h, h->L, n_modes, coef, freq, b)) return rc;
  VPS_CK(h, cudaStreamSynchronize(h->stream));
  return VPS_OK;
}

int vps_fmg(vps_handle h, int n_modes, const double* coef, const int* freq, double tol,
            int max_it, double* x, int* iters, double* rel_res) {
  if (!h) return VPS_EINVAL;
  if (n_modes < 1 || n_modes > 4096 || !coef || !freq || !x)
    return fail(h, VPS_EINVAL, "bad arguments");
  if (!(tol > 0.0) || max_it < 1) return fail(h, VPS_EINVAL, "tol must be > 0 and max_it >= 1");
  for (int i = 0; i < n_modes * h->dim; ++i)
    if (freq[i] < 0) return fail(h, VPS_EINVAL, "negative frequency");
  if (int rc = set_device(h)) return rc;
  LaunchTally tally(h);
  int rc = fmg_solve(h, n_modes, coef, freq, tol, max_it, iters, rel_res);
  const LevelGeom& g = h->geom[h->L];
  cudaError_t e = launch_unpack<double>(g, h->cx, x, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess && rc == VPS_OK) return fail(h, VPS_ECUDA, "fmg: %s", cudaGetErrorString(e));
  if (rc == VPS_OK) rc = check_waits(h);
  return rc;
}

int vps_l2_error_sine(vps_handle h, const double* x, double* err) {
  if (!h) return VPS_EINVAL;
  if (!x || !err) return fail(h, VPS_EINVAL, "NULL pointer");
  if (int rc = set_device(h)) return rc;
  LaunchTally tally(h);
  const LevelGeom& g = h->geom[h->L];
  const int k = h->k, q = k + 2, nl = k + 1;
  double xq[16], wq[16], val[kMaxK + 1];
  gauss_rule(q, xq, wq);
  std::vector<double> tab(nl * q + 2 * q);
  for (int qq = 0; qq < q; ++qq) {
    lagrange_eval(k, h->tab.z, xq[qq], val);
    for (int a = 0; a <= k; ++a) tab[a * q + qq] = val[a];
  }
  for (int qq = 0; qq < q; ++qq) {
    tab[nl * q + qq] = xq[qq];
    tab[nl * q + q + qq] = wq[qq];
  }
  VPS_CK(h, cudaMemcpyAsync(h->l2_tab, tab.data(), tab.size() * sizeof(double),
                            cudaMemcpyHostToDevice, h->stream));
  VPS_CK(h, launch_pack<double>(g, x, h->cx, h->stream));
  VPS_CK(h, launch_l2_error_sine(g, h->cx, h->l2_tab, q, h->partial, h->dots, h->stream));
  VPS_CK(h, cudaMemcpyAsync(h->host_dots, h->dots, sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
  VPS_CK(h, cudaStreamSynchronize(h->stream));
  *err = std::sqrt(h->host_dots[0]);
  return VPS_OK;
}

int vps_set_smooth_variant(vps_handle h, int level, int variant) {
  if (!h) return VPS_EINVAL;
  if (!variant_ok(h, variant)) return fail(h, VPS_EINVAL, "smoother variant %d unavailable", variant);
  if (level != 0)
    if (int rc = check_level(h, level, 1)) return rc;
  for (int l = 1; l <= h->L; ++l)
    if (level == 0 || l == level) h->smooth_var[l] = variant;
  drop_graphs(h);
  return VPS_OK;
}

int vps_get_smooth_variant(vps_handle h, int level, int* variant, int* patches_per_block) {
  if (!h) return VPS_EINVAL;
  if (int rc = check_level(h, level, 1)) return rc;
  const int v = h->smooth_var[level];
  if (variant) *variant = v;
  if (patches_per_block)
    *patches_per_block = h->prec == VPS_FP64 ? h->ks->d.variant_p[v] : h->ks->f.variant_p[v];
  return VPS_OK;
}

int vps_autotune(vps_handle h, const char* cache_path, int* from_cache) {
  if (!h) return VPS_EINVAL;
  if (int rc = set_device(h)) return rc;
  LaunchTally tally(h);
  const std::string key = tune_key(h);
  int var[kMaxLevels + 1] = {};
  int ops[kMaxLevels + 1] = {};
  int coarse = 0, schedule = VPS_SCHEDULE_PDL, coarse_solver = 0;
  if (from_cache) *from_cache = 0;
  const bool has_alt = h->prec == VPS_FP64 ? h->ks->d.apply_alt != nullptr
                                           : h->ks->f.apply_alt != nullptr;
  if (cache_path && cache_lookup(cache_path, key, &coarse, var + 1, ops + 1, &schedule,
                                 &coarse_solver, h->L)) {
    bool ok = coarse >= 1 && coarse <= h->L && schedule >= VPS_SCHEDULE_PLAIN &&
              schedule <= VPS_SCHEDULE_SWEEP &&
              coarse_solver >= 0 && coarse_solver <= 3 &&
              (!(coarse_solver & VPS_COARSE_COOPERATIVE) || h->coop_ok);
    for (int l = 1; l <= h->L; ++l)
      ok = ok && variant_ok(h, var[l]) && (ops[l] == 0 || (ops[l] == 1 && has_alt));
    if (ok) {
      for (int l = 1; l <= h->L; ++l) {
        h->smooth_var[l] = var[l];
        h->op_var[l] = ops[l];
      }
      h->schedule = schedule;
      if (coarse != h->coarse)
        if (int rc = setup_coarse(h, coarse)) return rc;
      h->coarse_coop = (coarse_solver & VPS_COARSE_COOPERATIVE) != 0;
      h->coarse_wide = (coarse_solver & VPS_COARSE_WIDE_TILES) != 0;
      drop_graphs(h);
      if (from_cache) *from_cache = 1;
      return VPS_OK;
    }
  }
  // 1) smoother variant per level and colour schedule: for each schedule
  //    (multiplicative smoother: programmatic dependent launches, the
  //    dataflow sweep, ordinary launches; additive: the handle's), the
  //    fastest smoothing step of every level on the level's buffers.  The
  //    schedule is chosen once the coarsest level is known (step 3): the one
  //    whose fastest steps on the levels above the coarsest -- the levels a
  //    V-cycle smooths -- add up to the least time.
  const bool mult = h->smoother == VPS_MULTIPLICATIVE;
  const int scheds[3] = {VPS_SCHEDULE_PDL, VPS_SCHEDULE_SWEEP, VPS_SCHEDULE_PLAIN};
  const int nsched = mult ? 3 : 1;
  float t_s[3][kMaxLevels + 1] = {};
  int v_s[3][kMaxLevels + 1] = {};
  for (int si = 0; si < nsched; ++si) {
    if (mult) h->schedule = scheds[si];
    for (int l = 1; l <= h->L; ++l) v_s[si][l] = h->smooth_var[l];
    for (int l = 2; l <= h->L; ++l) {
      float best = 1e30f;
      int bestv = h->smooth_var[l];
      for (int v = 0; v < kSmoothVariants; ++v) {
        if (!variant_ok(h, v)) continue;
        h->smooth_var[l] = v;
        float ms = 0.f;
        int rc = h->prec == VPS_FP64
                     ? time_ms(h, 3, [&] { return smooth_step<double>(h, l, (const double*)h->bv[l],
                                                                      (double*)h->xv[l], true); }, &ms)
                     : time_ms(h, 3, [&] { return smooth_step<float>(h, l, (const float*)h->bv[l],
                                                                     (float*)h->xv[l], true); }, &ms);
        if (rc) return rc;
        if (ms < best * 0.98f) {  // prefer the earlier (smaller) variant on near ties
          best = ms;
          bestv = v;
        }
      }
      v_s[si][l] = bestv;
      t_s[si][l] = best;
      h->smooth_var[l] = bestv;
    }
  }
  if (int rc = check_waits(h)) return rc;
  // the schedule for levels lc+1 .. L smoothed, with each level's fastest
  // variant under it; returns its index in scheds
  auto choose_schedule = [&](int lc) {
    float best_total = 1e30f;
    int best_si = 0;
    for (int si = 0; si < nsched; ++si) {
      float total = 0.f;
      for (int l = std::max(2, lc + 1); l <= h->L; ++l) total += t_s[si][l];
      if (total < best_total * 0.99f) {  // prefer the earlier schedule on near ties
        best_total = total;
        best_si = si;
      }
    }
    if (mult) h->schedule = scheds[best_si];
    for (int l = 2; l <= h->L; ++l) h->smooth_var[l] = v_s[best_si][l];
    drop_graphs(h);  // graphs captured under another schedule or variant
    return best_si;
  };
  int sched_now = choose_schedule(1);
  // 2) operator tile structure per level where two exist: the faster
  //    residual b - A x on the level's buffers
  for (int l = 1; l <= h->L; ++l) {
    h->op_var[l] = 0;
    if (!has_alt || l < 2) continue;
    float best = 1e30f;
    int bestv = 0;
    for (int v = 0; v < 2; ++v) {
      h->op_var[l] = v;
      float ms = 0.f;
      int rc = h->prec == VPS_FP64
                   ? time_ms(h, 5, [&] { return level_apply<double>(h, l, (const double*)h->xv[l],
                                                                    (const double*)h->bv[l],
                                                                    (double*)h->rv[l]) == cudaSuccess
                                                ? VPS_OK : VPS_ECUDA; }, &ms)
                   : time_ms(h, 5, [&] { return level_apply<float>(h, l, (const float*)h->xv[l],
                                                                   (const float*)h->bv[l],
                                                                   (float*)h->rv[l]) == cudaSuccess
                                                ? VPS_OK : VPS_ECUDA; }, &ms);
      if (rc) return rc;
      if (ms < best * 0.98f) {
        best = ms;
        bestv = v;
      }
    }
    h->op_var[l] = bestv;
  }
  // 3) coarsest level: fastest full CG solve of a smooth right-hand side;
  //    then the colour schedule for the levels above it (step 1), and, if
  //    that changed the schedule, the coarsest level once more under it
  auto tune_coarse = [&]() -> int {
    const LevelGeom& g = h->geom[h->L];
    const int ni = g.n1 - 2;
    std::vector<double> b1d((size_t)h->dim * ni);
    for (int t = 0; t < h->dim; ++t)
      for (int j = 0; j < ni; ++j) b1d[(size_t)t * ni + j] = std::sin(M_PI * (j + 1.0) / (ni + 1.0));
    const size_t need = b1d.size() * sizeof(double);
    if (need > h->rhs_cap) {
      if (h->rhs_buf) cudaFree(h->rhs_buf);
      h->rhs_buf = nullptr;
      h->rhs_cap = 0;
      VPS_CK(h, cudaMalloc(&h->rhs_buf, need));
      h->rhs_cap = need;
    }
    VPS_CK(h, cudaMemcpy(h->rhs_buf, b1d.data(), need, cudaMemcpyHostToDevice));
    VPS_CK(h, launch_rhs_tensor(g, 1, h->rhs_buf, h->comp_b, h->stream));
    float best = 1e30f;
    int bestc = h->coarse;
    bool bestcoop = h->coarse_coop, bestwide = h->coarse_wide;
    const bool can_coop = h->coop_ok;
    for (int c = 1; c <= h->L - 1 || c == 1; ++c) {
      if (h->k * (1 << c) - 1 > 64) break;  // the global solve grows as ni^(d+1)
      if (int rc = setup_coarse(h, c)) return rc;
      // the coarse solver's form on this level (one cooperative launch or
      // one launch per pass; tiles of 32 or 64 outputs), whichever solves
      // the level's system fastest
      {
        float tbest = 1e30f;
        int sbest = 0;
        for (int sv = 0; sv < 4; ++sv) {
          if ((sv & VPS_COARSE_COOPERATIVE) && !can_coop) continue;
          h->coarse_coop = (sv & VPS_COARSE_COOPERATIVE) != 0;
          h->coarse_wide = (sv & VPS_COARSE_WIDE_TILES) != 0;
          float t = 0.f;
          int rc = h->prec == VPS_FP64
                       ? time_ms(h, 5, [&] { return coarse_solve<double>(h, (const double*)h->bv[c],
                                                                         (double*)h->xv[c]); }, &t)
                       : time_ms(h, 5, [&] { return coarse_solve<float>(h, (const float*)h->bv[c],
                                                                        (float*)h->xv[c]); }, &t);
          if (rc) return rc;
          if (t < tbest * 0.98f) {
            tbest = t;
            sbest = sv;
          }
        }
        h->coarse_coop = (sbest & VPS_COARSE_COOPERATIVE) != 0;
        h->coarse_wide = (sbest & VPS_COARSE_WIDE_TILES) != 0;
      }
      float ms = 0.f;
      int rc = time_ms(h, 2, [&] { return trial_solve(h); }, &ms);
      if (rc == VPS_ENOCONV || rc == VPS_EBREAKDOWN) ms = 1e30f;  // not a usable candidate
      else if (rc) return rc;
      if (ms < best * 0.98f) {
        best = ms;
        bestc = c;
        bestcoop = h->coarse_coop;
        bestwide = h->coarse_wide;
      }
      if (c >= h->L) break;
    }
    if (int rc = check_waits(h)) return rc;
    if (int rc = setup_coarse(h, bestc)) return rc;
    h->coarse_coop = bestcoop;
    h->coarse_wide = bestwide;
    return VPS_OK;
  };
  if (int rc = tune_coarse()) return rc;
  if (choose_schedule(h->coarse) != sched_now) {
    if (int rc = tune_coarse()) return rc;
    choose_schedule(h->coarse);
  }
  if (cache_path) {
    for (int l = 1; l <= h->L; ++l) {
      var[l] = h->smooth_var[l];
      ops[l] = h->op_var[l];
    }
    cache_store(cache_path, key, h->coarse, var + 1, ops + 1, h->schedule,
                (h->coarse_coop ? VPS_COARSE_COOPERATIVE : 0) |
                    (h->coarse_wide ? VPS_COARSE_WIDE_TILES : 0), h->L);
  }
  drop_graphs(h);
  return VPS_OK;
}

int vps_set_operator_variant(vps_handle h, int level, int variant) {
  if (!h) return VPS_EINVAL;
  if (int rc = check_level(h, level, 1)) return rc;
  const bool has_alt = h->prec == VPS_FP64 ? h->ks->d.apply_alt != nullptr
                                           : h->ks->f.apply_alt != nullptr;
  if (variant != 0 && !(variant == 1 && has_alt))
    return fail(h, VPS_EINVAL, "operator variant %d unavailable", variant);
  h->op_var[level] = variant;
  drop_graphs(h);
  return VPS_OK;
}

int vps_get_operator_variant(vps_handle h, int level, int* variant, int* n_variants) {
  if (!h) return VPS_EINVAL;
  if (int rc = check_level(h, level, 1)) return rc;
  if (variant) *variant = h->op_var[level];
  if (n_variants)
    *n_variants = (h->prec == VPS_FP64 ? h->ks->d.apply_alt != nullptr
                                       : h->ks->f.apply_alt != nullptr) ? 2 : 1;
  return VPS_OK;
}

int vps_set_colour_schedule(vps_handle h, int schedule) {
  if (!h) return VPS_EINVAL;
  if (schedule < VPS_SCHEDULE_PLAIN || schedule > VPS_SCHEDULE_SWEEP)
    return fail(h, VPS_EINVAL, "colour schedule %d unknown", schedule);
  h->schedule = schedule;
  drop_graphs(h);
  return VPS_OK;
}

int vps_get_colour_schedule(vps_handle h, int* schedule) {
  if (!h || !schedule) return VPS_EINVAL;
  *schedule = h->schedule;
  return VPS_OK;
}

int vps_set_coarse_solver(vps_handle h, int solver) {
  if (!h) return VPS_EINVAL;
  if (solver < 0 || solver > (VPS_COARSE_COOPERATIVE | VPS_COARSE_WIDE_TILES))
    return fail(h, VPS_EINVAL, "coarse solver %d unknown", solver);
  if ((solver & VPS_COARSE_COOPERATIVE) && !h->coop_ok)
    return fail(h, VPS_EINVAL, "the device does not support cooperative launches");
  h->coarse_coop = (solver & VPS_COARSE_COOPERATIVE) != 0;
  h->coarse_wide = (solver & VPS_COARSE_WIDE_TILES) != 0;
  drop_graphs(h);
  return VPS_OK;
}

int vps_get_coarse_solver(vps_handle h, int* solver) {
  if (!h || !solver) return VPS_EINVAL;
  *solver = (h->coarse_coop ? VPS_COARSE_COOPERATIVE : 0) | (h->coarse_wide ? VPS_COARSE_WIDE_TILES : 0);
  return VPS_OK;
}

int vps_check_waits(vps_handle h) {
  if (!h) return VPS_EINVAL;
  if (int rc = set_device(h)) return rc;
  return check_waits(h);
}

int vps_skip_sweep_tiles(vps_handle h, int level, int64_t tiles) {
  if (!h) return VPS_EINVAL;
  if (int rc = check_level(h, level, 1)) return rc;
  if (tiles < 0) return fail(h, VPS_EINVAL, "tiles < 0");
  if (int rc = set_device(h)) return rc;
  const unsigned long long head = (unsigned long long)tiles;
  VPS_CK(h, cudaStreamSynchronize(h->stream));
  VPS_CK(h, cudaMemcpy(&h->sweep_ctr[level].head, &head, sizeof(head), cudaMemcpyHostToDevice));
  return VPS_OK;
}

int vps_set_coarse_level(vps_handle h, int level) {
  if (!h) return VPS_EINVAL;
  if (int rc = set_device(h)) return rc;
  if (level == 0) level = auto_coarse_level(h->k, h->L);
  if (level < 1 || level > h->L)
    return fail(h, VPS_EINVAL, "coarse level %d outside 1..%d", level, h->L);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess)
    return fail(h, VPS_ECUDA, "stream synchronisation failed");
  return setup_coarse(h, level);
}

int vps_get_coarse_level(vps_handle h, int* level) {
  if (!h || !level) return VPS_EINVAL;
  *level = h->coarse;
  return VPS_OK;
}

int vps_kernel_launches(vps_handle h, int64_t* count) {
  if (!h || !count) return VPS_EINVAL;
  *count = h->kernels;
  return VPS_OK;
}

int vps_set_outer_operator(vps_handle h, int mode) {
  if (!h) return VPS_EINVAL;
  if (mode != VPS_OUTER_FP64 && mode != VPS_OUTER_DOUBLE_FLOAT)
    return fail(h, VPS_EINVAL, "outer operator mode %d (expected 0 or 1)", mode);
  if (mode == VPS_OUTER_DOUBLE_FLOAT && !h->cph) {
    if (int rc = set_device(h)) return rc;
    const size_t fb = (size_t)h->geom[h->L].total * sizeof(float);
    void* p;
    if (int rc = dalloc(h, &p, fb)) return rc;
    h->cph = (float*)p;
    if (int rc = dalloc(h, &p, fb)) return rc;
    h->cpl = (float*)p;
  }
  h->outer = mode;
  return VPS_OK;
}

int vps_set_smoother_kernel(vps_handle h, int kind) {
  if (!h) return VPS_EINVAL;
  if (kind < VPS_KERNEL_FUSED || kind > VPS_KERNEL_GLOBAL_INVERSE)
    return fail(h, VPS_EINVAL, "smoother kernel %d (expected 0..3)", kind);
  if (kind != VPS_KERNEL_FUSED && h->smoother != VPS_MULTIPLICATIVE)
    return fail(h, VPS_EINVAL, "kernel structures apply to the multiplicative smoother");
  if (kind == VPS_KERNEL_GLOBAL_INVERSE && !h->ainv) {
    const int m = h->tab.m, d = h->dim;
    const int md = d == 3 ? m * m * m : m * m;
    const bool ok = h->prec == VPS_FP64 ? h->ks->d.inverse_solve != nullptr
                                        : h->ks->f.inverse_solve != nullptr;
    if (!ok) return fail(h, VPS_EINVAL, "dense inverse of %d rows exceeds 1024", md);
    if (int rc = set_device(h)) return rc;
    // A_j^-1 = W diag(1 / sum of eigenvalues) W^T, W = S (x) S [(x) S], in FP64
    std::vector<double> A((size_t)md * md, 0.0), dq(md);
    auto digit = [&](int e, int t) { return t == 0 ? e % m : (t == 1 ? (e / m) % m : e / (m * m)); };
    for (int q = 0; q < md; ++q) {
      double sl = 0.0;
      for (int t = 0; t < d; ++t) sl += h->tab.lam[digit(q, t)];
      dq[q] = 1.0 / sl;
    }
    std::vector<double> W((size_t)md * md);
    for (int e = 0; e < md; ++e)
      for (int q = 0; q < md; ++q) {
        double w = 1.0;
        for (int t = 0; t < d; ++t) w *= h->tab.S[digit(e, t) * m + digit(q, t)];
        W[(size_t)e * md + q] = w;
      }
    for (int e = 0; e < md; ++e)
      for (int f = 0; f <= e; ++f) {
        double acc = 0.0;
        const double* we = &W[(size_t)e * md];
        const double* wf = &W[(size_t)f * md];
        for (int q = 0; q < md; ++q) acc += we[q] * dq[q] * wf[q];
        A[(size_t)e * md + f] = A[(size_t)f * md + e] = acc;
      }
    void* p;
    if (int rc = dalloc(h, &p, (size_t)md * md * h->esz)) return rc;
    cudaError_t e;
    if (h->prec == VPS_FP64) {
      e = cudaMemcpyAsync(p, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    } else {
      std::vector<float> Af(A.begin(), A.end());
      e = cudaMemcpyAsync(p, Af.data(), Af.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    if (e != cudaSuccess) return fail(h, VPS_ECUDA, "dense inverse: %s", cudaGetErrorString(e));
    h->ainv = p;
  }
  h->kernel_kind = kind;
  drop_graphs(h);
  return VPS_OK;
}

int vps_get_smoother_kernel(vps_handle h, int* kind) {
  if (!h || !kind) return VPS_EINVAL;
  *kind = h->kernel_kind;
  return VPS_OK;
}

int vps_get_solve_info(vps_handle h, int* restarts, int* at_rounding_bound) {
  if (!h) return VPS_EINVAL;
  if (restarts) *restarts = h->last_restarts;
  if (at_rounding_bound) *at_rounding_bound = h->last_at_floor;
  return VPS_OK;
}

int vps_get_outer_operator(vps_handle h, int* mode) {
  if (!h || !mode) return VPS_EINVAL;
  *mode = h->outer;
  return VPS_OK;
}

int vps_set_graphs(vps_handle h, int enable) {
  if (!h) return VPS_EINVAL;
  if (enable && !h->stream) return fail(h, VPS_EINVAL, "CUDA graphs need a non-default stream");
  h->use_graphs = enable != 0;
  return VPS_OK;
}

}  // extern "C"
