// One additive smoothing step that allocates no memory.
//
// Every other entry point needs a handle, and vps_create allocates its level
// vectors with cudaMalloc.  Some callers cannot allocate: a host application
// whose framework reserves nearly all device memory for its own pool at
// start-up (a cudaMalloc then fails, or takes memory the pool counted on),
// a latency-bound loop that cannot afford the device-wide synchronisation a
// cudaFree implies, or a deployment whose device-memory budget is fixed and
// audited when it starts.  vps_smooth_additive_static serves them: the
// caller passes b and x, and the step's scratch lives in two file-scope
// device arrays below: g_scratch (kScratchBytes = 32 MiB) holds the global
// residual r = b - A x, and g_tables (kTableBytes) holds the table of
// 1/(lambda_i + lambda_j [+ lambda_l]) of every (dimension, degree,
// precision), each in a slot of its own.  A GPU holds both arrays from the
// moment the library's device code is loaded on it (with CUDA's default lazy
// loading: the first call of this entry point there) until the process exits.
//
// All calls share g_scratch: two calls whose work overlaps on the same GPU
// (different streams, or different host threads without ordering) race on
// it and corrupt each other's residual.  Issue them in one stream or order
// them explicitly.  Nothing in g_scratch has to start at zero: every call
// rewrites the residual at every node before reading it.
//
// Host code must not use &g_scratch or &g_tables directly: on the host those
// names are stand-ins, not device addresses.  Once per device, with that
// device current, the first call takes both arrays' device addresses with
// cudaGetSymbolAddress and keeps them; every later call on that device reuses
// them.  The first call of a (dimension, degree, precision) on a device also
// fills that shape's slot of g_tables and the degree's 1D tables in the
// kernels' constant memory, with synchronous copies; later calls of the shape
// issue kernels only.  So make the first call of each shape on a device
// before any stream capture begins there.  No call allocates: no cudaMalloc,
// no cudaFree, no allocating library routine.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "vps.h"
#include "vps_internal.h"

namespace vps {
namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB: the residual
constexpr int kMaxDev = 64;

// Byte offset of the eigenvalue table of (dim, degree, precision) in
// g_tables: the slots of all shapes one after another, each m^dim entries
// (m = 2 degree - 1) rounded up to 256 bytes.
constexpr size_t table_slot(int dim, int degree, int fp64) {
  size_t off = 0;
  for (int d = 2; d <= 3; ++d)
    for (int k = 1; k <= kMaxK; ++k)
      for (int p = 0; p < 2; ++p) {
        if (d == dim && k == degree && p == fp64) return off;
        const size_t mm = 2 * k - 1, md = d == 3 ? mm * mm * mm : mm * mm;
        off += (md * (p ? 8 : 4) + 255) / 256 * 256;
      }
  return off;
}
constexpr size_t kTableBytes = table_slot(4, 0, 0);  // past the last slot: 66,048 bytes

// The scratch shared by every call of vps_smooth_additive_static.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static __device__ __align__(256) unsigned char g_tables[kTableBytes];

std::mutex g_mu;
void* g_scratch_dev[kMaxDev] = {};              // device address of g_scratch, per device
void* g_tables_dev[kMaxDev] = {};               // device address of g_tables, per device
bool g_consts_up[kMaxDev][2][kMaxK] = {};       // 1D constant tables uploaded
bool g_table_up[kMaxDev][2][kMaxK][2] = {};     // eigenvalue table slot filled

int fail(int code, const char* fmt, ...) {
  char buf[384];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_thread_error(buf);
  return code;
}

template <typename T>
const KernelFns<T>& fns_of(const KernelSet* ks);
template <>
const KernelFns<float>& fns_of<float>(const KernelSet* ks) { return ks->f; }
template <>
const KernelFns<double>& fns_of<double>(const KernelSet* ks) { return ks->d; }

// Fills the eigenvalue table slot of (dim, degree, T) on the current device
// (synchronous copy from host memory to the symbol, at set-up only).
template <typename T>
cudaError_t fill_table(const HostTables& tab, int dim, int degree) {
  const int m = tab.m, md = dim == 3 ? m * m * m : m * m;
  T il[13 * 13 * 13];
  for (int a = 0; a < md; ++a) {
    const int i0 = a % m, i1 = (a / m) % m, i2 = a / (m * m);
    il[a] = (T)(1.0 / (tab.lam[i0] + tab.lam[i1] + (dim == 3 ? tab.lam[i2] : 0.0)));
  }
  return cudaMemcpyToSymbol(g_tables, il, md * sizeof(T),
                            table_slot(dim, degree, sizeof(T) == 8 ? 1 : 0),
                            cudaMemcpyHostToDevice);
}

template <typename T>
int run(const KernelSet* ks, const LevelGeom& g, double damping, const T* b, T* x, void* scratch,
        void* tables, cudaStream_t s) {
  const KernelFns<T>& F = fns_of<T>(ks);
  const T* il_dev = reinterpret_cast<const T*>(
      static_cast<unsigned char*>(tables) + table_slot(g.dim, g.k, sizeof(T) == 8 ? 1 : 0));
  T* r = static_cast<T*>(scratch);
  // r is rewritten at every node before the colour passes read it; nothing in
  // the scratch has to start at zero.
  cudaError_t e = F.apply(g, x, b, r, s);
  if (e != cudaSuccess) return fail(VPS_ECUDA, "residual: %s", cudaGetErrorString(e));
  for (int c = 0; c < (1 << g.dim); ++c) {
    e = F.smooth_add(g, make_colour(g, c), r, x, il_dev, (T)damping, s);
    if (e != cudaSuccess) return fail(VPS_ECUDA, "colour %d: %s", c, cudaGetErrorString(e));
  }
  return VPS_OK;
}

}  // namespace
}  // namespace vps

extern "C" int vps_smooth_additive_static(int dim, int degree, int level, int precision,
                                          double damping, const void* b, void* x,
                                          void* cuda_stream) {
  using namespace vps;
  set_thread_error("");
  if (dim != 2 && dim != 3) return fail(VPS_EINVAL, "dim must be 2 or 3 (got %d)", dim);
  if (degree < 1 || degree > VPS_MAX_DEGREE)
    return fail(VPS_EINVAL, "degree must be 1..%d (got %d)", VPS_MAX_DEGREE, degree);
  if (level < 2 || level > 24) return fail(VPS_EINVAL, "level must be 2..24 (got %d)", level);
  if (precision != VPS_FP64 && precision != VPS_FP32)
    return fail(VPS_EINVAL, "precision must be VPS_FP64 or VPS_FP32");
  if (!(damping > 0.0) || !std::isfinite(damping))
    return fail(VPS_EINVAL, "damping must be positive and finite");
  if (!b || !x || b == x) return fail(VPS_EINVAL, "b and x must be distinct non-NULL vectors");
  // size check in floating point, before any integer geometry: levels whose
  // element count overflows 64-bit integers are rejected here as well
  const double esz = precision == VPS_FP64 ? sizeof(double) : sizeof(float);
  const double need = level_elements(dim, degree, level) * esz;
  if (!(need <= (double)kScratchBytes))
    return fail(VPS_EINVAL,
                "level %d needs %.4g bytes of scratch for its residual; the static scratch "
                "holds %zu bytes (use a handle: vps_create + vps_smooth)",
                level, need, kScratchBytes);
  const LevelGeom g = make_geom(dim, degree, level);
  HostTables tab;
  char ebuf[256];
  if (!build_tables(degree, &tab, ebuf, sizeof(ebuf))) return fail(VPS_EINVAL, "%s", ebuf);
  ensure_registered();
  const KernelSet* ks = kernel_registry(dim, degree);
  if (!ks || !ks->present) return fail(VPS_EINVAL, "no kernels for dim %d degree %d", dim, degree);

  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(VPS_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDev) return fail(VPS_ECUDA, "device index %d out of range", dev);
  const int fp64 = precision == VPS_FP64 ? 1 : 0;
  void* scratch = nullptr;
  void* tables = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
      void* p = nullptr;
      void* q = nullptr;
      e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess || !p)
        return fail(VPS_ECUDA, "cudaGetSymbolAddress(g_scratch): %s", cudaGetErrorString(e));
      e = cudaGetSymbolAddress(&q, g_tables);
      if (e != cudaSuccess || !q)
        return fail(VPS_ECUDA, "cudaGetSymbolAddress(g_tables): %s", cudaGetErrorString(e));
      g_tables_dev[dev] = q;
      g_scratch_dev[dev] = p;
    }
    if (!g_consts_up[dev][dim - 2][degree - 1]) {
      e = ks->upload(tab);
      if (e != cudaSuccess) return fail(VPS_ECUDA, "constant upload: %s", cudaGetErrorString(e));
      g_consts_up[dev][dim - 2][degree - 1] = true;
    }
    if (!g_table_up[dev][dim - 2][degree - 1][fp64]) {
      e = fp64 ? fill_table<double>(tab, dim, degree) : fill_table<float>(tab, dim, degree);
      if (e != cudaSuccess) return fail(VPS_ECUDA, "table upload: %s", cudaGetErrorString(e));
      g_table_up[dev][dim - 2][degree - 1][fp64] = true;
    }
    scratch = g_scratch_dev[dev];
    tables = g_tables_dev[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return fp64 ? run<double>(ks, g, damping, static_cast<const double*>(b),
                            static_cast<double*>(x), scratch, tables, s)
              : run<float>(ks, g, damping, static_cast<const float*>(b), static_cast<float*>(x),
                           scratch, tables, s);
}
