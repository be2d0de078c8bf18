// One additive smoothing step that allocates no memory.
//
// Every other entry point needs a handle, and vps_create allocates its level
// vectors with cudaMalloc.  Some callers cannot allocate: a host application
// whose framework reserves nearly all device memory for its own pool at
// start-up (a cudaMalloc then fails, or takes memory the pool counted on),
// a latency-bound loop that cannot afford the device-wide synchronisation a
// cudaFree implies, or a deployment whose device-memory budget is fixed and
// audited when it starts.  vps_smooth_additive_static serves them: the
// caller passes b and x, and the step's scratch -- the global residual
// r = b - A x and the table of 1/(lambda_i + lambda_j [+ lambda_l]) -- lives
// in the file-scope device array g_scratch below, of fixed size
// kScratchBytes (32 MiB).  A GPU holds that array from the moment the
// library's device code is loaded on it (with CUDA's default lazy loading:
// the first call of this entry point there) until the process exits.
//
// All calls share the one array: two calls whose work overlaps on the same
// GPU (different streams, or different host threads without ordering) race
// on it and corrupt each other's residual.  Issue them in one stream or
// order them explicitly.
//
// Host code must not use &g_scratch directly: on the host that name is a
// stand-in, not a device address.  Once per device, with that device
// current, the first call takes the array's device address with
// cudaGetSymbolAddress and keeps it; every later call on that device reuses
// it.  The first call on a device also copies the degree's 1D tables into
// the kernels' constant memory.  Make that first call before any stream
// capture begins on the device.  No call allocates: no cudaMalloc, no
// cudaFree, no allocating library routine.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "vps.h"
#include "vps_internal.h"

namespace vps {
namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr size_t kTableBytes = size_t(32) << 10;    // first 32 KiB: eigenvalue table
constexpr int kMaxDev = 64;

// The scratch shared by every call of vps_smooth_additive_static.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_dev[kMaxDev] = {};          // device address of g_scratch, per device
bool g_tables_up[kMaxDev][2][kMaxK] = {};   // constant tables uploaded, per device

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

template <typename T>
int run(const KernelSet* ks, const LevelGeom& g, const HostTables& tab, double damping,
        const T* b, T* x, void* base, cudaStream_t s) {
  const KernelFns<T>& F = fns_of<T>(ks);
  // eigenvalue table (at most 13^3 entries) from a stack array
  const int m = tab.m, md = g.dim == 3 ? m * m * m : m * m;
  T il[13 * 13 * 13];
  for (int a = 0; a < md; ++a) {
    const int i0 = a % m, i1 = (a / m) % m, i2 = a / (m * m);
    il[a] = (T)(1.0 / (tab.lam[i0] + tab.lam[i1] + (g.dim == 3 ? tab.lam[i2] : 0.0)));
  }
  T* il_dev = static_cast<T*>(base);
  T* r = reinterpret_cast<T*>(static_cast<unsigned char*>(base) + kTableBytes);
  cudaError_t e = cudaMemcpyAsync(il_dev, il, md * sizeof(T), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(VPS_ECUDA, "table copy: %s", cudaGetErrorString(e));
  // r is rewritten at every node before the colour passes read it; nothing in
  // the scratch has to start at zero.
  e = F.apply(g, x, b, r, s);
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
  const LevelGeom g = make_geom(dim, degree, level);
  const size_t esz = precision == VPS_FP64 ? sizeof(double) : sizeof(float);
  const double need = (double)g.total * (double)esz;
  if (need > (double)(kScratchBytes - kTableBytes))
    return fail(VPS_EINVAL,
                "level %d needs %.0f bytes of scratch for its residual; the static scratch "
                "holds %zu bytes (use a handle: vps_create + vps_smooth)",
                level, need, kScratchBytes - kTableBytes);
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
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess || !p)
        return fail(VPS_ECUDA, "cudaGetSymbolAddress(g_scratch): %s", cudaGetErrorString(e));
      g_scratch_dev[dev] = p;
    }
    if (!g_tables_up[dev][dim - 2][degree - 1]) {
      e = ks->upload(tab);
      if (e != cudaSuccess) return fail(VPS_ECUDA, "constant upload: %s", cudaGetErrorString(e));
      g_tables_up[dev][dim - 2][degree - 1] = true;
    }
    base = g_scratch_dev[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return precision == VPS_FP64
             ? run<double>(ks, g, tab, damping, static_cast<const double*>(b),
                           static_cast<double*>(x), base, s)
             : run<float>(ks, g, tab, damping, static_cast<const float*>(b), static_cast<float*>(x),
                          base, s);
}
