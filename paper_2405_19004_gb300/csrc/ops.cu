// Vector kernels of the solver: layout conversion, deterministic
// reductions, the CG updates, the separable load vector and the L2 error.
//
// The paper runs these "vector operations" through a library vector class
// (Section 3, building blocks); here they are plain kernels.  Reductions use
// a fixed grid and fixed trees, so a result does not depend on scheduling:
// the same inputs give bit-identical scalars on every run.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "fp_bits.cuh"
#include "vps.h"
#include "vps_internal.h"

namespace vps {

namespace {

constexpr int kThreads = 256;

// Chunked grid-stride loop of the vector kernels: thread t of block B takes
// the chunks that start at i0 = (B + j gridDim) kU kThreads + t (j = 0, 1,
// ..), elements i0 + u kThreads (u < kU; coalesced for every u).  A kernel
// loads all kU elements of a chunk before it uses any, so each thread keeps
// kU loads in flight (the fixed 608-block grid of the reductions holds 1024
// threads per SM: with one element per thread and iteration, few bytes are
// in flight for the DRAM latency).
constexpr int kU = 4;
#define VPS_CHUNKS(i0, n)                                                         \
  for (int64_t i0 = blockIdx.x * (int64_t)(kU * kThreads) + threadIdx.x; i0 < (n); \
       i0 += (int64_t)gridDim.x * (kU * kThreads))

inline unsigned grid_for(int64_t n, int per_thread = 1) {
  int64_t g = (n + (int64_t)kThreads * per_thread - 1) / ((int64_t)kThreads * per_thread);
  if (g < 1) g = 1;
  if (g > 4 * 152 * 8) g = 4 * 152 * 8;
  return (unsigned)g;
}

template <typename T>
__global__ void pack_kernel(const T* __restrict__ comp, T* __restrict__ lev, int dim, int n1,
                            int64_t px, int64_t pz, int64_t total) {
  const int ni = n1 - 2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = e % px;
    const int64_t i1 = (e / px) % n1;
    const int64_t i2 = dim == 3 ? e / pz : 1;
    T v = T(0);
    if (i0 >= 1 && i0 <= ni && i1 >= 1 && i1 <= ni && i2 >= 1 && i2 <= ni)
      v = comp[(i0 - 1) + (int64_t)ni * ((i1 - 1) + (int64_t)ni * (dim == 3 ? i2 - 1 : 0))];
    lev[e] = v;
  }
}

template <typename T>
__global__ void unpack_kernel(const T* __restrict__ lev, T* __restrict__ comp, int dim, int n1,
                              int64_t px, int64_t pz, int64_t ncomp) {
  const int ni = n1 - 2;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncomp;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j0 = c % ni;
    const int64_t j1 = (c / ni) % ni;
    const int64_t j2 = dim == 3 ? c / ((int64_t)ni * ni) : 0;
    comp[c] = lev[(j0 + 1) + (j1 + 1) * px + (dim == 3 ? (j2 + 1) * pz : 0)];
  }
}

// Fixed-order block reduction of NV values per thread; every thread gets
// the sums.  Butterflies of shuffles within each warp, then over the warp
// sums in warp 0 (the partners of a butterfly add the same two values, so
// all lanes hold identical bits).  sh: at least NV * 33 doubles.  The
// additions are FP64 instructions, the slow pipe of this GPU: a tree over
// shared memory costs every warp one addition per level, the butterflies
// five per warp plus three.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh) {
  constexpr int kWarps = kThreads / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
    if (lane == 0) sh[j * 32 + w] = v[j];
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double t = lane < kWarps ? sh[j * 32 + lane] : 0.0;
#pragma unroll
      for (int o = kWarps / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) sh[NV * 32 + j] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = sh[NV * 32 + j];
}

__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return f2d(v); }

// s += a b for a double a = ah + al (split_f2) and a float b in double-float
// arithmetic, FP32 instructions only: ah b exactly as p + e (one FMA for e),
// al b rounded, the high words summed by TwoSum and every error into s.lo.
// Relative error about 2^-46 of the sum of |a b| over a thread's terms.
struct F2 {
  float hi, lo;
};
__device__ __forceinline__ void f2_madd(F2& s, float ah, float al, float b) {
  const float p = ah * b;
  const float e = fmaf(ah, b, -p);
  const float t = s.hi + p;
  const float bb = t - s.hi;
  const float err = (s.hi - (t - bb)) + (p - bb);
  s.hi = t;
  s.lo += err + fmaf(al, b, e);
}

// partial[j * kDotBlocks + block] = sum over this block's fixed subset of
// the products a.b (j = 0) and, with NP = 2, a.e (j = 1; partial[1..] is
// 0 for NP = 1).  b and e in FP64, or in FP32: then the per-thread sums are
// double-float (the FP64 multiply-adds, which issue at 1/64 of the FP32 rate
// on this GPU, bounded the kernel), widened to FP64 for the block sum.
template <typename TB, int NP>
__global__ void __launch_bounds__(kThreads)
dot_partial_kernel(const double* __restrict__ a, const TB* __restrict__ b,
                   const TB* __restrict__ e, int64_t n, double* __restrict__ partial) {
  __shared__ double sh[2 * 33];
  double v[NP];
  if constexpr (sizeof(TB) == 4) {
    F2 f[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) f[j] = F2{0.f, 0.f};
    VPS_CHUNKS(i0, n) {
      double av[kU];
      float bv[kU], ev[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int64_t i = i0 + u * kThreads;
        const bool in = i < n;
        av[u] = in ? a[i] : 0.0;
        bv[u] = in ? b[i] : 0.f;
        if constexpr (NP == 2) ev[u] = in ? e[i] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        float ah, al;
        split_f2(av[u], ah, al);
        f2_madd(f[0], ah, al, bv[u]);
        if constexpr (NP == 2) f2_madd(f[NP - 1], ah, al, ev[u]);
      }
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) v[j] = f2d(f[j].hi) + f2d(f[j].lo);
  } else {
#pragma unroll
    for (int j = 0; j < NP; ++j) v[j] = 0.0;
    VPS_CHUNKS(i0, n) {
      double av[kU], bv[kU], ev[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int64_t i = i0 + u * kThreads;
        const bool in = i < n;
        av[u] = in ? a[i] : 0.0;
        bv[u] = in ? to_d(b[i]) : 0.0;
        if constexpr (NP == 2) ev[u] = in ? to_d(e[i]) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        v[0] = fma(av[u], bv[u], v[0]);
        if constexpr (NP == 2) v[NP - 1] = fma(av[u], ev[u], v[NP - 1]);
      }
    }
  }
  block_sum<NP>(v, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = v[0];
    partial[kDotBlocks + blockIdx.x] = NP == 2 ? v[NP - 1] : 0.0;
  }
}

__global__ void __launch_bounds__(kThreads)
dot_final_kernel(const double* __restrict__ partial, double* __restrict__ out, int nprod) {
  __shared__ double sh[2 * kThreads];
  double v[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < kDotBlocks; i += kThreads) {
    v[0] += partial[i];
    v[1] += partial[kDotBlocks + i];
  }
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    out[0] = v[0];
    if (nprod > 1) out[1] = v[1];
  }
}

// Block-Krylov helpers (GMRES).  V: nv vectors of length n, vector i at
// V + i * ld.  partial[i * kDotBlocks + block] = V_i . w over the block's
// fixed subset (the same fixed order as dot_partial_kernel).
__global__ void __launch_bounds__(kThreads)
multi_dot_partial_kernel(const double* __restrict__ V, int64_t ld, const double* __restrict__ w,
                         int64_t n, double* __restrict__ partial) {
  __shared__ double sh[kThreads];
  const double* v = V + blockIdx.y * ld;
  double acc[1] = {0.0};
  VPS_CHUNKS(i0, n) {
    double vv[kU], wv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = i0 + u * kThreads;
      vv[u] = i < n ? v[i] : 0.0;
      wv[u] = i < n ? w[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) acc[0] = fma(vv[u], wv[u], acc[0]);
  }
  block_sum<1>(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.y * kDotBlocks + blockIdx.x] = acc[0];
}

// out[i] = sum of partial[i * kDotBlocks ..] in a fixed order (one block per i).
__global__ void __launch_bounds__(kThreads)
multi_dot_final_kernel(const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double sh[kThreads];
  double acc[1] = {0.0};
  for (int i = threadIdx.x; i < kDotBlocks; i += kThreads) acc[0] += partial[blockIdx.x * kDotBlocks + i];
  block_sum<1>(acc, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = acc[0];
}

// w += sign * sum_i c[i] V_i  (c on the device).
__global__ void multi_axpy_kernel(double* __restrict__ w, const double* __restrict__ V, int64_t ld,
                                  int nv, const double* __restrict__ c, double sign, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double acc = w[e];
    for (int i = 0; i < nv; ++i) acc = fma(sign * __ldg(c + i), V[i * ld + e], acc);
    w[e] = acc;
  }
}

__global__ void scale_kernel(double* __restrict__ y, const double* __restrict__ x, double a,
                             int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = a * x[e];
}

// p (and, when ph is given, its split into two floats ph + pl, the input
// of the double-float operator: split_f2, p - ph - pl below 2^-47 |p|)
__device__ __forceinline__ void store_p(double* p, float* ph, float* pl, int64_t i, double v) {
  p[i] = v;
  if (ph) {
    float hi, lo;
    split_f2(v, hi, lo);
    ph[i] = hi;
    pl[i] = lo;
  }
}

// p = z_new, z_old = z_new (the first direction, or after a restart); z_old
// is kept in the type of z_new (exact).
template <typename TZ>
__global__ void cg_init_p_kernel(double* __restrict__ p, TZ* __restrict__ z,
                                 const TZ* __restrict__ zn, float* __restrict__ ph,
                                 float* __restrict__ pl, int64_t n) {
  VPS_CHUNKS(i0, n) {
    TZ zi[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = i0 + u * kThreads;
      zi[u] = i < n ? zn[i] : TZ(0);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = i0 + u * kThreads;
      if (i < n) {
        store_p(p, ph, pl, i, to_d(zi[u]));
        z[i] = zi[u];
      }
    }
  }
}

__global__ void split_df_kernel(const double* __restrict__ a, float* __restrict__ ph,
                                float* __restrict__ pl, int64_t n) {
  VPS_CHUNKS(i0, n) {
    double v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = i0 + u * kThreads;
      v[u] = i < n ? a[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = i0 + u * kThreads;
      if (i < n) {
        float hi, lo;
        split_f2(v[u], hi, lo);
        ph[i] = hi;
        pl[i] = lo;
      }
    }
  }
}

// The sum of the kDotBlocks partials of a dot product, in the fixed order
// of dot_final_kernel (every block of a grid computes the same value).
template <int NV>
__device__ __forceinline__ void reduce_partials(const double* __restrict__ partial,
                                                double (&v)[NV], double* sh) {
  for (int j = 0; j < NV; ++j) v[j] = 0.0;
  for (int i = threadIdx.x; i < kDotBlocks; i += kThreads)
    for (int j = 0; j < NV; ++j) v[j] += partial[j * kDotBlocks + i];
  block_sum<NV>(v, sh);
  __syncthreads();  // sh is reused by the caller
}

// CG, after z_new = B r: beta = (r.z_new - r.z_old) / rz from the partials
// of the two products, p = z_new + beta p (and its double-float split),
// z_old = z_new; rzn (r.z_new) is kept for alpha.  z_new and z_old in FP32
// (the FP32 V-cycle's output, converted exactly) or FP64.
template <typename TZ>
__global__ void __launch_bounds__(kThreads)
cg_update_p_fused_kernel(double* __restrict__ p, TZ* __restrict__ z,
                         const TZ* __restrict__ zn, const double* __restrict__ partial,
                         CgScalars* __restrict__ sc, float* __restrict__ ph,
                         float* __restrict__ pl, int64_t n) {
  __shared__ double sh[2 * 33];
  double v[2];
  reduce_partials<2>(partial, v, sh);
  const double rzn = v[0], rzo = v[1], rz = sc->rz;
  const bool bad = !(rz != 0.0) || !isfinite(rzn) || !isfinite(rzo);
  const double beta = bad ? 0.0 : (rzn - rzo) / rz;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->rzn = rzn;
    sc->rzo = rzo;
    sc->beta = beta;
    if (bad) sc->flag = 1;
  }
  VPS_CHUNKS(i0, n) {
    TZ zi[kU];
    double pi[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = i0 + u * kThreads;
      zi[u] = i < n ? zn[i] : TZ(0);
      pi[u] = i < n ? p[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = i0 + u * kThreads;
      if (i < n) {
        store_p(p, ph, pl, i, fma(beta, pi[u], to_d(zi[u])));
        z[i] = zi[u];
      }
    }
  }
}

// CG, after A p: alpha = rzn / p.Ap from the partials of p.Ap, x += alpha p,
// r -= alpha A p, and the partials of r.r (same chunks and order as
// dot_partial_kernel: the grid is kDotBlocks blocks).  rz <- rzn for beta.
__global__ void __launch_bounds__(kThreads)
cg_update_xr_fused_kernel(double* __restrict__ x, double* __restrict__ r,
                          const double* __restrict__ p, const double* __restrict__ Ap,
                          const double* __restrict__ partial_pAp, CgScalars* __restrict__ sc,
                          double* __restrict__ partial_rr, int64_t n) {
  __shared__ double sh[33];
  double v[1];
  reduce_partials<1>(partial_pAp, v, sh);
  const double pAp = v[0], rz = sc->rzn;
  const bool bad = !(pAp > 0.0) || !isfinite(pAp) || !isfinite(rz);
  const double alpha = bad ? 0.0 : rz / pAp;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->pAp = pAp;
    sc->alpha = alpha;
    sc->rz = rz;
    if (bad) sc->flag = 1;
  }
  double acc[1] = {0.0};
  VPS_CHUNKS(i0, n) {
    double xv[kU], pv[kU], av[kU], rv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = i0 + u * kThreads;
      const bool in = i < n;
      xv[u] = in ? x[i] : 0.0;
      pv[u] = in ? p[i] : 0.0;
      av[u] = in ? Ap[i] : 0.0;
      rv[u] = in ? r[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = i0 + u * kThreads;
      const double ri = fma(-alpha, av[u], rv[u]);
      if (i < n) {
        x[i] = fma(alpha, pv[u], xv[u]);
        r[i] = ri;
      }
      acc[0] = fma(ri, ri, acc[0]);
    }
  }
  block_sum<1>(acc, sh);
  if (threadIdx.x == 0) partial_rr[blockIdx.x] = acc[0];
}

__global__ void cg_loop_check_kernel(cudaGraphConditionalHandle cond, CgScalars* sc) {
  const int it = sc->it + 1;
  sc->it = it;
  const double rr = sc->rr, lim = sc->rtol * sc->nb;
  const bool more = !sc->flag && isfinite(rr) && rr > lim * lim && it < sc->max_it;
  cudaGraphSetConditional(cond, more ? 1u : 0u);
}

__global__ void cg_loop_init_kernel(CgScalars* sc, int it, int max_it, double nb, double rtol) {
  sc->it = it;
  sc->max_it = max_it;
  sc->nb = nb;
  sc->rtol = rtol;
}

__global__ void cast_d2f_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  VPS_CHUNKS(i0, n) {
    double v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = i0 + u * kThreads;
      v[u] = i < n ? a[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = i0 + u * kThreads;
      if (i < n) b[i] = d2f_rn(v[u]);
    }
  }
}

__global__ void cast_f2d_kernel(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = f2d(a[i]);
}

// Diagnostic: the conversions of fp_bits.cuh against the hardware ones on
// bit patterns pat[i] (low 32 bits as a float, all 64 as a double).
// bad[0]: f2d differs from the cast; bad[1]: d2f_rn differs from the cast
// (NaNs compare as equal); bad[2]: split_f2 breaks its contract.
__global__ void check_fp_bits_kernel(const unsigned long long* __restrict__ pat, int64_t n,
                                     unsigned long long* __restrict__ bad) {
  unsigned long long nb[3] = {0ull, 0ull, 0ull};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long b = pat[i];
    const float f = __uint_as_float((unsigned)b);
    const double d = __longlong_as_double((long long)b);
    const double x = f2d(f), xr = (double)f;
    if (isnan(xr) ? !isnan(x) : __double_as_longlong(x) != __double_as_longlong(xr)) ++nb[0];
    const float y = d2f_rn(d), yr = (float)d;
    if (isnan(yr) ? !isnan(y) : __float_as_uint(y) != __float_as_uint(yr)) ++nb[1];
    float hi, lo;
    split_f2(d, hi, lo);
    bool ok = true;
    const unsigned E = (unsigned)(b >> 52) & 0x7ffu;
    if (d == 0.0) {
      ok = __float_as_uint(hi) == __float_as_uint(lo) && signbit(hi) == signbit(d) &&
           hi == 0.0f;
    } else if (E - 950u < 201u) {
      const double t = (d - (double)hi) - (double)lo;  // both differences are exact
      const double ulp = ldexp(1.0, ilogbf(hi) - 23);
      ok = fabs(t) < ldexp(fabs(d), -47) && signbit(hi) == signbit(d) &&
           (lo == 0.0f || signbit(lo) == signbit(d)) && fabs((double)hi) <= fabs(d) &&
           fabs((double)lo) < ulp && fabs(d - (double)hi) < ulp;
    } else if (!isnan(d)) {
      const float h2 = (float)d, l2 = (float)(d - (double)h2);
      ok = __float_as_uint(hi) == __float_as_uint(h2) &&
           (isnan(l2) ? isnan(lo) : __float_as_uint(lo) == __float_as_uint(l2));
    }
    if (!ok) ++nb[2];
  }
  for (int j = 0; j < 3; ++j)
    if (nb[j]) atomicAdd(bad + j, nb[j]);
}

template <typename T>
__global__ void axpy_kernel(T* __restrict__ y, const T* __restrict__ x, T a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}

// b[c] = sum_m prod_t b1d[(mode*dim + t)*ni + j_t]
__global__ void rhs_tensor_kernel(const double* __restrict__ b1d, double* __restrict__ b, int dim,
                                  int ni, int n_modes, int64_t ncomp) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncomp;
       c += (int64_t)gridDim.x * blockDim.x) {
    int64_t j[3];
    j[0] = c % ni;
    j[1] = (c / ni) % ni;
    j[2] = dim == 3 ? c / ((int64_t)ni * ni) : 0;
    double s = 0.0;
    for (int md = 0; md < n_modes; ++md) {
      double p = 1.0;
      for (int t = 0; t < dim; ++t) p *= b1d[(int64_t)(md * dim + t) * ni + j[t]];
      s += p;
    }
    b[c] = s;
  }
}

// Squared L2 error contributions: one thread per (cell, Gauss point).
// tab: [ (k+1)*q basis values V[a][qq] | q points | q weights ] (FP64).
__global__ void __launch_bounds__(kThreads)
l2_partial_kernel(const double* __restrict__ x, const double* __restrict__ tab, int dim, int k,
                  int q, int ncell, int64_t px, int64_t pz, double h, double* __restrict__ partial) {
  __shared__ double sh[2 * kThreads];
  const int nl = k + 1;
  const double* V = tab;
  const double* xq = tab + nl * q;
  const double* wq = xq + q;
  const int64_t qd = dim == 3 ? (int64_t)q * q * q : (int64_t)q * q;
  const int64_t cells = dim == 3 ? (int64_t)ncell * ncell * ncell : (int64_t)ncell * ncell;
  const int64_t work = cells * qd;
  double acc[2] = {0.0, 0.0};
  for (int64_t e = blockIdx.x * (int64_t)kThreads + threadIdx.x; e < work;
       e += (int64_t)kDotBlocks * kThreads) {
    const int64_t cell = e / qd;
    const int64_t qi = e % qd;
    int qa[3] = {(int)(qi % q), (int)((qi / q) % q), dim == 3 ? (int)(qi / ((int64_t)q * q)) : 0};
    int64_t ca[3] = {cell % ncell, (cell / ncell) % ncell, dim == 3 ? cell / ((int64_t)ncell * ncell) : 0};
    double uh = 0.0;
    const int na = dim == 3 ? nl * nl * nl : nl * nl;
    for (int a = 0; a < na; ++a) {
      const int a0 = a % nl, a1 = (a / nl) % nl, a2 = a / (nl * nl);
      double phi = V[a0 * q + qa[0]] * V[a1 * q + qa[1]];
      int64_t idx = (k * ca[0] + a0) + (k * ca[1] + a1) * px;
      if (dim == 3) {
        phi *= V[a2 * q + qa[2]];
        idx += (k * ca[2] + a2) * pz;
      }
      uh = fma(phi, x[idx], uh);
    }
    double u = 1.0, w = 1.0;
    for (int t = 0; t < dim; ++t) {
      u *= sin(M_PI * (ca[t] + xq[qa[t]]) * h);
      w *= wq[qa[t]] * h;
    }
    const double d = uh - u;
    acc[0] = fma(w * d, d, acc[0]);
  }
  block_sum<2>(acc, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = acc[0];
    partial[kDotBlocks + blockIdx.x] = 0.0;
  }
}

// One pass of the global fast diagonalisation: for every line L of the
// ni^(d-1) lines along the slowest index c,
//   out[L][o] = sum_c in[c][L] W[c][o]   (scaled: times inv[L][o]),
// i.e. the product In^T W of an (ni x NL) and an (ni x ni) matrix, written
// with o fastest (the next pass contracts the next direction).  The work
// tensors between passes hold rows of NLp = fd_pad(NL) elements (in[c][L] at
// c NLp + L) and the weights rows of fd_pad(ni) (zero past ni), so a block
// stages its tiles with 16-byte asynchronous copies (the first pass reads the
// level layout element by element).  A block computes FD_TL lines x TO
// outputs with the whole contraction length in shared memory (ni <= 255);
// each of its 128 threads owns 2 lines x TO/16 outputs.  Two tile widths,
// chosen per coarse level by the autotuner: TO = 32 (2 x 2 per thread, twice
// the blocks: small or FP64 problems) and TO = 64 (2 x 4, 8 FMAs per pair of
// shared loads; all outputs of a line for ni <= 64).
constexpr int FD_TL = 16, FD_RL = 2, FD_THREADS = 128;


// One element global -> shared without staging in registers; with valid
// false the element is filled with zeros and nothing is read (src is then
// only a placeholder address inside the source buffer).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int sz = valid ? (int)sizeof(T) : 0;
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(sz)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(sz)
                 : "memory");
}

// 16 bytes global -> shared (both 16-byte aligned), zero-filled when !valid.
__device__ __forceinline__ void cp_async_16(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int sz = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(sz)
               : "memory");
}

// N consecutive elements from shared memory, p aligned to N elements
// (16 bytes at most per access).
template <typename T, int N>
__device__ __forceinline__ void lds_vec(const T* p, T (&v)[N]) {
  if constexpr (sizeof(T) == 4 && N == 2) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    v[0] = q.x; v[1] = q.y;
  } else if constexpr (sizeof(T) == 4 && N == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
#pragma unroll
    for (int i = 0; i < N; i += 2) {
      const double2 q = *reinterpret_cast<const double2*>(p + i);
      v[i] = q.x; v[i + 1] = q.y;
    }
  }
}

// One FD_TL x FD_TO tile (lines L0.., outputs o0..) of a pass.
template <typename T, int FD_TO>
__device__ __forceinline__ void fd_pass_tile(const T* __restrict__ in, T* __restrict__ out,
                                             const T* __restrict__ W, const T* __restrict__ inv,
                                             bool scale, int ni, int dim, int in_lev, int out_lev,
                                             int px, int pz, int L0, int o0, T* As, T* Bs) {
  constexpr int V = 16 / (int)sizeof(T);  // elements per 16-byte copy
  const int NL = dim == 3 ? ni * ni : ni, NLp = fd_pad(NL), nip = fd_pad(ni);
  for (int u = threadIdx.x; u < ni * (FD_TO / V); u += FD_THREADS) {
    const int c = u / (FD_TO / V), o = o0 + (u % (FD_TO / V)) * V;
    cp_async_16(Bs + c * FD_TO + (o - o0), o < nip ? W + ((size_t)c * nip + o) : W, o < nip);
  }
  if (in_lev) {
    for (int u = threadIdx.x; u < ni * FD_TL; u += FD_THREADS) {
      const int l = u % FD_TL, c = u / FD_TL, L = L0 + l;
      const T* src = in;
      if (L < NL) {
        const int a = dim == 3 ? L / ni : 0, bb = dim == 3 ? L % ni : L;
        src = dim == 3 ? in + ((c + 1) * pz + (a + 1) * px + bb + 1) : in + ((c + 1) * px + bb + 1);
      }
      cp_async_elem(As + u, src, L < NL);
    }
  } else {
    for (int u = threadIdx.x; u < ni * (FD_TL / V); u += FD_THREADS) {
      const int c = u / (FD_TL / V), L = L0 + (u % (FD_TL / V)) * V;
      cp_async_16(As + c * FD_TL + (L - L0), L < NLp ? in + ((size_t)c * NLp + L) : in, L < NLp);
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  constexpr int FD_RO = FD_TO / 16;
  static_assert((FD_TL / FD_RL) * (FD_TO / FD_RO) == FD_THREADS, "one output tile per thread");
  const int tl = threadIdx.x % (FD_TL / FD_RL), to = threadIdx.x / (FD_TL / FD_RL);
  T acc[FD_RL][FD_RO];
#pragma unroll
  for (int i = 0; i < FD_RL; ++i)
#pragma unroll
    for (int j = 0; j < FD_RO; ++j) acc[i][j] = T(0);
#pragma unroll 4
  for (int c = 0; c < ni; ++c) {
    T av[FD_RL], bv[FD_RO];
    lds_vec(As + c * FD_TL + FD_RL * tl, av);
    lds_vec(Bs + c * FD_TO + FD_RO * to, bv);
#pragma unroll
    for (int i = 0; i < FD_RL; ++i)
#pragma unroll
      for (int j = 0; j < FD_RO; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
  }
#pragma unroll
  for (int i = 0; i < FD_RL; ++i) {
    const int L = L0 + FD_RL * tl + i;
    if (L >= NL) continue;
    const int a = dim == 3 ? L / ni : L, bb = dim == 3 ? L % ni : 0;
#pragma unroll
    for (int j = 0; j < FD_RO; ++j) {
      const int o = o0 + FD_RO * to + j;
      if (o >= ni) continue;
      T r = acc[i][j];
      if (scale) r *= inv[(size_t)L * ni + o];
      if (out_lev) {
        if (dim == 3) out[(a + 1) * pz + (bb + 1) * px + o + 1] = r;
        else out[(L + 1) * px + o + 1] = r;
      } else {
        out[(size_t)a * NLp + bb * ni + o] = r;
      }
    }
  }
}

template <typename T, int MODE, int FD_TO>
__global__ void __launch_bounds__(FD_THREADS, 8)
fd_global_pass_kernel(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ W,
                      const T* __restrict__ inv, int ni, int dim, int in_lev, int out_lev, int px,
                      int pz) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* As = reinterpret_cast<T*>(smem_raw);  // [ni][FD_TL]
  T* Bs = As + (size_t)ni * FD_TL;         // [ni][FD_TO]
  fd_pass_tile<T, FD_TO>(in, out, W, inv, MODE == 1, ni, dim, in_lev, out_lev, px, pz,
                         blockIdx.x * FD_TL, blockIdx.y * FD_TO, As, Bs);
}

// Grid-wide barrier of a cooperative launch (every block resident): the last
// block to arrive resets the count and advances the generation; the others
// poll the generation at most `limit` times, then record the expiry in *err
// and go on (the result is then undefined, the memory accesses are not).
__device__ __forceinline__ void grid_barrier(const GridSync& gs) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned g;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(g) : "l"(gs.gen) : "memory");
    __threadfence();
    if (atomicAdd(gs.count, 1u) == gridDim.x - 1) {
      *gs.count = 0u;
      __threadfence();
      asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(gs.gen), "r"(g + 1u) : "memory");
    } else {
      unsigned polls = 0, cur;
      for (;;) {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(cur) : "l"(gs.gen) : "memory");
        if (cur != g) break;
        if ((polls & 31u) == 31u && *reinterpret_cast<volatile const int*>(gs.err)) break;
        if (++polls >= gs.limit) {
          atomicOr(gs.err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
  }
  __syncthreads();
}

// The whole exact coarse solve x = A^-1 b by global fast diagonalisation in
// one cooperative launch: the passes of launch_fd_global_pass (S^T along
// each direction, the last of them scaled by 1/(sum of eigenvalues), then S
// along each), separated by grid barriers instead of kernel boundaries;
// every block takes the pass's tiles in a grid-stride loop.  x is zeroed
// (boundary and padding) during the first pass; its interior is written by
// the last.
template <typename T, int FD_TO>
__global__ void __launch_bounds__(FD_THREADS, 8)
fd_global_solve_kernel(const T* __restrict__ b, T* __restrict__ x, const T* __restrict__ S,
                       const T* __restrict__ St, const T* __restrict__ inv, T* __restrict__ t1,
                       T* __restrict__ t2, int ni, int dim, int px, int pz, int64_t xtotal,
                       GridSync gs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* As = reinterpret_cast<T*>(smem_raw);
  T* Bs = As + (size_t)ni * FD_TL;
  const int NL = dim == 3 ? ni * ni : ni;
  const int gx = (NL + FD_TL - 1) / FD_TL, gy = (ni + FD_TO - 1) / FD_TO;
  const int ntiles = gx * gy;
  const int npass = dim == 3 ? 6 : 4;
  for (int64_t e = blockIdx.x * (int64_t)FD_THREADS + threadIdx.x; e < xtotal;
       e += (int64_t)gridDim.x * FD_THREADS)
    x[e] = T(0);
  for (int p = 0; p < npass; ++p) {
    // 3D: b->t1 (S^T), t1->t2 (S^T), t2->t1 (S^T, scaled), t1->t2 (S), t2->t1 (S), t1->x (S)
    // 2D: b->t1 (S^T), t1->t2 (S^T, scaled), t2->t1 (S), t1->x (S)
    const int half = npass / 2;
    const T* in = p == 0 ? b : ((p & 1) ? t1 : t2);
    T* out = p == npass - 1 ? x : ((p & 1) ? t2 : t1);
    const T* W = p < half ? S : St;
    const bool scale = p == half - 1;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      fd_pass_tile<T, FD_TO>(in, out, W, inv, scale, ni, dim, p == 0, p == npass - 1, px, pz,
                             (tile % gx) * FD_TL, (tile / gx) * FD_TO, As, Bs);
      __syncthreads();  // the next tile reloads As and Bs
    }
    if (p < npass - 1) grid_barrier(gs);
  }
}

}  // namespace

template <typename T, int FD_TO>
cudaError_t fd_global_pass_launch(int mode, const T* in, T* out, const T* W, const T* inv, int ni,
                                  int dim, bool in_lev, bool out_lev, int px, int pz,
                                  cudaStream_t s) {
  const int NL = dim == 3 ? ni * ni : ni;
  const dim3 grid((unsigned)((NL + FD_TL - 1) / FD_TL), (unsigned)((ni + FD_TO - 1) / FD_TO));
  const size_t smem = (size_t)ni * (FD_TL + FD_TO) * sizeof(T);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  auto kern = mode == 0 ? fd_global_pass_kernel<T, 0, FD_TO>
                        : (mode == 1 ? fd_global_pass_kernel<T, 1, FD_TO>
                                     : fd_global_pass_kernel<T, 2, FD_TO>);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  VPS_COUNT_LAUNCH();
  kern<<<grid, FD_THREADS, smem, s>>>(in, out, W, inv, ni, dim, in_lev, out_lev, px, pz);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fd_global_pass(int mode, const T* in, T* out, const T* W, const T* inv, int ni,
                                  int dim, bool in_lev, bool out_lev, int px, int pz, bool wide,
                                  cudaStream_t s) {
  return wide ? fd_global_pass_launch<T, 64>(mode, in, out, W, inv, ni, dim, in_lev, out_lev, px,
                                             pz, s)
              : fd_global_pass_launch<T, 32>(mode, in, out, W, inv, ni, dim, in_lev, out_lev, px,
                                             pz, s);
}

template <typename T, int FD_TO>
cudaError_t fd_global_solve_launch(const T* b, T* x, const T* S, const T* St, const T* inv, T* t1,
                                   T* t2, int ni, int dim, int px, int pz, int64_t xtotal,
                                   const GridSync& gs, cudaStream_t s) {
  const int NL = dim == 3 ? ni * ni : ni;
  const int ntiles = ((NL + FD_TL - 1) / FD_TL) * ((ni + FD_TO - 1) / FD_TO);
  const size_t smem = (size_t)ni * (FD_TL + FD_TO) * sizeof(T);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  auto kern = fd_global_solve_kernel<T, FD_TO>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FD_THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::min(ntiles, per_sm * nsm);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(FD_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  VPS_COUNT_LAUNCH();
  return cudaLaunchKernelEx(&cfg, kern, b, x, S, St, inv, t1, t2, ni, dim, px, pz, xtotal, gs);
}

template <typename T>
cudaError_t launch_fd_global_solve(const T* b, T* x, const T* S, const T* St, const T* inv, T* t1,
                                   T* t2, int ni, int dim, int px, int pz, int64_t xtotal,
                                   const GridSync& gs, bool wide, cudaStream_t s) {
  return wide ? fd_global_solve_launch<T, 64>(b, x, S, St, inv, t1, t2, ni, dim, px, pz, xtotal,
                                              gs, s)
              : fd_global_solve_launch<T, 32>(b, x, S, St, inv, t1, t2, ni, dim, px, pz, xtotal,
                                              gs, s);
}

template cudaError_t launch_fd_global_solve<float>(const float*, float*, const float*, const float*,
                                                   const float*, float*, float*, int, int, int, int,
                                                   int64_t, const GridSync&, bool, cudaStream_t);
template cudaError_t launch_fd_global_solve<double>(const double*, double*, const double*,
                                                    const double*, const double*, double*, double*,
                                                    int, int, int, int, int64_t, const GridSync&,
                                                    bool, cudaStream_t);

template cudaError_t launch_fd_global_pass<float>(int, const float*, float*, const float*,
                                                  const float*, int, int, bool, bool, int, int,
                                                  bool, cudaStream_t);
template cudaError_t launch_fd_global_pass<double>(int, const double*, double*, const double*,
                                                   const double*, int, int, bool, bool, int, int,
                                                   bool, cudaStream_t);

template <typename T>
cudaError_t launch_pack(const LevelGeom& g, const T* compact, T* lev, cudaStream_t s) {
  VPS_COUNT_LAUNCH();
  pack_kernel<T><<<grid_for(g.total, 4), kThreads, 0, s>>>(compact, lev, g.dim, g.n1, g.px, g.pz,
                                                            g.total);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_unpack(const LevelGeom& g, const T* lev, T* compact, cudaStream_t s) {
  const int64_t ni = g.n1 - 2;
  const int64_t nc = g.dim == 3 ? ni * ni * ni : ni * ni;
  VPS_COUNT_LAUNCH();
  unpack_kernel<T><<<grid_for(nc, 4), kThreads, 0, s>>>(lev, compact, g.dim, g.n1, g.px, g.pz, nc);
  return cudaGetLastError();
}

cudaError_t launch_dot1(const double* a, const double* b, int64_t n, double* partial, double* out,
                        cudaStream_t s) {
  VPS_COUNT_LAUNCH();
  dot_partial_kernel<double, 1><<<kDotBlocks, kThreads, 0, s>>>(a, b, nullptr, n, partial);
  VPS_COUNT_LAUNCH();
  dot_final_kernel<<<1, kThreads, 0, s>>>(partial, out, 1);
  return cudaGetLastError();
}

cudaError_t launch_multi_dot(const double* V, int64_t ld, int nv, const double* w, int64_t n,
                             double* partial, double* out, cudaStream_t s) {
  VPS_COUNT_LAUNCH();
  multi_dot_partial_kernel<<<dim3(kDotBlocks, nv), kThreads, 0, s>>>(V, ld, w, n, partial);
  VPS_COUNT_LAUNCH();
  multi_dot_final_kernel<<<nv, kThreads, 0, s>>>(partial, out);
  return cudaGetLastError();
}

cudaError_t launch_multi_axpy(double* w, const double* V, int64_t ld, int nv, const double* c,
                              double sign, int64_t n, cudaStream_t s) {
  VPS_COUNT_LAUNCH();
  multi_axpy_kernel<<<grid_for(n, 4), kThreads, 0, s>>>(w, V, ld, nv, c, sign, n);
  return cudaGetLastError();
}

cudaError_t launch_scale(double* y, const double* x, double a, int64_t n, cudaStream_t s) {
  VPS_COUNT_LAUNCH();
  scale_kernel<<<grid_for(n, 4), kThreads, 0, s>>>(y, x, a, n);
  return cudaGetLastError();
}


template <typename TZ>
cudaError_t launch_cg_start(double* p, double* z, const TZ* zn, const double* r, int64_t n,
                            double* partial, CgScalars* sc, cudaStream_t s, float* ph,
                            float* pl) {
  VPS_COUNT_LAUNCH();
  cg_init_p_kernel<TZ>
      <<<grid_for(n, kU), kThreads, 0, s>>>(p, reinterpret_cast<TZ*>(z), zn, ph, pl, n);
  VPS_COUNT_LAUNCH();
  dot_partial_kernel<TZ, 1><<<kDotBlocks, kThreads, 0, s>>>(r, zn, nullptr, n, partial);
  VPS_COUNT_LAUNCH();
  dot_final_kernel<<<1, kThreads, 0, s>>>(partial, &sc->rzn, 1);
  return cudaGetLastError();
}

template <typename TZ>
cudaError_t launch_cg_next_p(double* p, double* z, const TZ* zn, const double* r, int64_t n,
                             double* partial, CgScalars* sc, cudaStream_t s, float* ph,
                             float* pl) {
  VPS_COUNT_LAUNCH();
  TZ* zo = reinterpret_cast<TZ*>(z);  // z_old in the type of z_new
  dot_partial_kernel<TZ, 2><<<kDotBlocks, kThreads, 0, s>>>(r, zn, zo, n, partial);
  VPS_COUNT_LAUNCH();
  // kDotBlocks blocks: every block reduces the partials once
  cg_update_p_fused_kernel<TZ><<<kDotBlocks, kThreads, 0, s>>>(p, zo, zn, partial, sc, ph, pl, n);
  return cudaGetLastError();
}

cudaError_t launch_cg_step_xr(double* x, double* r, const double* p, const double* Ap, int64_t n,
                              double* partial, double* partial2, CgScalars* sc, cudaStream_t s) {
  VPS_COUNT_LAUNCH();
  dot_partial_kernel<double, 1><<<kDotBlocks, kThreads, 0, s>>>(p, Ap, nullptr, n, partial);
  VPS_COUNT_LAUNCH();
  cg_update_xr_fused_kernel<<<kDotBlocks, kThreads, 0, s>>>(x, r, p, Ap, partial, sc, partial2, n);
  VPS_COUNT_LAUNCH();
  dot_final_kernel<<<1, kThreads, 0, s>>>(partial2, &sc->rr, 1);
  return cudaGetLastError();
}

template cudaError_t launch_cg_start<float>(double*, double*, const float*, const double*, int64_t,
                                            double*, CgScalars*, cudaStream_t, float*, float*);
template cudaError_t launch_cg_start<double>(double*, double*, const double*, const double*,
                                             int64_t, double*, CgScalars*, cudaStream_t, float*,
                                             float*);
template cudaError_t launch_cg_next_p<float>(double*, double*, const float*, const double*, int64_t,
                                             double*, CgScalars*, cudaStream_t, float*, float*);
template cudaError_t launch_cg_next_p<double>(double*, double*, const double*, const double*,
                                              int64_t, double*, CgScalars*, cudaStream_t, float*,
                                              float*);

cudaError_t launch_split_df(const double* a, float* ph, float* pl, int64_t n, cudaStream_t s) {
  VPS_COUNT_LAUNCH();
  split_df_kernel<<<grid_for(n, kU), kThreads, 0, s>>>(a, ph, pl, n);
  return cudaGetLastError();
}

cudaError_t launch_cg_loop_check(cudaGraphConditionalHandle cond, CgScalars* sc, cudaStream_t s) {
  VPS_COUNT_LAUNCH();
  cg_loop_check_kernel<<<1, 1, 0, s>>>(cond, sc);
  return cudaGetLastError();
}

cudaError_t launch_cg_loop_init(CgScalars* sc, int it, int max_it, double nb, double rtol,
                                cudaStream_t s) {
  VPS_COUNT_LAUNCH();
  cg_loop_init_kernel<<<1, 1, 0, s>>>(sc, it, max_it, nb, rtol);
  return cudaGetLastError();
}

cudaError_t launch_cast_d2f(const double* a, float* b, int64_t n, cudaStream_t s) {
  VPS_COUNT_LAUNCH();
  cast_d2f_kernel<<<grid_for(n, kU), kThreads, 0, s>>>(a, b, n);
  return cudaGetLastError();
}

cudaError_t launch_cast_f2d(const float* a, double* b, int64_t n, cudaStream_t s) {
  VPS_COUNT_LAUNCH();
  cast_f2d_kernel<<<grid_for(n, 4), kThreads, 0, s>>>(a, b, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_axpy_inplace(T* y, const T* x, T a, int64_t n, cudaStream_t s) {
  VPS_COUNT_LAUNCH();
  axpy_kernel<T><<<grid_for(n, 4), kThreads, 0, s>>>(y, x, a, n);
  return cudaGetLastError();
}

cudaError_t launch_rhs_tensor(const LevelGeom& g, int n_modes, const double* b1d, double* b,
                              cudaStream_t s) {
  const int64_t ni = g.n1 - 2;
  const int64_t nc = g.dim == 3 ? ni * ni * ni : ni * ni;
  VPS_COUNT_LAUNCH();
  rhs_tensor_kernel<<<grid_for(nc, 4), kThreads, 0, s>>>(b1d, b, g.dim, (int)ni, n_modes, nc);
  return cudaGetLastError();
}

cudaError_t launch_l2_error_sine(const LevelGeom& g, const double* xlev, const double* tab, int q,
                                 double* partial, double* out, cudaStream_t s) {
  VPS_COUNT_LAUNCH();
  l2_partial_kernel<<<kDotBlocks, kThreads, 0, s>>>(xlev, tab, g.dim, g.k, q, g.ncell, g.px, g.pz,
                                                     g.h, partial);
  VPS_COUNT_LAUNCH();
  dot_final_kernel<<<1, kThreads, 0, s>>>(partial, out, 1);
  return cudaGetLastError();
}

template cudaError_t launch_pack<float>(const LevelGeom&, const float*, float*, cudaStream_t);
template cudaError_t launch_pack<double>(const LevelGeom&, const double*, double*, cudaStream_t);
template cudaError_t launch_unpack<float>(const LevelGeom&, const float*, float*, cudaStream_t);
template cudaError_t launch_unpack<double>(const LevelGeom&, const double*, double*, cudaStream_t);
template cudaError_t launch_axpy_inplace<float>(float*, const float*, float, int64_t, cudaStream_t);
template cudaError_t launch_axpy_inplace<double>(double*, const double*, double, int64_t,
                                                 cudaStream_t);

}  // namespace vps

extern "C" int vps_check_fp_conversions(const void* patterns, int64_t n, int64_t* mismatches,
                                        void* cuda_stream) {
  using namespace vps;
  set_thread_error("");
  char buf[256];
  if (!mismatches || n < 0 || (n > 0 && !patterns)) {
    set_thread_error("mismatches must be non-NULL, n >= 0, patterns non-NULL if n > 0");
    return VPS_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  unsigned long long* bad = nullptr;
  unsigned long long host[3] = {0ull, 0ull, 0ull};
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&bad), sizeof(host), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(host), s);
  if (e == cudaSuccess && n > 0) {
    check_fp_bits_kernel<<<grid_for(n, 4), kThreads, 0, s>>>(
        static_cast<const unsigned long long*>(patterns), n, bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, bad, sizeof(host), cudaMemcpyDeviceToHost, s);
  if (bad) {
    const cudaError_t e2 = cudaFreeAsync(bad, s);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    snprintf(buf, sizeof(buf), "vps_check_fp_conversions: %s", cudaGetErrorString(e));
    set_thread_error(buf);
    return VPS_ECUDA;
  }
  for (int j = 0; j < 3; ++j) mismatches[j] = (int64_t)host[j];
  return VPS_OK;
}

// ------------------------------------------------------- FMA throughput
namespace vps {
namespace {

// Sink of the throughput kernel: written only when the accumulators take a
// value they never take, so that the compiler keeps every multiply-add.
__device__ double g_fma_sink;

constexpr int kFmaChains = 8;   // independent accumulators per thread
constexpr int kFmaUnroll = 16;  // multiply-adds per chain and loop trip

// kFmaChains x kFmaUnroll dependent-free multiply-adds per trip: x = x a + c
// with |a| < 1, so the values stay bounded.  Every multiply-add is one FMA
// instruction of the type's pipe.
template <typename T>
__global__ void __launch_bounds__(256) fma_throughput_kernel(int trips, T a, T c) {
  T x[kFmaChains];
#pragma unroll
  for (int j = 0; j < kFmaChains; ++j) x[j] = (T)(threadIdx.x + j);
  for (int i = 0; i < trips; ++i) {
#pragma unroll
    for (int u = 0; u < kFmaUnroll; ++u)
#pragma unroll
      for (int j = 0; j < kFmaChains; ++j) x[j] = fma(x[j], a, c);
  }
  T s = T(0);
#pragma unroll
  for (int j = 0; j < kFmaChains; ++j) s += x[j];
  if (s == (T)-1.2345e30) g_fma_sink = (double)s;
}

}  // namespace
}  // namespace vps

extern "C" int vps_fma_peak(int precision, double* flops_per_s, double* seconds,
                            int* sm_count, void* cuda_stream) {
  using namespace vps;
  set_thread_error("");
  char buf[256];
  if (!flops_per_s || (precision != VPS_FP32 && precision != VPS_FP64)) {
    set_thread_error("vps_fma_peak: flops_per_s must be non-NULL, precision VPS_FP32 or VPS_FP64");
    return VPS_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // 8 blocks of 256 threads per SM (2048 threads: every warp slot busy);
  // trips chosen for tens of milliseconds per launch
  const int blocks = 8 * (sms > 0 ? sms : 1);
  const int trips = precision == VPS_FP32 ? 16384 : 512;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.0f;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {  // launch 0 warms up
    if (rep > 0) e = cudaEventRecord(e0, s);
    if (e != cudaSuccess) break;
    if (precision == VPS_FP32)
      fma_throughput_kernel<float><<<blocks, 256, 0, s>>>(trips, 0.9999999f, 1e-7f);
    else
      fma_throughput_kernel<double><<<blocks, 256, 0, s>>>(trips, 0.9999999, 1e-7);
    VPS_COUNT_LAUNCH();
    e = cudaGetLastError();
    if (e == cudaSuccess && rep > 0) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess && rep > 0) e = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (e == cudaSuccess && rep > 0) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess && rep > 0 && (ms == 0.0f || t < ms)) ms = t;  // best of two
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess || !(ms > 0.0f)) {
    snprintf(buf, sizeof(buf), "vps_fma_peak: %s",
             e != cudaSuccess ? cudaGetErrorString(e) : "no time measured");
    set_thread_error(buf);
    return VPS_ECUDA;
  }
  const double flops = 2.0 * blocks * 256.0 * trips * kFmaUnroll * kFmaChains;
  *flops_per_s = flops / (ms * 1e-3);
  if (seconds) *seconds = ms * 1e-3;
  if (sm_count) *sm_count = sms;
  return VPS_OK;
}
