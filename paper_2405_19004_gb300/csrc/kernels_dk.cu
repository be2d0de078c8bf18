// Hot-path kernels for one (dimension, degree) pair.
//
// This file is compiled once per pair with -DVPS_DIM=<2|3> -DVPS_K=<1..7>;
// each object registers its entry points in the library's kernel registry.
// Every 1D matrix lives in this unit's __constant__ memory and is indexed
// with compile-time offsets only (all contraction loops are unrolled), so
// the multiply-adds take their matrix operand straight from the constant
// bank and shared memory only carries tensor data.
//
// Kernels
//  * smooth_mult  -- one colour of the multiplicative vertex-patch smoother
//                    (Algorithm 3, the "Fused" kernel of Section 3.1.3): per
//                    patch, gather the closure x and interior b, local
//                    residual r = b - Abar x by sum factorisation with the
//                    reuse of Section 3.1.1, local solve by fast
//                    diagonalisation (Eq. 2.13/2.14), interior update.
//  * smooth_add   -- one colour of the additive smoother from a global
//                    residual (fast diagonalisation only).
//  * apply        -- y = A x or r = b - A x: the operator as a Kronecker sum
//                    of banded global 1D matrices (Section 2.3, Cartesian
//                    mesh), evaluated on output tiles without atomics.
//  * prolong_add / restrict_ -- tensor-product interpolation and its
//                    transpose (Section 2.1), per coarse-cell tile.
//
// Shared-memory layouts.  A contraction stage reads a tensor whose slowest
// index is the contracted one, in[c][L], and writes out[L][o]: the output's
// slowest index is then the next direction to contract, so directions
// rotate z -> y -> x without transposes.  With P patches per block the
// patch index is the fastest index ([c][L][p]); P is a power of two, so
// for both 4- and 8-byte words every warp access is free of bank conflicts
// (the odd extents 2k+1 and 2k-1 keep the strided writes conflict free).
#include <cmath>
#include <cstdio>

#include "fp_bits.cuh"
#include "vps_internal.h"

#ifndef VPS_DIM
#error "compile with -DVPS_DIM=2|3"
#endif
#ifndef VPS_K
#error "compile with -DVPS_K=1..7"
#endif

namespace vps {
namespace {

constexpr int DIM = VPS_DIM;
constexpr int K = VPS_K;
constexpr int n = 2 * K + 1;   // patch closure nodes per direction
constexpr int m = 2 * K - 1;   // patch interior nodes per direction
constexpr int nl = K + 1;      // nodes per cell and direction
// Even/odd split (reflection about the patch centre): a closure line of n =
// 2K+1 values has K+1 even parts e_c = x_c + x_{n-1-c} (c < K), e_K = x_K and
// K odd parts d_c = x_c - x_{n-1-c}; an interior line of m = 2H+1 values has
// H+1 even and H odd parts (centre H).
constexpr int H = K - 1;
constexpr int KE = K + 1;
constexpr int HE = H + 1;
constexpr int HO = H > 0 ? H : 1;   // array extent of the odd parts (none for K = 1)

template <typename T>
struct DevTab {
  T Ap[m * n];
  T Mp[m * n];
  T S[m * m];
  // Halves of the centrosymmetric interior rows of Mp, Ap (W[m-1-o][n-1-c] =
  // W[o][c]): WE[o][c] = (W[o][c] + W[o][n-1-c]) / 2 (c < K), WE[o][K] =
  // W[o][K], o = 0..H; WO[o][c] = (W[o][c] - W[o][n-1-c]) / 2, o < H, c < K.
  // Then (W x)_o = E_o + O_o, (W x)_{m-1-o} = E_o - O_o with E_o = WE[o] . e,
  // O_o = WO[o] . d (O_H = 0).
  T MpE[HE * KE];
  T MpO[HO * K];
  T ApE[HE * KE];
  T ApO[HO * K];
  // Halves of S, whose first H+1 columns are even and last H odd
  // eigenvectors: SE[c][a] = S[c][a] (c, a <= H), SO[c][a] = S[c][H+1+a]
  // (c, a < H).
  T SE[HE * HE];
  T SO[HO * HO];
  T Kb[K * n];
  T Mb[K * n];
  T P1[n * nl];
  // low words of Kb, Mb (FP32 table only): Kb + Kb_lo is the FP64 value to
  // about 48 bits, for the double-float operator
  T Kb_lo[K * n];
  T Mb_lo[K * n];
};

template <typename T>
__constant__ DevTab<T> c_tab;

// |Kb|, |Mb| in FP64: the absolute-value operator |K|x|M|x|M| + ... that
// bounds the rounding error of an evaluation of A x (FP64 residual checks)
struct AbsTab {
  double Kb[K * n];
  double Mb[K * n];
};
__constant__ AbsTab c_abs;

// Band coefficients of the operator (ABS: their absolute values, FP64 only).
template <typename T, bool ABS>
__device__ __forceinline__ T coefK(int i) {
  if constexpr (ABS) return (T)c_abs.Kb[i];
  else return c_tab<T>.Kb[i];
}
template <typename T, bool ABS>
__device__ __forceinline__ T coefM(int i) {
  if constexpr (ABS) return (T)c_abs.Mb[i];
  else return c_tab<T>.Mb[i];
}

// Programmatic dependent launch (launch_pdl): let the next kernel of the
// stream be scheduled as this one's blocks start, and wait until every
// earlier kernel has completed and its writes are visible.  Both are no-ops
// for a kernel launched without the attribute.
__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

// ---------------------------------------------------------------- config
// ------------------------------------------------------------- smoother
// A block holds P = G * Q patches.  In every contraction stage thread t
// handles line L = t / G of the Q patches g*Q .. g*Q+Q-1 (g = t % G): each
// coefficient (constant memory) and each address is shared by Q FMAs, and
// the Q values of a tensor entry are adjacent in shared memory (patch index
// fastest), so they move as one vector access.  With G and Q powers of two
// and the odd extents 2k+-1, every warp access is free of bank conflicts.
// Block shapes (the autotuner picks one per level): shape s has kShapeG[s]
// patch groups of kShapeQ[s] patches per thread.  G is chosen so that the
// G n^2, G n m and G m^2 lines of the 3D stages (G n and G m in 2D) nearly
// fill whole warps -- a stage whose lines leave most of a warp idle costs
// the same issue slots and shared-memory wavefronts as a full one -- within
// 1024 threads: 3D k = 4 fills 88-98 % of the lanes with G = 4 against
// 77-98 % with one patch per block.
constexpr int kLinesMax = DIM == 3 ? n * n : n;
constexpr int kG1 = DIM == 3 ? (K == 1 ? 32 : K == 2 ? 16 : K == 3 ? 8 : K <= 5 ? 4 : 2)
                             : (K <= 6 ? 32 : 16);
constexpr int kG2 = DIM == 3 ? (K == 1 ? 16 : K == 2 ? 32 : K == 3 ? 16 : K <= 5 ? 8 : 4)
                             : (K <= 6 ? 16 : 32);
constexpr int kShapeG[kQVariants] = {kG1, kG1, kG2};
constexpr int kShapeQ[kQVariants] = {1, 2, 1};
// Fewest warps of a block of shape s that still covers the lines of the
// residual stage after the first (3D: G n m, 2D: G m) in one round (kinds 3
// and 4): the first stage, whose G n^2 (2D: G n) lines are the most, takes
// two rounds, and the threads that every later stage leaves idle are not
// launched.  A block then holds fewer registers (3D Q4 FP32: 256 threads
// instead of 352 at 32 registers), so more blocks -- and patches -- are
// resident on an SM.
constexpr int warps_min(int s) {
  return (kShapeG[s] * (DIM == 3 ? n * m : m) + 31) / 32;
}
// Contract the first and the middle direction of the fast diagonalisation in
// registers (two stages and two barriers fewer); above k = 5 the extra live
// values cost more resident blocks than the barriers save.
constexpr bool kFuseFD = K <= 5;
// Blocks of one warp (variants 6-8) only for k <= 3: measured faster at
// k = 1 and never faster from k = 4 on, where their many unrolled rounds of
// 32 lines dominated the compile time.
constexpr bool kOneWarpVariants = K <= 3;

template <class T, int Q>
struct alignas(sizeof(T) * Q) Pack {
  T v[Q];
};

// W_ = 0: enough warps for every line of the first stage in one round
// (at most 1024 threads); W_ > 0: W_ warps, each stage in several rounds
// (one-warp blocks wait at their barriers for no other warp).
template <typename T, int S_, int W_ = 0>
struct SmoothCfg {
  static constexpr int G = kShapeG[S_], Q = kShapeQ[S_], P = G * Q;
  static constexpr int NT0 = ((G * kLinesMax + 31) / 32) * 32;
  static constexpr int NT = W_ > 0 ? 32 * W_ : (NT0 > 1024 ? 1024 : NT0);
  static constexpr int md = DIM == 3 ? m * m * m : m * m;
  // interleaved buffers [..][p] (elements):
  //   3D: A0, A1 = n n m P (stage-0 outputs), B0, B1 = n m m P (stage-1
  //       outputs), F0, F1 (stage-2 output and the fast-diagonalisation
  //       ping-pong, md P each), bI, xI = md P, il = md.
  //       With `alias` (blocks that run every stage in one round of lines)
  //       stage 1 reads its lines into registers and crosses a barrier
  //       before it writes, so B0, B1 overlay A0, A1; F0 follows them and F1
  //       overlays B0: one region of max(2 n n m, 2 n m m + md) P elements
  //       (3D Q4: 6.3 KB per patch in FP32 instead of 10.8 KB).  Otherwise
  //       F0 = A0, F1 = A1.
  //   2D: A0, A1 = n m P, B0 = m m P (residual), bI, xI = md P, il = md
  static constexpr int sizeA = DIM == 3 ? n * n * m : n * m;
  static constexpr int sizeB = DIM == 3 ? n * m * m : m * m;
  static constexpr int nB = DIM == 3 ? 2 : 1;
  // (stage 1 reads its line into registers before a barrier: one round)
  static constexpr bool alias = DIM == 3 && (W_ == 0 || 32 * W_ >= G * n * m);
  static constexpr int region =
      alias ? (2 * sizeA > 2 * sizeB + md ? 2 * sizeA : 2 * sizeB + md) : 2 * sizeA + nB * sizeB;
  static constexpr size_t elems_mult = (size_t)P * (region + 2 * md) + md;
  static constexpr size_t smem_mult = sizeof(T) * elems_mult + sizeof(int) * P;
  // Boundary kernel: no staged copy of the interior of x
  static constexpr size_t smem_bnd = smem_mult - sizeof(T) * (size_t)P * md;
  static constexpr size_t smem_add = sizeof(T) * ((size_t)P * 2 * md + md) + sizeof(int) * P;
  static constexpr bool fits = smem_mult <= 227 * 1024 && G * kLinesMax <= 1024;
  static constexpr bool fits_bnd = smem_bnd <= 227 * 1024 && G * kLinesMax <= 1024;
};

// Calls f(t) for every line t = threadIdx.x + r * NT < TOTAL, with the
// rounds r unrolled at compile time (no loop control per line).
template <int TOTAL, int NT, class F>
__device__ __forceinline__ void for_lines(F&& f) {
  constexpr int R = (TOTAL + NT - 1) / NT;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int t = (int)threadIdx.x + r * NT;
    if (TOTAL % NT == 0 || t < TOTAL) f(t);
  }
}

// Offset of the first closure node of patch gp of a colour (int: every
// level vector holds fewer than 2^31 elements).
__device__ __forceinline__ int closure_origin(int gp, const ColourGeom& cg, int px, int pz) {
  const int i0 = gp % cg.cnt[0];
  const int r = gp / cg.cnt[0];
  const int i1 = r % cg.cnt[1];
  const int i2 = r / cg.cnt[1];
  const int o0 = K * (cg.par[0] + 2 * i0);
  const int o1 = K * (cg.par[1] + 2 * i1);
  const int o2 = DIM == 3 ? K * (cg.par[2] + 2 * i2) : 0;
  return o0 + o1 * px + o2 * pz;
}

// Origins of the block's P patches (-1: beyond the colour), computed once;
// P may exceed the block's NT threads (2D, k = 1, 2 patches per thread).
template <int P, int NT>
__device__ __forceinline__ void load_origins(int* s_org, const ColourGeom& cg, int px, int pz,
                                             int64_t tile) {
  for (int i = threadIdx.x; i < P; i += NT) {
    const int64_t gp = tile * P + i;
    s_org[i] = gp < cg.npatch ? closure_origin((int)gp, cg, px, pz) : -1;
  }
}

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// Asynchronous element copy global -> shared (cp.async, sizes 4 or 8 bytes).
template <typename T>
__device__ __forceinline__ void async_copy(T* dst, const T* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_addr(dst)), "l"(src),
               "n"((int)sizeof(T)));
}
__device__ __forceinline__ void async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::);
}

struct NoWait {
  __device__ void operator()() const {}
};

// ------------------------------------------------- even/odd contractions
// Coefficients of the halves of Mp (MAT 0) and Ap (MAT 1).
template <typename T, int MAT>
__device__ __forceinline__ T coefE(int i) {
  if constexpr (MAT == 0) return c_tab<T>.MpE[i];
  else return c_tab<T>.ApE[i];
}
template <typename T, int MAT>
__device__ __forceinline__ T coefO(int i) {
  if constexpr (MAT == 0) return c_tab<T>.MpO[i];
  else return c_tab<T>.ApO[i];
}

// Even and odd parts of a closure line x[0..n-1].
template <typename T, int Q>
__device__ __forceinline__ void split_closure(const T (&x)[n][Q], T (&e)[KE][Q], T (&d)[K][Q]) {
#pragma unroll
  for (int c = 0; c < K; ++c)
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      e[c][j] = x[c][j] + x[n - 1 - c][j];
      d[c][j] = x[c][j] - x[n - 1 - c][j];
    }
#pragma unroll
  for (int j = 0; j < Q; ++j) e[K][j] = x[K][j];
}

// acc += (interior row o of W's even half) . e   (o <= H)
template <typename T, int Q, int MAT>
__device__ __forceinline__ void row_even(int o, const T (&e)[KE][Q], T (&acc)[Q]) {
#pragma unroll
  for (int c = 0; c <= K; ++c) {
    const T w = coefE<T, MAT>(o * KE + c);
#pragma unroll
    for (int j = 0; j < Q; ++j) acc[j] = fma(w, e[c][j], acc[j]);
  }
}
// acc += (interior row o of W's odd half) . d   (o < H)
template <typename T, int Q, int MAT>
__device__ __forceinline__ void row_odd(int o, const T (&d)[K][Q], T (&acc)[Q]) {
#pragma unroll
  for (int c = 0; c < K; ++c) {
    const T w = coefO<T, MAT>(o * K + c);
#pragma unroll
    for (int j = 0; j < Q; ++j) acc[j] = fma(w, d[c][j], acc[j]);
  }
}

// t = S^T x for an interior line: the even eigen-components t[0..H] from the
// even parts of x, the odd ones t[H+1..m-1] from the odd parts.
template <typename T, int Q>
__device__ __forceinline__ void st_line(const T (&x)[m][Q], T (&t)[m][Q]) {
  T e[HE][Q], d[HO][Q];
#pragma unroll
  for (int c = 0; c < H; ++c)
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      e[c][j] = x[c][j] + x[m - 1 - c][j];
      d[c][j] = x[c][j] - x[m - 1 - c][j];
    }
#pragma unroll
  for (int j = 0; j < Q; ++j) e[H][j] = x[H][j];
#pragma unroll
  for (int a = 0; a <= H; ++a) {
#pragma unroll
    for (int j = 0; j < Q; ++j) t[a][j] = T(0);
#pragma unroll
    for (int c = 0; c <= H; ++c) {
      const T w = c_tab<T>.SE[c * HE + a];
#pragma unroll
      for (int j = 0; j < Q; ++j) t[a][j] = fma(w, e[c][j], t[a][j]);
    }
  }
#pragma unroll
  for (int a = 0; a < H; ++a) {
#pragma unroll
    for (int j = 0; j < Q; ++j) t[HE + a][j] = T(0);
#pragma unroll
    for (int c = 0; c < H; ++c) {
      const T w = c_tab<T>.SO[c * HO + a];
#pragma unroll
      for (int j = 0; j < Q; ++j) t[HE + a][j] = fma(w, d[c][j], t[HE + a][j]);
    }
  }
}

// y = S t for a line in eigen-components: y_o = E_o + O_o and
// y_{m-1-o} = E_o - O_o (o < H), y_H = E_H, E from the even components,
// O from the odd ones.
template <typename T, int Q>
__device__ __forceinline__ void s_line(const T (&t)[m][Q], T (&y)[m][Q]) {
#pragma unroll
  for (int o = 0; o <= H; ++o) {
    T E[Q], O[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) E[j] = O[j] = T(0);
#pragma unroll
    for (int a = 0; a <= H; ++a) {
      const T w = c_tab<T>.SE[o * HE + a];
#pragma unroll
      for (int j = 0; j < Q; ++j) E[j] = fma(w, t[a][j], E[j]);
    }
    if (o < H) {
#pragma unroll
      for (int a = 0; a < H; ++a) {
        const T w = c_tab<T>.SO[o * HO + a];
#pragma unroll
        for (int j = 0; j < Q; ++j) O[j] = fma(w, t[HE + a][j], O[j]);
      }
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        y[o][j] = E[j] + O[j];
        y[m - 1 - o][j] = E[j] - O[j];
      }
    } else {
#pragma unroll
      for (int j = 0; j < Q; ++j) y[o][j] = E[j];
    }
  }
}

// One fast-diagonalisation contraction over interleaved tensors.
// MODE 0: out = S^T in, MODE 1: out = (S^T in) * il, MODE 2: out = S in.
template <typename T, int G, int Q, int NT, int MODE>
__device__ __forceinline__ void fd_stage(const T* __restrict__ in, T* __restrict__ out,
                                         const T* __restrict__ il) {
  constexpr int NL = DIM == 3 ? m * m : m;
  constexpr int P = G * Q;
  using PK = Pack<T, Q>;
  for_lines<G * NL, NT>([&](const int t) {
    const int L = t / G, g = t % G;
    const PK* src = reinterpret_cast<const PK*>(in + L * P + g * Q);
    T v[m][Q];
#pragma unroll
    for (int c = 0; c < m; ++c) {
      const PK pk = src[c * NL * G];
#pragma unroll
      for (int j = 0; j < Q; ++j) v[c][j] = pk.v[j];
    }
    T u[m][Q];
    if constexpr (MODE == 2) s_line<T, Q>(v, u);
    else st_line<T, Q>(v, u);
    PK* dst = reinterpret_cast<PK*>(out + L * m * P + g * Q);
#pragma unroll
    for (int o = 0; o < m; ++o) {
      PK r;
      const T sc = MODE == 1 ? il[L * m + o] : T(1);
#pragma unroll
      for (int j = 0; j < Q; ++j) r.v[j] = MODE == 1 ? u[o][j] * sc : u[o][j];
      dst[o * G] = r;
    }
  });
}

// S^T along the contracted direction, the scaling by 1/(sum of eigenvalues),
// and S back along the same direction, in registers (one stage instead of
// two: the directions of the fast diagonalisation may be taken in any order,
// and the scaling table is symmetric in its three indices).  SWAP: the
// output line index exchanges its two digits, so that the direction that
// was the faster one of the line becomes the slowest (contracted next).
template <typename T, int G, int Q, int NT, bool SWAP>
__device__ __forceinline__ void fd_pair(const T* __restrict__ in, T* __restrict__ out,
                                        const T* __restrict__ il) {
  constexpr int NL = DIM == 3 ? m * m : m;
  constexpr int P = G * Q;
  using PK = Pack<T, Q>;
  for_lines<G * NL, NT>([&](const int t) {
    const int L = t / G, g = t % G;
    const PK* src = reinterpret_cast<const PK*>(in + L * P + g * Q);
    T v[m][Q];
#pragma unroll
    for (int c = 0; c < m; ++c) {
      const PK pk = src[c * NL * G];
#pragma unroll
      for (int j = 0; j < Q; ++j) v[c][j] = pk.v[j];
    }
    T tt[m][Q];
    st_line<T, Q>(v, tt);
#pragma unroll
    for (int o = 0; o < m; ++o) {
      const T sc = il[L * m + o];
#pragma unroll
      for (int j = 0; j < Q; ++j) tt[o][j] *= sc;
    }
    T u[m][Q];
    s_line<T, Q>(tt, u);
    const int Lw = SWAP ? (L % m) * m + L / m : L;
    PK* dst = reinterpret_cast<PK*>(out + Lw * m * P + g * Q);
#pragma unroll
    for (int o = 0; o < m; ++o) {
      PK r;
#pragma unroll
      for (int j = 0; j < Q; ++j) r.v[j] = u[o][j];
      dst[o * G] = r;
    }
  });
}

// S along the last direction and the update of the interior:
// x_I = base + scale * u, base from the staged xI (xs) or from x itself;
// SET: x_I = scale * u.
template <typename T, int G, int Q, int NT, bool SET = false>
__device__ __forceinline__ void fd_final(const T* __restrict__ in, T* __restrict__ x,
                                         const T* xs, const int* s_org, int px, int pz, T scale) {
  constexpr int NL = DIM == 3 ? m * m : m;
  constexpr int P = G * Q;
  using PK = Pack<T, Q>;
  for_lines<G * NL, NT>([&](const int t) {
    const int L = t / G, g = t % G;
    const PK* src = reinterpret_cast<const PK*>(in + L * P + g * Q);
    T v[m][Q];
#pragma unroll
    for (int c = 0; c < m; ++c) {
      const PK pk = src[c * NL * G];
#pragma unroll
      for (int j = 0; j < Q; ++j) v[c][j] = pk.v[j];
    }
    int rowoff;
    if constexpr (DIM == 3) {
      const int zz = L / m, yy = L % m;
      rowoff = (zz + 1) * pz + (yy + 1) * px + 1;
    } else {
      rowoff = (L + 1) * px + 1;
    }
    T u[m][Q];
    s_line<T, Q>(v, u);
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      const int org = s_org[g * Q + j];
      if (org < 0) continue;
      T* dst = x + org + rowoff;
#pragma unroll
      for (int o = 0; o < m; ++o) {
        if constexpr (SET) {
          dst[o] = scale * u[o][j];
        } else {
          const T base = xs ? xs[(L * m + o) * P + g * Q + j] : dst[o];
          dst[o] = fma(scale, u[o][j], base);
        }
      }
    }
  });
}

// Prefetch of the interior of b (scaled later) into the interleaved layout
// [z][y][x][p] by the threads that consume it in the residual stage.
template <typename T, int G, int Q, int NT>
__device__ __forceinline__ void prefetch_b(const T* __restrict__ b, T* bI, const int* s_org,
                                           int px, int pz) {
  constexpr int NL = DIM == 3 ? m * m : m;
  constexpr int P = G * Q;
  for_lines<G * NL, NT>([&](const int t) {
    const int L = t / G, g = t % G;
    int rowoff;
    if constexpr (DIM == 3) {
      rowoff = (L / m + 1) * pz + (L % m + 1) * px + 1;
    } else {
      rowoff = (L + 1) * px + 1;
    }
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      const int org = s_org[g * Q + j];
      T* d = bI + L * m * P + g * Q + j;
      if (org >= 0) {
        const T* srow = b + org + rowoff;
#pragma unroll
        for (int o = 0; o < m; ++o) async_copy(d + o * P, srow + o);
      } else {
#pragma unroll
        for (int o = 0; o < m; ++o) d[o * P] = T(0);
      }
    }
  });
}

// Writes the interleaved interior tensor buf[(L * m + o) * P + p] of the
// block's patches to the level vector out (times scale): the local residual
// of the Separate kernel.
template <typename T, int G, int Q, int NT>
__device__ __forceinline__ void store_lines(const T* __restrict__ buf, T* __restrict__ out,
                                            const int* s_org, int px, int pz, T scale) {
  constexpr int NL = DIM == 3 ? m * m : m;
  constexpr int P = G * Q;
  for_lines<G * NL, NT>([&](const int t) {
    const int L = t / G, g = t % G;
    int rowoff;
    if constexpr (DIM == 3) rowoff = (L / m + 1) * pz + (L % m + 1) * px + 1;
    else rowoff = (L + 1) * px + 1;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      const int org = s_org[g * Q + j];
      if (org < 0) continue;
      T* dst = out + org + rowoff;
#pragma unroll
      for (int o = 0; o < m; ++o) dst[o] = scale * buf[(L * m + o) * P + g * Q + j];
    }
  });
}

// ------------------------------------------------------- multiplicative
// Closure lines along the first contracted direction, in the order the
// Boundary kernel assigns them to threads: the 8K lines on the faces of the
// other directions first (2D: the 2 lines at x = 0, 2K), then the interior
// lines, which meet the patch boundary only at their two end nodes.
// Returns the layout index of the line; *full: all its nodes are boundary
// nodes of the patch.
__device__ __forceinline__ int boundary_first_line(int L, bool* full) {
  if constexpr (DIM == 3) {
    constexpr int nb = 2 * n + 2 * m;  // = 8K
    int yy, xx;
    if (L < n) {
      yy = 0; xx = L;
    } else if (L < 2 * n) {
      yy = n - 1; xx = L - n;
    } else if (L < nb) {
      const int r = L - 2 * n;
      yy = 1 + r / 2; xx = (r & 1) ? n - 1 : 0;
    } else {
      const int r = L - nb;
      yy = 1 + r / m; xx = 1 + r % m;
    }
    *full = L < nb;
    return yy * n + xx;
  } else {
    *full = L < 2;
    return L == 0 ? 0 : (L == 1 ? n - 1 : L - 1);
  }
}

// BND = false: the fused kernel, x_I += A_j^-1 (b_I - Abar x) (Algorithm 3).
// BND = true: the Boundary kernel, x_I = A_j^-1 (b_I - A^IB x_B) (Section
// 3.2), equal for the exact local solver: the interior of x is neither read
// nor staged, and lines of the first contraction that run through the
// patch interior contract only their two end (boundary) nodes.
// RES = true (with the fused layout): the first half of the Separate kernel
// of Section 3.1 -- the local residual b_I - Abar_j x of every patch of the
// colour is written to rout (physical units, scaled back by 1 / bscale) and
// x is left unchanged.
//
// The body processes tile `tile` of the colour (patches tile*P .. tile*P+P-1);
// smooth_mult_kernel runs tile blockIdx.x, smooth_mult_batch_kernel the
// tiles it takes from a queue of several levels' colour passes.
//
// SW = true (the dataflow sweep): x changes under the kernel (other blocks
// update it).  `wait`, the tile's dependency wait, runs first; its acquire
// loads and the barrier after the prologue order every thread's loads of x
// after the release of the patches it waited for, so they observe those
// updates (the memory model's acquire, which also covers data the SM's L1
// cached earlier).
template <typename T, int QQ, bool BND, int W, bool RES = false, bool SW = false,
          class WaitF = NoWait>
__device__ __forceinline__ void smooth_mult_body(const T* __restrict__ b, T* __restrict__ x,
                                                 const T* __restrict__ inv_lam, int px, int pz,
                                                 const ColourGeom& cg, T bscale,
                                                 T* __restrict__ rout, int64_t tile,
                                                 const WaitF& wait = WaitF()) {
  static_assert(!(RES && BND), "the residual-only kernel reads the whole closure");
  using C = SmoothCfg<T, QQ, W>;
  constexpr int G = C::G, Q = C::Q, P = C::P, NT = C::NT, MD = C::md;
  using PK = Pack<T, Q>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool kAlias = C::alias;
  T* const base = reinterpret_cast<T*>(smem_raw);
  T* A0 = base;
  T* A1 = A0 + P * C::sizeA;
  T* B0 = kAlias ? base : A1 + P * C::sizeA;
  T* F0 = kAlias ? base + 2 * P * C::sizeB : A0;
  T* F1 = kAlias ? base : A1;
  T* bI = base + (size_t)P * C::region;
  T* xI = BND ? nullptr : bI + P * MD;
  T* il = bI + (BND ? 1 : 2) * P * MD;
  int* s_org = reinterpret_cast<int*>(il + MD);
  if constexpr (SW) wait();
  // the origins and the eigenvalue table (written at setup) do not depend
  // on the previous kernel: read them before waiting for it to complete
  load_origins<P, NT>(s_org, cg, px, pz, tile);
  if constexpr (!RES)
    for (int e = threadIdx.x; e < MD; e += NT) il[e] = __ldg(inv_lam + e);
  grid_dependency_wait();
  __syncthreads();
  prefetch_b<T, G, Q, NT>(b, bI, s_org, px, pz);

  if constexpr (DIM == 3) {
    T* B1 = B0 + P * C::sizeB;
    // Stage 0: z-lines of the closure from global memory; M x and A x along
    // z (interior rows) into [y][x][oz]; the interior of x is kept in xI.
    for_lines<G * n * n, NT>([&](const int t) {
      int L = t / G;
      const int g = t % G;
      bool full = true;
      if constexpr (BND) L = boundary_first_line(L, &full);
      const int yy = L / n, xx = L % n;
      PK* dM = reinterpret_cast<PK*>(A0 + L * m * P + g * Q);
      PK* dA = reinterpret_cast<PK*>(A1 + L * m * P + g * Q);
      if (BND && !full) {
        // interior line: the patch interior of x counts as zero
        T v0[Q], v1[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          const int org = s_org[g * Q + j];
          const T* src = x + (org >= 0 ? org : 0) + yy * px + xx;
          v0[j] = org >= 0 ? src[0] : T(0);
          v1[j] = org >= 0 ? src[(n - 1) * pz] : T(0);
        }
#pragma unroll
        for (int o = 0; o < m; ++o) {
          PK am, aa;
#pragma unroll
          for (int j = 0; j < Q; ++j) {
            am.v[j] = fma(c_tab<T>.Mp[o * n + n - 1], v1[j], c_tab<T>.Mp[o * n] * v0[j]);
            aa.v[j] = fma(c_tab<T>.Ap[o * n + n - 1], v1[j], c_tab<T>.Ap[o * n] * v0[j]);
          }
          dM[o * G] = am;
          dA[o * G] = aa;
        }
        return;
      }
      T v[n][Q];
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        const int org = s_org[g * Q + j];
        const T* src = x + (org >= 0 ? org : 0) + yy * px + xx;
#pragma unroll
        for (int c = 0; c < n; ++c) v[c][j] = org >= 0 ? src[c * pz] : T(0);
      }
      if (!BND && yy >= 1 && yy <= m && xx >= 1 && xx <= m) {
        PK* d = reinterpret_cast<PK*>(xI + ((yy - 1) * m + xx - 1) * P + g * Q);
#pragma unroll
        for (int c = 1; c <= m; ++c) {
          PK pk;
#pragma unroll
          for (int j = 0; j < Q; ++j) pk.v[j] = v[c][j];
          d[(c - 1) * m * m * G] = pk;
        }
      }
      // M x and A x on the interior rows, by the even/odd halves
      T ev[KE][Q], od[K][Q];
      split_closure<T, Q>(v, ev, od);
#pragma unroll
      for (int o = 0; o <= H; ++o) {
        T em[Q], ea[Q], om[Q], oa[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) em[j] = ea[j] = om[j] = oa[j] = T(0);
        row_even<T, Q, 0>(o, ev, em);
        row_even<T, Q, 1>(o, ev, ea);
        if (o < H) {
          row_odd<T, Q, 0>(o, od, om);
          row_odd<T, Q, 1>(o, od, oa);
        }
        PK m0, m1, a0, a1;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          m0.v[j] = em[j] + om[j];
          m1.v[j] = em[j] - om[j];
          a0.v[j] = ea[j] + oa[j];
          a1.v[j] = ea[j] - oa[j];
        }
        dM[o * G] = m0;
        dA[o * G] = a0;
        if (o < H) {
          dM[(m - 1 - o) * G] = m1;
          dA[(m - 1 - o) * G] = a1;
        }
      }
    });
    __syncthreads();
    // Stage 1: along y.  U = M (M x), W = A (M x) + M (A x)  (the inner sum
    // M x along z is shared by two terms, Section 3.1.1).
    constexpr int NL1 = n * m;
    // with kAlias, B0/B1 overlay A0/A1: every line is read into registers
    // before the barrier, written after it (one round: NT >= G n m)
    static_assert(!kAlias || NT >= G * NL1, "aliased stage 1 needs one round of lines");
    const bool act1 = !kAlias || (int)threadIdx.x < G * NL1;
    T vm[n][Q], va[n][Q];
    auto load1 = [&](const int t) {
      const int L = t / G, g = t % G;
      const PK* sM = reinterpret_cast<const PK*>(A0 + L * P + g * Q);
      const PK* sA = reinterpret_cast<const PK*>(A1 + L * P + g * Q);
#pragma unroll
      for (int c = 0; c < n; ++c) {
        const PK a = sM[c * NL1 * G], bb = sA[c * NL1 * G];
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          vm[c][j] = a.v[j];
          va[c][j] = bb.v[j];
        }
      }
    };
    if constexpr (kAlias) {
      if (act1) load1(threadIdx.x);
      __syncthreads();
    }
    for_lines<G * NL1, NT>([&](const int t) {
      const int L = t / G, g = t % G;
      if constexpr (!kAlias) load1(t);
      PK* dU = reinterpret_cast<PK*>(B0 + L * m * P + g * Q);
      PK* dW = reinterpret_cast<PK*>(B1 + L * m * P + g * Q);
      T em[KE][Q], dm[K][Q], ea[KE][Q], da[K][Q];
      split_closure<T, Q>(vm, em, dm);
      split_closure<T, Q>(va, ea, da);
#pragma unroll
      for (int o = 0; o <= H; ++o) {
        T eu[Q], ew[Q], ou[Q], ow[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) eu[j] = ew[j] = ou[j] = ow[j] = T(0);
        row_even<T, Q, 0>(o, em, eu);
        row_even<T, Q, 1>(o, em, ew);
        row_even<T, Q, 0>(o, ea, ew);
        if (o < H) {
          row_odd<T, Q, 0>(o, dm, ou);
          row_odd<T, Q, 1>(o, dm, ow);
          row_odd<T, Q, 0>(o, da, ow);
        }
        PK u0, u1, w0, w1;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          u0.v[j] = eu[j] + ou[j];
          u1.v[j] = eu[j] - ou[j];
          w0.v[j] = ew[j] + ow[j];
          w1.v[j] = ew[j] - ow[j];
        }
        dU[o * G] = u0;
        dW[o * G] = w0;
        if (o < H) {
          dU[(m - 1 - o) * G] = u1;
          dW[(m - 1 - o) * G] = w1;
        }
      }
    });
    async_wait_all();
    __syncthreads();
    // Stage 2: along x.  r = bscale * b - (A U + M W) on the interior, into A0.
    constexpr int NL2 = m * m;
    for_lines<G * NL2, NT>([&](const int t) {
      const int L = t / G, g = t % G;
      const PK* sU = reinterpret_cast<const PK*>(B0 + L * P + g * Q);
      const PK* sW = reinterpret_cast<const PK*>(B1 + L * P + g * Q);
      T vu[n][Q], vw[n][Q];
#pragma unroll
      for (int c = 0; c < n; ++c) {
        const PK a = sU[c * NL2 * G], bb = sW[c * NL2 * G];
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          vu[c][j] = a.v[j];
          vw[c][j] = bb.v[j];
        }
      }
      const PK* sb = reinterpret_cast<const PK*>(bI + L * m * P + g * Q);
      constexpr bool kKeep = !RES && kFuseFD;  // keep the line for S^T along x
      PK* dR = reinterpret_cast<PK*>(F0 + L * m * P + g * Q);
      T rr[kKeep ? m : 1][Q];
      // A vu + M vw on the interior rows, by the even/odd halves
      T ex[KE][Q], dx[K][Q], ey[KE][Q], dy[K][Q];
      split_closure<T, Q>(vu, ex, dx);
      split_closure<T, Q>(vw, ey, dy);
#pragma unroll
      for (int o = 0; o <= H; ++o) {
        T E[Q], O[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) E[j] = O[j] = T(0);
        row_even<T, Q, 1>(o, ex, E);
        row_even<T, Q, 0>(o, ey, E);
        if (o < H) {
          row_odd<T, Q, 1>(o, dx, O);
          row_odd<T, Q, 0>(o, dy, O);
        }
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          if (side == 1 && o == H) continue;
          const int oo = side == 0 ? o : m - 1 - o;
          const PK bv = sb[oo * G];
          T acc[Q];
#pragma unroll
          for (int j = 0; j < Q; ++j) acc[j] = side == 0 ? E[j] + O[j] : E[j] - O[j];
          if constexpr (kKeep) {
#pragma unroll
            for (int j = 0; j < Q; ++j) rr[oo][j] = fma(bscale, bv.v[j], -acc[j]);
          } else {  // the residual itself, [z][y][x]
            PK r;
#pragma unroll
            for (int j = 0; j < Q; ++j) r.v[j] = fma(bscale, bv.v[j], -acc[j]);
            dR[oo * G] = r;
          }
        }
      }
      if constexpr (kKeep) {
        // first direction of the fast diagonalisation in registers: S^T along
        // x, written as [y][z][x'] (y contracted next)
        const int Ls = (L % m) * m + L / m;
        PK* dT = reinterpret_cast<PK*>(F0 + Ls * m * P + g * Q);
        T tt[m][Q];
        st_line<T, Q>(rr, tt);
#pragma unroll
        for (int o = 0; o < m; ++o) {
          PK pk;
#pragma unroll
          for (int j = 0; j < Q; ++j) pk.v[j] = tt[o][j];
          dT[o * G] = pk;
        }
      }
    });
    __syncthreads();
    if constexpr (RES) {
      store_lines<T, G, Q, NT>(F0, rout, s_org, px, pz, T(1) / bscale);
      return;
    }
    if constexpr (kFuseFD) {
      // Rest of the fast diagonalisation (Eq. 2.14): S^T along y; S^T along z,
      // the eigenvalue scaling and S along z in one stage; S along y; S along x
      // with the update of the interior.
      fd_stage<T, G, Q, NT, 0>(F0, F1, nullptr);  // [y][z][x'] -> [z][x'][y']
      __syncthreads();
      fd_pair<T, G, Q, NT, true>(F1, F0, il);     // [z][x'][y'] -> [y'][x'][z'']
      __syncthreads();
      fd_stage<T, G, Q, NT, 2>(F0, F1, nullptr);  // [y'][x'][z''] -> [x'][z''][y'']
      __syncthreads();
    } else {
      // S^T along z, y, x (scaled), then S along z, y; S along x below
      fd_stage<T, G, Q, NT, 0>(F0, F1, nullptr);
      __syncthreads();
      fd_stage<T, G, Q, NT, 0>(F1, F0, nullptr);
      __syncthreads();
      fd_stage<T, G, Q, NT, 1>(F0, F1, il);
      __syncthreads();
      fd_stage<T, G, Q, NT, 2>(F1, F0, nullptr);
      __syncthreads();
      fd_stage<T, G, Q, NT, 2>(F0, F1, nullptr);
      __syncthreads();
    }
    fd_final<T, G, Q, NT, BND>(F1, x, xI, s_org, px, pz, T(1));
  } else {
    // 2D.  Stage 0: lines along y from global; M x and A x along y into [x][oy].
    for_lines<G * n, NT>([&](const int t) {
      int L = t / G;
      const int g = t % G;
      bool full = true;
      if constexpr (BND) L = boundary_first_line(L, &full);
      if (BND && !full) {
        // interior line (x in 1..m): only its two end nodes in y are boundary nodes
        T v0[Q], v1[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          const int org = s_org[g * Q + j];
          const T* src = x + (org >= 0 ? org : 0) + L;
          v0[j] = org >= 0 ? src[0] : T(0);
          v1[j] = org >= 0 ? src[(n - 1) * px] : T(0);
        }
        PK* dM = reinterpret_cast<PK*>(A0 + L * m * P + g * Q);
        PK* dA = reinterpret_cast<PK*>(A1 + L * m * P + g * Q);
#pragma unroll
        for (int o = 0; o < m; ++o) {
          PK am, aa;
#pragma unroll
          for (int j = 0; j < Q; ++j) {
            am.v[j] = fma(c_tab<T>.Mp[o * n + n - 1], v1[j], c_tab<T>.Mp[o * n] * v0[j]);
            aa.v[j] = fma(c_tab<T>.Ap[o * n + n - 1], v1[j], c_tab<T>.Ap[o * n] * v0[j]);
          }
          dM[o * G] = am;
          dA[o * G] = aa;
        }
        return;
      }
      T v[n][Q];
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        const int org = s_org[g * Q + j];
        const T* src = x + (org >= 0 ? org : 0) + L;
#pragma unroll
        for (int c = 0; c < n; ++c) v[c][j] = org >= 0 ? src[c * px] : T(0);
      }
      if (!BND && L >= 1 && L <= m) {
        PK* d = reinterpret_cast<PK*>(xI + (L - 1) * P + g * Q);
#pragma unroll
        for (int c = 1; c <= m; ++c) {
          PK pk;
#pragma unroll
          for (int j = 0; j < Q; ++j) pk.v[j] = v[c][j];
          d[(c - 1) * m * G] = pk;
        }
      }
      PK* dM = reinterpret_cast<PK*>(A0 + L * m * P + g * Q);
      PK* dA = reinterpret_cast<PK*>(A1 + L * m * P + g * Q);
      // M x and A x on the interior rows, by the even/odd halves
      T ev[KE][Q], od[K][Q];
      split_closure<T, Q>(v, ev, od);
#pragma unroll
      for (int o = 0; o <= H; ++o) {
        T em[Q], ea[Q], om[Q], oa[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) em[j] = ea[j] = om[j] = oa[j] = T(0);
        row_even<T, Q, 0>(o, ev, em);
        row_even<T, Q, 1>(o, ev, ea);
        if (o < H) {
          row_odd<T, Q, 0>(o, od, om);
          row_odd<T, Q, 1>(o, od, oa);
        }
        PK m0, m1, a0, a1;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          m0.v[j] = em[j] + om[j];
          m1.v[j] = em[j] - om[j];
          a0.v[j] = ea[j] + oa[j];
          a1.v[j] = ea[j] - oa[j];
        }
        dM[o * G] = m0;
        dA[o * G] = a0;
        if (o < H) {
          dM[(m - 1 - o) * G] = m1;
          dA[(m - 1 - o) * G] = a1;
        }
      }
    });
    async_wait_all();
    __syncthreads();
    // Stage 1: along x.  r = b - (A (M x) + M (A x)) on the interior, into B0.
    for_lines<G * m, NT>([&](const int t) {
      const int L = t / G, g = t % G;
      const PK* sM = reinterpret_cast<const PK*>(A0 + L * P + g * Q);
      const PK* sA = reinterpret_cast<const PK*>(A1 + L * P + g * Q);
      T vm[n][Q], va[n][Q];
#pragma unroll
      for (int c = 0; c < n; ++c) {
        const PK a = sM[c * m * G], bb = sA[c * m * G];
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          vm[c][j] = a.v[j];
          va[c][j] = bb.v[j];
        }
      }
      const PK* sb = reinterpret_cast<const PK*>(bI + L * m * P + g * Q);
      PK* dR = reinterpret_cast<PK*>(B0 + L * m * P + g * Q);
      constexpr bool kKeep = !RES && kFuseFD;  // keep the line for S^T along x
      T rr[kKeep ? m : 1][Q];
      // A vm + M va on the interior rows, by the even/odd halves
      T ex[KE][Q], dx[K][Q], ey[KE][Q], dy[K][Q];
      split_closure<T, Q>(vm, ex, dx);
      split_closure<T, Q>(va, ey, dy);
#pragma unroll
      for (int o = 0; o <= H; ++o) {
        T E[Q], O[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) E[j] = O[j] = T(0);
        row_even<T, Q, 1>(o, ex, E);
        row_even<T, Q, 0>(o, ey, E);
        if (o < H) {
          row_odd<T, Q, 1>(o, dx, O);
          row_odd<T, Q, 0>(o, dy, O);
        }
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          if (side == 1 && o == H) continue;
          const int oo = side == 0 ? o : m - 1 - o;
          const PK bv = sb[oo * G];
          T acc[Q];
#pragma unroll
          for (int j = 0; j < Q; ++j) acc[j] = side == 0 ? E[j] + O[j] : E[j] - O[j];
          if constexpr (kKeep) {
#pragma unroll
            for (int j = 0; j < Q; ++j) rr[oo][j] = fma(bscale, bv.v[j], -acc[j]);
          } else {  // the residual itself, [y][x]
            PK r;
#pragma unroll
            for (int j = 0; j < Q; ++j) r.v[j] = fma(bscale, bv.v[j], -acc[j]);
            dR[oo * G] = r;
          }
        }
      }
      if constexpr (kKeep) {  // S^T along x in registers, [y][x']
        T tt[m][Q];
        st_line<T, Q>(rr, tt);
#pragma unroll
        for (int o = 0; o < m; ++o) {
          PK pk;
#pragma unroll
          for (int j = 0; j < Q; ++j) pk.v[j] = tt[o][j];
          dR[o * G] = pk;
        }
      }
    });
    __syncthreads();
    if constexpr (RES) {
      store_lines<T, G, Q, NT>(B0, rout, s_org, px, pz, T(1) / bscale);
      return;
    }
    if constexpr (kFuseFD) {
      // S^T along y, scaling and S along y in one stage; then S along x with
      // the update of the interior
      fd_pair<T, G, Q, NT, false>(B0, A0, il);  // [y][x'] -> [x'][y'']
      __syncthreads();
    } else {
      fd_stage<T, G, Q, NT, 0>(B0, A0, nullptr);
      __syncthreads();
      fd_stage<T, G, Q, NT, 1>(A0, A1, il);
      __syncthreads();
      fd_stage<T, G, Q, NT, 2>(A1, A0, nullptr);
      __syncthreads();
    }
    fd_final<T, G, Q, NT, BND>(A0, x, xI, s_org, px, pz, T(1));
  }
}

template <typename T, int QQ, bool BND, int W, bool RES = false>
__global__ void __launch_bounds__(SmoothCfg<T, QQ, W>::NT)
smooth_mult_kernel(const T* __restrict__ b, T* __restrict__ x, const T* __restrict__ inv_lam,
                   int px, int pz, ColourGeom cg, T bscale, T* __restrict__ rout = nullptr) {
  smooth_mult_body<T, QQ, BND, W, RES>(b, x, inv_lam, px, pz, cg, bscale, rout, blockIdx.x);
}

// Takes the next tile of a batched launch from the queue (one atomic per
// tile, by thread 0) and finds the queue item it belongs to; returns false
// once every tile has been taken.  Tiles of one item are processed exactly
// as the single-level kernel processes its blocks, so a level's result does
// not depend on the other items of the launch or on which block ran a tile.
__device__ __forceinline__ bool next_batch_tile(BatchQueue* q, int64_t* tile, int* item) {
  __shared__ int64_t s_tile;
  __shared__ int s_item;
  if (threadIdx.x == 0) {
    const int64_t t = (int64_t)atomicAdd(&q->head, 1ull);
    const int ni = q->nitems;
    int it = 0;
    while (it + 1 < ni && q->items[it + 1].tile0 <= t) ++it;
    s_tile = t;
    s_item = it;
  }
  __syncthreads();
  *tile = s_tile;
  *item = s_item;
  const bool more = s_tile < q->ntiles;
  __syncthreads();  // s_tile / s_item are rewritten by the next call
  return more;
}

// Persistent multiplicative colour passes of several levels (one queue item
// per level: b, x, layout, colour, bscale): each block takes tiles until
// the queue is empty.
template <typename T, int QQ, bool BND, int W>
__global__ void __launch_bounds__(SmoothCfg<T, QQ, W>::NT)
smooth_mult_batch_kernel(BatchQueue* __restrict__ q, const T* __restrict__ inv_lam) {
  int64_t t;
  int it;
  while (next_batch_tile(q, &t, &it)) {
    const BatchItem& I = q->items[it];
    smooth_mult_body<T, QQ, BND, W, false>(static_cast<const T*>(I.in), static_cast<T*>(I.out),
                                           inv_lam, (int)I.pxa, (int)I.pza, I.cg, (T)I.bscale,
                                           nullptr, t - I.tile0);
    __syncthreads();  // the next tile reuses the shared memory
  }
}

// ------------------------------------------------------- dataflow sweep
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// The dependency wait of a tile of the sweep: until every patch of an
// earlier colour that overlaps a patch of the tile is done (its flag holds
// this sweep's epoch ep).  Two vertex patches overlap -- the interior of one
// meets the closure of the other -- exactly when their vertices differ by
// at most one in every direction, so each patch checks its 3^d - 1
// neighbouring vertices (one thread per neighbour).  A wait polls at most
// spin_limit times; on expiry it sets *err and returns (the step's values
// are then undefined, its memory accesses are not), and once *err is set
// every later wait returns at once.
template <int P, int NT>
__device__ __forceinline__ void sweep_wait(const SweepGeom& sg, int pos, int64_t tile,
                                           unsigned ep) {
  constexpr int NNB = DIM == 3 ? 26 : 8;
  const ColourGeom& cg = sg.cg[pos];
  for (int u = threadIdx.x; u < P * NNB; u += NT) {
    const int64_t gp = tile * P + u / NNB;
    if (gp >= cg.npatch) continue;
    int code = u % NNB;
    code += code >= NNB / 2 ? 1 : 0;  // offsets in {-1,0,1}^d without the centre
    int iv[3];
    iv[0] = (int)(gp % cg.cnt[0]);
    const int r = (int)(gp / cg.cnt[0]);
    iv[1] = r % cg.cnt[1];
    iv[2] = r / cg.cnt[1];
    int w[3], cn = 0;
    bool inside = true;
#pragma unroll
    for (int t = 0; t < DIM; ++t) {
      const int d = (t == 0 ? code : t == 1 ? code / 3 : code / 9) % 3 - 1;
      w[t] = cg.par[t] + 2 * iv[t] + 1 + d;  // vertex of the neighbour
      inside = inside && w[t] >= 1 && w[t] <= sg.ncell - 1;
      cn |= ((w[t] - 1) & 1) << t;
    }
    if (!inside) continue;
    const int pn = sg.pos_of[cn];
    if (pn >= pos) continue;  // a later colour of the sweep
    const ColourGeom& cc = sg.cg[pn];
    int64_t gq = 0;
#pragma unroll
    for (int t = DIM - 1; t >= 0; --t) gq = gq * cc.cnt[t] + (w[t] - 1 - cc.par[t]) / 2;
    const unsigned* f = sg.flags + sg.flag_off[cn] + gq;
    unsigned polls = 0;
    while (ld_acquire(f) != ep) {
      if ((polls & 31u) == 31u && *reinterpret_cast<volatile const int*>(sg.err)) break;
      if (++polls >= sg.spin_limit) {
        atomicOr(sg.err, 1);
        break;
      }
      __nanosleep(128);
    }
  }
}

// A multiplicative smoothing step of one level in one launch of one block
// per tile: each block takes the next tile of the sweep (one atomic
// increment, so tiles are taken in the order blocks start), waits for the
// tile's dependencies, runs the colour-pass body on it and marks its patches
// done.  A block waits only for tiles taken before its own, each by a block
// that is running or has finished, so the waits end.  (One block per tile
// rather than a loop over tiles in resident blocks: the loop kept values
// live across tiles and needed twice the registers.)  The last block to
// finish resets the counters for the next sweep and advances the epoch.
template <typename T, int QQ, bool BND, int W = 0>
__global__ void __launch_bounds__(SmoothCfg<T, QQ, W>::NT)
smooth_sweep_kernel(const T* __restrict__ b, T* __restrict__ x, const T* __restrict__ inv_lam,
                    int px, int pz, const __grid_constant__ SweepGeom sg, T bscale) {
  using C = SmoothCfg<T, QQ, W>;
  constexpr int P = C::P, NT = C::NT;
  __shared__ int64_t s_tile;
  __shared__ unsigned s_ep;
  grid_dependency_wait();  // the counters and x are written by earlier kernels
  if (threadIdx.x == 0) {
    s_ep = *reinterpret_cast<volatile const unsigned*>(&sg.ctr->epoch) + 1u;
    s_tile = (int64_t)atomicAdd(&sg.ctr->head, 1ull);
  }
  __syncthreads();
  const int64_t t = s_tile;
  const unsigned ep = s_ep;
  if (t < sg.tile_end[sg.ncol - 1]) {
    int pos = 0;
    while (t >= sg.tile_end[pos]) ++pos;
    const int64_t tile = t - (pos > 0 ? sg.tile_end[pos - 1] : 0);
    const ColourGeom& cg = sg.cg[pos];
    smooth_mult_body<T, QQ, BND, W, false, true>(
        b, x, inv_lam, px, pz, cg, bscale, nullptr, tile,
        [&] { sweep_wait<P, NT>(sg, pos, tile, ep); });
    __syncthreads();  // every store of the tile is issued
    // (a block of few warps may hold more patches than threads)
    for (int i = threadIdx.x; i < P; i += NT) {
      const int64_t gp = tile * P + i;
      if (gp < cg.npatch) {
        __threadfence();
        st_release(sg.flags + sg.flag_off[sg.colour[pos]] + gp, ep);
      }
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&sg.ctr->done, 1u) == gridDim.x - 1) {
      sg.ctr->head = 0ull;
      sg.ctr->done = 0u;
      __threadfence();
      *reinterpret_cast<volatile unsigned*>(&sg.ctr->epoch) = ep;
    }
  }
}

// ------------------------------------------------------------- additive
// x_I += scale * A_ref^-1 r_I for every patch of one colour.
template <typename T, int QQ>
__global__ void __launch_bounds__(SmoothCfg<T, QQ>::NT)
smooth_add_kernel(const T* __restrict__ r, T* __restrict__ x, const T* __restrict__ inv_lam,
                  int px, int pz, ColourGeom cg, T scale) {
  using C = SmoothCfg<T, QQ>;
  constexpr int G = C::G, Q = C::Q, P = C::P, NT = C::NT, MD = C::md;
  using PK = Pack<T, Q>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* X0 = reinterpret_cast<T*>(smem_raw);
  T* X1 = X0 + P * MD;
  T* il = X1 + P * MD;
  int* s_org = reinterpret_cast<int*>(il + MD);
  load_origins<P, NT>(s_org, cg, px, pz, blockIdx.x);
  for (int e = threadIdx.x; e < MD; e += NT) il[e] = __ldg(inv_lam + e);
  __syncthreads();
  constexpr int NL = DIM == 3 ? m * m : m;
  // first S^T contraction reads the interior residual lines from global
  for_lines<G * NL, NT>([&](const int t) {
    const int L = t / G, g = t % G;
    T v[m][Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      const int org = s_org[g * Q + j];
      const T* src;
      int stride;
      if constexpr (DIM == 3) {
        src = r + (org >= 0 ? org : 0) + pz + (L / m + 1) * px + 1 + L % m;
        stride = pz;
      } else {
        src = r + (org >= 0 ? org : 0) + px + 1 + L;
        stride = px;
      }
#pragma unroll
      for (int c = 0; c < m; ++c) v[c][j] = org >= 0 ? src[c * stride] : T(0);
    }
    PK* dst = reinterpret_cast<PK*>(X1 + L * m * P + g * Q);
    T u[m][Q];
    st_line<T, Q>(v, u);
#pragma unroll
    for (int o = 0; o < m; ++o) {
      PK pk;
#pragma unroll
      for (int j = 0; j < Q; ++j) pk.v[j] = u[o][j];
      dst[o * G] = pk;
    }
  });
  __syncthreads();
  if constexpr (DIM == 3) {
    fd_stage<T, G, Q, NT, 0>(X1, X0, nullptr);
    __syncthreads();
    fd_stage<T, G, Q, NT, 1>(X0, X1, il);
    __syncthreads();
    fd_stage<T, G, Q, NT, 2>(X1, X0, nullptr);
    __syncthreads();
    fd_stage<T, G, Q, NT, 2>(X0, X1, nullptr);
    __syncthreads();
    fd_final<T, G, Q, NT>(X1, x, nullptr, s_org, px, pz, scale);
  } else {
    fd_stage<T, G, Q, NT, 1>(X1, X0, il);
    __syncthreads();
    fd_stage<T, G, Q, NT, 2>(X0, X1, nullptr);
    __syncthreads();
    fd_final<T, G, Q, NT>(X1, x, nullptr, s_org, px, pz, scale);
  }
}

// ------------------------------------------------------ degree 1 (Q1)
// For k = 1 a vertex patch has a single interior DoF, its vertex (m = 1):
// the colour pass of the multiplicative smoother (Algorithm 3) is a
// 2^d-colour point Gauss-Seidel pass, x_v += A_vv^-1 (b - A x)_v.  A block
// first forms the 3^d stencil of the patch's interior row, the Kronecker
// sum of the interior rows of the patch matrices (Ap, Mp: 1 x 3), in
// shared memory; then one thread per patch of the colour evaluates the
// local residual over its 3^d closure (3^d multiply-adds) and applies the
// local solve of Eq. 2.14 with 1 x 1 factors, u = S^(2d) (d lambda)^-1 r.
// Without the stages, barriers and staging of the general kernel the FP32
// pass is bound by memory and the FP64 pass by its 3^d multiply-adds.
constexpr int kQ1Threads = 256;

template <typename T>
__global__ void __launch_bounds__(kQ1Threads)
smooth_q1_kernel(const T* __restrict__ b, T* __restrict__ x, const T* __restrict__ inv_lam,
                 int px, int pz, ColourGeom cg, T bscale) {
  constexpr int NS = DIM == 3 ? 27 : 9;
  __shared__ T st[NS];  // st[(cz * 3 + cy) * 3 + cx] (2D: st[cy * 3 + cx])
  if (threadIdx.x < NS) {
    const int t = threadIdx.x;
    const int cx = t % 3, cy = (t / 3) % 3, cz = t / 9;
    const T ax = c_tab<T>.Ap[cx], mx = c_tab<T>.Mp[cx];
    const T ay = c_tab<T>.Ap[cy], my = c_tab<T>.Mp[cy];
    if constexpr (DIM == 3) {
      const T az = c_tab<T>.Ap[cz], mz = c_tab<T>.Mp[cz];
      st[t] = az * my * mx + mz * ay * mx + mz * my * ax;
    } else {
      st[t] = ay * mx + my * ax;
    }
  }
  __syncthreads();
  grid_dependency_wait();  // x and b are written by earlier kernels
  const int64_t gp = blockIdx.x * (int64_t)kQ1Threads + threadIdx.x;
  if (gp >= cg.npatch) return;
  const T s2 = c_tab<T>.S[0] * c_tab<T>.S[0];
  const T scale = DIM == 3 ? s2 * s2 * s2 * __ldg(inv_lam) : s2 * s2 * __ldg(inv_lam);
  const int org = closure_origin((int)gp, cg, px, pz);
  T acc = T(0);
#pragma unroll
  for (int cz = 0; cz < (DIM == 3 ? 3 : 1); ++cz) {
#pragma unroll
    for (int cy = 0; cy < 3; ++cy) {
      const T* row = x + org + cz * pz + cy * px;
#pragma unroll
      for (int cx = 0; cx < 3; ++cx) acc = fma(st[(cz * 3 + cy) * 3 + cx], row[cx], acc);
    }
  }
  const int c = org + (DIM == 3 ? pz : 0) + px + 1;  // the patch's vertex
  const T r = fma(bscale, b[c], -acc);
  x[c] = fma(scale, r, x[c]);
}

// 2D, k = 2, 3: one thread per patch, the whole patch in registers (closure
// n^2 = 25 or 49 values, interior m^2 = 9 or 25).  The same contractions as
// smooth_mult_body in the same even/odd form -- M and A along y on the
// interior rows, A_x (M_y x) + M_x (A_y x) along x, then S^T along x and
// y, the eigenvalue scaling, S along y and x (Eq. 2.13/2.14) -- on register
// arrays, with no shared memory and no barriers; lines that the block
// kernel spreads over threads are here loops of one thread.
template <typename T>
__global__ void __launch_bounds__(kQ1Threads)
smooth_patch2d_kernel(const T* __restrict__ b, T* __restrict__ x, const T* __restrict__ inv_lam,
                      int px, int pz, ColourGeom cg, T bscale) {
  static_assert(DIM == 2 && sizeof(T) > 0, "2D only");
  grid_dependency_wait();  // x and b are written by earlier kernels
  const int64_t gp = blockIdx.x * (int64_t)kQ1Threads + threadIdx.x;
  if (gp >= cg.npatch) return;
  const int org = closure_origin((int)gp, cg, px, pz);
  // along y, column by column: my[o][c] = (M_y x)(o, c), ay[o][c] = (A_y x)(o, c)
  T my[m][n], ay[m][n];
#pragma unroll
  for (int c = 0; c < n; ++c) {
    T v[n][1];
#pragma unroll
    for (int r = 0; r < n; ++r) v[r][0] = x[org + r * px + c];
    T ev[KE][1], od[K][1];
    split_closure<T, 1>(v, ev, od);
#pragma unroll
    for (int o = 0; o <= H; ++o) {
      T em[1] = {T(0)}, ea[1] = {T(0)}, om[1] = {T(0)}, oa[1] = {T(0)};
      row_even<T, 1, 0>(o, ev, em);
      row_even<T, 1, 1>(o, ev, ea);
      if (o < H) {
        row_odd<T, 1, 0>(o, od, om);
        row_odd<T, 1, 1>(o, od, oa);
      }
      my[o][c] = em[0] + om[0];
      ay[o][c] = ea[0] + oa[0];
      if (o < H) {
        my[m - 1 - o][c] = em[0] - om[0];
        ay[m - 1 - o][c] = ea[0] - oa[0];
      }
    }
  }
  // along x on each interior row: r = bscale b - (A_x my + M_x ay), then S^T along x
  T w[m][m];  // w[oy][a]
#pragma unroll
  for (int oy = 0; oy < m; ++oy) {
    T vm[n][1], va[n][1];
#pragma unroll
    for (int c = 0; c < n; ++c) {
      vm[c][0] = my[oy][c];
      va[c][0] = ay[oy][c];
    }
    T ex[KE][1], dx[K][1], ey[KE][1], dy[K][1];
    split_closure<T, 1>(vm, ex, dx);
    split_closure<T, 1>(va, ey, dy);
    const T* brow = b + org + (oy + 1) * px + 1;
    T rr[m][1];
#pragma unroll
    for (int o = 0; o <= H; ++o) {
      T E[1] = {T(0)}, O[1] = {T(0)};
      row_even<T, 1, 1>(o, ex, E);
      row_even<T, 1, 0>(o, ey, E);
      if (o < H) {
        row_odd<T, 1, 1>(o, dx, O);
        row_odd<T, 1, 0>(o, dy, O);
      }
      rr[o][0] = fma(bscale, brow[o], -(E[0] + O[0]));
      if (o < H) rr[m - 1 - o][0] = fma(bscale, brow[m - 1 - o], -(E[0] - O[0]));
    }
    T tt[m][1];
    st_line<T, 1>(rr, tt);
#pragma unroll
    for (int a = 0; a < m; ++a) w[oy][a] = tt[a][0];
  }
  // S^T along y, the scaling by 1/(lambda_a + lambda_b), S along y
#pragma unroll
  for (int a = 0; a < m; ++a) {
    T col[m][1], ty[m][1], u[m][1];
#pragma unroll
    for (int oy = 0; oy < m; ++oy) col[oy][0] = w[oy][a];
    st_line<T, 1>(col, ty);
#pragma unroll
    for (int be = 0; be < m; ++be) ty[be][0] *= __ldg(inv_lam + be * m + a);
    s_line<T, 1>(ty, u);
#pragma unroll
    for (int oy = 0; oy < m; ++oy) w[oy][a] = u[oy][0];
  }
  // S along x and the update of the interior
#pragma unroll
  for (int oy = 0; oy < m; ++oy) {
    T row[m][1], u[m][1];
#pragma unroll
    for (int a = 0; a < m; ++a) row[a][0] = w[oy][a];
    s_line<T, 1>(row, u);
    T* dst = x + org + (oy + 1) * px + 1;
#pragma unroll
    for (int o = 0; o < m; ++o) dst[o] = fma(T(1), u[o][0], dst[o]);
  }
}

// -------------------------------------------------- inverse-matrix solve
// x_I += scale * A_j^-1 r_I for every patch of one colour with the dense
// precomputed inverse (one copy: the coefficients are constant), the
// "inverse matrix" local solver that Section 3.1 compares with fast
// diagonalisation.  One patch per block, one interior node per thread;
// AinvT holds A_j^-1 transposed (column j contiguous) so that the threads
// of a warp read consecutive entries.
constexpr int kMDim = DIM == 3 ? m * m * m : m * m;
constexpr int kInvThreads = ((kMDim + 31) / 32) * 32;
constexpr bool kInvFits = kMDim <= 1024;

__device__ __forceinline__ int interior_offset(int e, int px, int pz) {
  if constexpr (DIM == 3) return (e / (m * m) + 1) * pz + ((e / m) % m + 1) * px + 1 + e % m;
  else return (e / m + 1) * px + 1 + e % m;
}

template <typename T>
__global__ void __launch_bounds__(kInvFits ? kInvThreads : 32)
inverse_solve_kernel(const T* __restrict__ r, T* __restrict__ x, const T* __restrict__ AinvT,
                     int px, int pz, ColourGeom cg, T scale) {
  __shared__ T rs[kInvFits ? kMDim : 1];
  if constexpr (kInvFits) {
    const int gp = blockIdx.x;
    if (gp >= cg.npatch) return;
    const int org = closure_origin(gp, cg, px, pz);
    for (int e = threadIdx.x; e < kMDim; e += kInvThreads) rs[e] = r[org + interior_offset(e, px, pz)];
    __syncthreads();
    const int i = threadIdx.x;
    if (i < kMDim) {
      T u = T(0);
      for (int j = 0; j < kMDim; ++j) u = fma(__ldg(AinvT + (size_t)j * kMDim + i), rs[j], u);
      T* dst = x + org + interior_offset(i, px, pz);
      *dst = fma(scale, u, *dst);
    }
  }
}

// ------------------------------------------------------------- operator
// y = A x on an output tile of TN = K*CT nodes per direction.  The first
// contraction (along the slowest direction) reads its lines of 2K+1 nodes
// straight from global memory; the halo of K nodes per side is only needed
// in the directions contracted later.  A = sum of Kronecker products of the
// banded global 1D matrices (Section 2.3): z -> M, K; y -> M M, K M + M K;
// x -> K (M M) + M (K M + M K).
struct ApplyCfg {
  // cells per tile: a power of two (see Apply3Cfg)
  static constexpr int CT = DIM == 3 ? (K == 1 ? 8 : K == 2 ? 4 : K <= 5 ? 2 : 1)
                                     : (K == 1 ? 32 : K == 2 ? 16 : K == 3 ? 16 : 8);
  static constexpr int TN = K * CT;
  static constexpr int BN = TN + 2 * K;
  static constexpr int RB = BN | 1;    // odd row stride
  static constexpr int NT = 256;
  // 3D: stage-A outputs [TN][BN][RB] x2, stage-B outputs [TN][TN][RB] x2
  // 2D: stage-A outputs [TN][RB] x2
  static constexpr int a_sz = DIM == 3 ? TN * BN * RB : TN * RB;
  static constexpr int b_sz = DIM == 3 ? TN * TN * RB : 0;
  template <typename T>
  static constexpr size_t smem() { return sizeof(T) * (size_t)(2 * a_sz + 2 * b_sz); }
};

// out[q] = sum over the band of node position q of B[q][j] * v[q + j]
// (q = 0: vertex node, all 2K+1 entries; else the K+1 entries of its cell).
#define VPS_BAND_LOOP(q, j) \
  _Pragma("unroll") for (int j = 0; j <= 2 * K; ++j) if (q == 0 || (j >= K - q && j <= 2 * K - q))

// The upper boundary layer of a level vector (index n1-1 in any direction)
// is owned by no operator or restriction tile; this zeroes the elements
// first, first + step, ... of it (faces x, y, z in turn).
template <typename T>
__device__ __forceinline__ void zero_upper_faces_body(T* __restrict__ v, int n1, int64_t px,
                                                      int64_t pz, int64_t first, int64_t step) {
  const int64_t nface = DIM == 3 ? (int64_t)n1 * n1 : n1;
  for (int64_t e = first; e < DIM * nface; e += step) {
    const int f = (int)(e / nface);
    const int64_t r = e % nface;
    const int a = (int)(r % n1), c = DIM == 3 ? (int)(r / n1) : 0;
    int64_t idx;
    if (f == 0) idx = (int64_t)c * pz + (int64_t)a * px + (n1 - 1);
    else if (f == 1) idx = (int64_t)c * pz + (int64_t)(n1 - 1) * px + a;
    else idx = (int64_t)(n1 - 1) * pz + (int64_t)c * px + a;
    v[idx] = T(0);
  }
}

// This block's share of the upper faces of y (every block of the grid takes
// a stride of them): the operator and transfer kernels write every node
// 0..n1-2 of each direction and zero the layer n1-1 this way, so no separate
// launch is needed.  The face nodes are disjoint from the nodes the tiles
// write.
template <typename T>
__device__ __forceinline__ void block_zero_faces(T* __restrict__ y, int n1, int64_t px, int64_t pz) {
  const int64_t nb = (int64_t)gridDim.x * gridDim.y * gridDim.z;
  const int64_t bid = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
  zero_upper_faces_body<T>(y, n1, px, pz, bid * blockDim.x + threadIdx.x, nb * blockDim.x);
}

template <typename T, bool ABS = false>
__global__ void __launch_bounds__(ApplyCfg::NT)
apply_kernel(const T* __restrict__ x, const T* __restrict__ bvec, T* __restrict__ y, int n1,
             int64_t px, int64_t pz, T scale) {
  using C = ApplyCfg;
  constexpr int TN = C::TN, BN = C::BN, RB = C::RB, CT = C::CT, NT = C::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tm = reinterpret_cast<T*>(smem_raw);
  T* tk = tm + C::a_sz;
  const int x0 = blockIdx.x * TN, y0 = blockIdx.y * TN;
  block_zero_faces<T>(y, n1, px, pz);
  if constexpr (DIM == 3) {
    const int z0 = blockIdx.z * TN;
    T* mm = tk + C::a_sz;
    T* ww = mm + C::b_sz;
    // stage A: along z from global; units (y, x) over the halo box, z segment
    for (int u = threadIdx.x; u < BN * BN * CT; u += NT) {
      const int xx = u % BN, yy = (u / BN) % BN, cz = u / (BN * BN);
      const int gx = x0 - K + xx, gy = y0 - K + yy, gz0 = z0 + cz * K - K;
      T v[2 * K + 1];
      const bool inxy = gx >= 0 && gx < n1 && gy >= 0 && gy < n1;
#pragma unroll
      for (int i = 0; i <= 2 * K; ++i) {
        const int gz = gz0 + i;
        v[i] = (inxy && gz >= 0 && gz < n1) ? x[(int64_t)gz * pz + (int64_t)gy * px + gx] : T(0);
        if constexpr (ABS) v[i] = fabs(v[i]);
      }
#pragma unroll
      for (int q = 0; q < K; ++q) {
        T am = T(0), ak = T(0);
        VPS_BAND_LOOP(q, j) {
          am = fma(coefM<T, ABS>(q * n + j), v[q + j], am);
          ak = fma(coefK<T, ABS>(q * n + j), v[q + j], ak);
        }
        tm[((cz * K + q) * BN + yy) * RB + xx] = am;
        tk[((cz * K + q) * BN + yy) * RB + xx] = ak;
      }
    }
    __syncthreads();
    // stage B: along y; units (z, y segment, x over the halo)
    for (int u = threadIdx.x; u < TN * CT * BN; u += NT) {
      const int xx = u % BN, cy = (u / BN) % CT, Z = u / (BN * CT);
      T vm[2 * K + 1], vk[2 * K + 1];
#pragma unroll
      for (int i = 0; i <= 2 * K; ++i) {
        vm[i] = tm[(Z * BN + cy * K + i) * RB + xx];
        vk[i] = tk[(Z * BN + cy * K + i) * RB + xx];
      }
#pragma unroll
      for (int q = 0; q < K; ++q) {
        T a = T(0), bb = T(0);
        VPS_BAND_LOOP(q, j) {
          a = fma(coefM<T, ABS>(q * n + j), vm[q + j], a);
          bb = fma(coefK<T, ABS>(q * n + j), vm[q + j], bb);
          bb = fma(coefM<T, ABS>(q * n + j), vk[q + j], bb);
        }
        mm[(Z * TN + cy * K + q) * RB + xx] = a;
        ww[(Z * TN + cy * K + q) * RB + xx] = bb;
      }
    }
    __syncthreads();
    // stage C: along x; units (y fastest, z, x segment); write the tile
    for (int u = threadIdx.x; u < TN * TN * CT; u += NT) {
      const int Y = u % TN, Z = (u / TN) % TN, cx = u / (TN * TN);
      const int gy = y0 + Y, gz = z0 + Z;
      if (gy >= n1 || gz >= n1) continue;
      T vm[2 * K + 1], vw[2 * K + 1];
#pragma unroll
      for (int i = 0; i <= 2 * K; ++i) {
        vm[i] = mm[(Z * TN + Y) * RB + cx * K + i];
        vw[i] = ww[(Z * TN + Y) * RB + cx * K + i];
      }
      const bool inner_yz = gy >= 1 && gy <= n1 - 2 && gz >= 1 && gz <= n1 - 2;
      const int64_t rowi = (int64_t)gz * pz + (int64_t)gy * px;
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const int gx = x0 + cx * K + q;
        if (gx >= n1) continue;
        T acc = T(0);
        VPS_BAND_LOOP(q, j) {
          acc = fma(coefK<T, ABS>(q * n + j), vm[q + j], acc);
          acc = fma(coefM<T, ABS>(q * n + j), vw[q + j], acc);
        }
        T out = T(0);
        if (inner_yz && gx >= 1 && gx <= n1 - 2)
          out = bvec ? bvec[rowi + gx] - scale * acc : scale * acc;
        y[rowi + gx] = out;
      }
    }
  } else {
    // stage A (2D): along y from global; units (x over the halo, y segment)
    for (int u = threadIdx.x; u < BN * CT; u += NT) {
      const int xx = u % BN, cy = u / BN;
      const int gx = x0 - K + xx, gy0 = y0 + cy * K - K;
      T v[2 * K + 1];
#pragma unroll
      for (int i = 0; i <= 2 * K; ++i) {
        const int gy = gy0 + i;
        v[i] = (gx >= 0 && gx < n1 && gy >= 0 && gy < n1) ? x[(int64_t)gy * px + gx] : T(0);
        if constexpr (ABS) v[i] = fabs(v[i]);
      }
#pragma unroll
      for (int q = 0; q < K; ++q) {
        T am = T(0), ak = T(0);
        VPS_BAND_LOOP(q, j) {
          am = fma(coefM<T, ABS>(q * n + j), v[q + j], am);
          ak = fma(coefK<T, ABS>(q * n + j), v[q + j], ak);
        }
        tm[(cy * K + q) * RB + xx] = am;
        tk[(cy * K + q) * RB + xx] = ak;
      }
    }
    __syncthreads();
    // stage B: along x; y = K0 (M1 x) + M0 (K1 x)
    for (int u = threadIdx.x; u < TN * CT; u += NT) {
      const int Y = u % TN, cx = u / TN;
      const int gy = y0 + Y;
      if (gy >= n1) continue;
      T vm[2 * K + 1], vk[2 * K + 1];
#pragma unroll
      for (int i = 0; i <= 2 * K; ++i) {
        vm[i] = tm[Y * RB + cx * K + i];
        vk[i] = tk[Y * RB + cx * K + i];
      }
      const int64_t rowi = (int64_t)gy * px;
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const int gx = x0 + cx * K + q;
        if (gx >= n1) continue;
        T acc = T(0);
        VPS_BAND_LOOP(q, j) {
          acc = fma(coefK<T, ABS>(q * n + j), vm[q + j], acc);
          acc = fma(coefM<T, ABS>(q * n + j), vk[q + j], acc);
        }
        T out = T(0);
        if (gx >= 1 && gx <= n1 - 2 && gy >= 1 && gy <= n1 - 2)
          out = bvec ? bvec[rowi + gx] - scale * acc : scale * acc;
        y[rowi + gx] = out;
      }
    }
  }
}

// 3D operator on wide x-y tiles marching in z.  A block owns TX x TY output
// columns (x, y) and a range of ZR planes.  For every plane it contracts z
// (lines of the band read from global memory, cached in L1 across planes)
// over the tile plus a halo of K in x and y, then y over the tile plus the x
// halo, then x; the z-contraction planes are double-buffered so each plane
// costs two barriers.  Halo recomputation: ((T+2K)/T)^2 in the z stage and
// (T+2K)/T in the y stage, against ((T+2K)/T)^2 and (T+2K)/T with T = K*CT
// small for cubic tiles.
struct Apply3Cfg {
  // cells per tile in x and y: a power of two, so that tiles of TX nodes
  // cover the nodes 0 .. n1-2 = k 2^l - 1 exactly (no ragged tiles)
  static constexpr int CX = K == 1 ? 32 : (K == 2 ? 16 : 8);
  static constexpr int TX = K * CX;
  static constexpr int BX = TX + 2 * K;
  static constexpr int RB = BX | 1;

  // threads: one y-stage unit each (BX * CX units), so that stage is one
  // round; the z and x stages then take about K+2 and one round
  static constexpr int UB = BX * CX;
  static constexpr int NT0 = ((UB + 31) / 32) * 32;
  static constexpr int NT = NT0 > 1024 ? ((UB / 2 + 31) / 32) * 32 : (NT0 < 256 ? 256 : NT0);
  static constexpr int MINB = (NT <= 512 && K <= 5) ? 2 : 1;
  template <typename T>
  static constexpr size_t smem() { return sizeof(T) * (size_t)(4 * BX * RB + 2 * TX * RB); }
  // apply3c_kernel: the z contractions of a cell's K planes, then two
  // buffers of the y stage's outputs
  template <typename T>
  static constexpr size_t smem_c() { return sizeof(T) * (size_t)(2 * K * BX * RB + 4 * TX * RB); }
};

// The FP32 operator takes apply3c_kernel where its shared memory leaves room
// for two blocks per SM (k <= 4); the FP64 and |A||x| operators, whose FP64
// arithmetic bounds them, keep apply3_kernel.
template <typename T>
constexpr bool kApply3C = sizeof(T) == 4 && K <= 4;
// cells of planes per block of apply3c_kernel
constexpr int kApply3CZ = K == 1 ? 8 : (K <= 3 ? 4 : 2);

// z contraction of plane z (Q: the plane's position in its cell, which
// selects the band) over the halo'd tile of apply3_kernel.
template <typename T, bool ABS, int Q>
__device__ __forceinline__ void apply3_zstage(const T* __restrict__ x, T* mZ, T* kZ, int x0, int y0,
                                              int z, int n1, int px, int pz) {
  using C = Apply3Cfg;
  constexpr int BX = C::BX, RB = C::RB, NT = C::NT;
  for (int u = threadIdx.x; u < BX * BX; u += NT) {
    const int xx = u % BX, yy = u / BX;
    const int gx = x0 - K + xx, gy = y0 - K + yy;
    T am = T(0), ak = T(0);
    if (gx >= 0 && gx < n1 && gy >= 0 && gy < n1) {
      const T* col = x + gy * px + gx;
      VPS_BAND_LOOP(Q, j) {
        const int gz = z - K + j;
        T v = (gz >= 0 && gz < n1) ? __ldg(col + gz * pz) : T(0);
        if constexpr (ABS) v = fabs(v);
        am = fma(coefM<T, ABS>(Q * n + j), v, am);
        ak = fma(coefK<T, ABS>(Q * n + j), v, ak);
      }
    }
    mZ[yy * RB + xx] = am;
    kZ[yy * RB + xx] = ak;
  }
}

// apply3_zstage<Qc> for a run-time plane position q < K.
template <typename T, bool ABS, int Qc>
__device__ __forceinline__ void apply3_zstage_at(int q, const T* __restrict__ x, T* mZ, T* kZ,
                                                 int x0, int y0, int z, int n1, int px, int pz) {
  if constexpr (Qc < K) {
    if (q == Qc) apply3_zstage<T, ABS, Qc>(x, mZ, kZ, x0, y0, z, n1, px, pz);
    else apply3_zstage_at<T, ABS, Qc + 1>(q, x, mZ, kZ, x0, y0, z, n1, px, pz);
  }
}

// The per-plane 3D operator: a block takes the planes zpb * blockIdx.z ..
// of its x-y tile (any run of planes: the launcher chooses zpb so that the
// grid fills the resident block slots of the GPU in few rounds), the z
// contraction of each plane dispatched by the plane's position in its cell.
template <typename T, bool ABS = false>
__global__ void __launch_bounds__(Apply3Cfg::NT, Apply3Cfg::MINB)
apply3_kernel(const T* __restrict__ x, const T* __restrict__ bvec, T* __restrict__ y, int n1,
              int px, int pz, T scale, int zpb) {
  using C = Apply3Cfg;
  constexpr int TX = C::TX, BX = C::BX, RB = C::RB, CX = C::CX, NT = C::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* zbuf = reinterpret_cast<T*>(smem_raw);  // [2][2][BX][RB]: (m, k) x double buffer
  T* MM = zbuf + 4 * BX * RB;                // [TX][RB]
  T* WW = MM + TX * RB;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TX;
  block_zero_faces<T>(y, n1, px, pz);
  const int zb = blockIdx.z * zpb;
  const int ze = min(zb + zpb, n1 - 1);  // plane n1-1 is zeroed by block_zero_faces
  int buf = 0;
  {
#pragma unroll 1
    for (int z = zb; z < ze; ++z) {
      T* mZ = zbuf + (2 * buf) * BX * RB;
      T* kZ = mZ + BX * RB;
      apply3_zstage_at<T, ABS, 0>(z % K, x, mZ, kZ, x0, y0, z, n1, px, pz);
      __syncthreads();
      // y contraction: units (x over the halo, cell segment in y)
      for (int u = threadIdx.x; u < BX * CX; u += NT) {
        const int xx = u % BX, cy = u / BX;
        T vm[2 * K + 1], vk[2 * K + 1];
#pragma unroll
        for (int i = 0; i <= 2 * K; ++i) {
          vm[i] = mZ[(cy * K + i) * RB + xx];
          vk[i] = kZ[(cy * K + i) * RB + xx];
        }
#pragma unroll
        for (int qy = 0; qy < K; ++qy) {
          T a = T(0), bb = T(0);
          VPS_BAND_LOOP(qy, j) {
            a = fma(coefM<T, ABS>(qy * n + j), vm[qy + j], a);
            bb = fma(coefK<T, ABS>(qy * n + j), vm[qy + j], bb);
            bb = fma(coefM<T, ABS>(qy * n + j), vk[qy + j], bb);
          }
          MM[(cy * K + qy) * RB + xx] = a;
          WW[(cy * K + qy) * RB + xx] = bb;
        }
      }
      __syncthreads();
      // x contraction and store: units (y fastest, cell segment in x)
      const bool inner_z = z >= 1 && z <= n1 - 2;
      for (int u = threadIdx.x; u < TX * CX; u += NT) {
        const int Y = u % TX, cx = u / TX;
        const int gy = y0 + Y;
        if (gy >= n1) continue;
        T vm[2 * K + 1], vw[2 * K + 1];
#pragma unroll
        for (int i = 0; i <= 2 * K; ++i) {
          vm[i] = MM[Y * RB + cx * K + i];
          vw[i] = WW[Y * RB + cx * K + i];
        }
        const bool inner_yz = inner_z && gy >= 1 && gy <= n1 - 2;
        const int rowi = z * pz + gy * px;
#pragma unroll
        for (int qx = 0; qx < K; ++qx) {
          const int gx = x0 + cx * K + qx;
          if (gx >= n1) continue;
          T acc = T(0);
          VPS_BAND_LOOP(qx, j) {
            acc = fma(coefK<T, ABS>(qx * n + j), vm[qx + j], acc);
            acc = fma(coefM<T, ABS>(qx * n + j), vw[qx + j], acc);
          }
          T out = T(0);
          if (inner_yz && gx >= 1 && gx <= n1 - 2)
            out = bvec ? bvec[rowi + gx] - scale * acc : scale * acc;
          y[rowi + gx] = out;
        }
      }
      buf ^= 1;
    }
  }
}

// 3D operator on the same tiles as apply3_kernel, with the z contraction
// taken a whole cell at a time.  The K planes z0 .. z0+K-1 of a cell couple
// only the 2K+1 planes z0-K .. z0+K (the vertex row both neighbouring cells,
// the interior rows their own cell), so each column of the halo'd tile
// loads that window once, all loads in flight together, and writes the M
// and K contractions of all K planes; then y and x per plane as before,
// with the y stage's outputs double-buffered (one barrier per plane).  The
// per-plane z stage of apply3_kernel loads 2K+1 values for the vertex plane
// and K+1 for each other plane, one plane at a time, and was bound by the
// latency of those loads (long-scoreboard stalls, a third of the issue
// slots used).
template <typename T>
__global__ void __launch_bounds__(Apply3Cfg::NT, Apply3Cfg::MINB)
apply3c_kernel(const T* __restrict__ x, const T* __restrict__ bvec, T* __restrict__ y, int n1,
               int px, int pz, T scale) {
  using C = Apply3Cfg;
  constexpr int TX = C::TX, BX = C::BX, RB = C::RB, CX = C::CX, NT = C::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* zb = reinterpret_cast<T*>(smem_raw);  // [K][M, K rows][BX][RB]
  T* mw = zb + 2 * K * BX * RB;            // [2 buffers][MM, WW][TX][RB]
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TX;
  block_zero_faces<T>(y, n1, px, pz);
  for (int cz = 0; cz < kApply3CZ; ++cz) {
    const int z0 = (blockIdx.z * kApply3CZ + cz) * K;
    if (z0 >= n1 - 1) break;  // uniform in the block; plane n1-1 is zeroed elsewhere
    for (int u = threadIdx.x; u < BX * BX; u += NT) {
      const int xx = u % BX, yy = u / BX;
      const int gx = x0 - K + xx, gy = y0 - K + yy;
      const bool in = gx >= 0 && gx < n1 && gy >= 0 && gy < n1;
      T w[2 * K + 1];
#pragma unroll
      for (int t = 0; t <= 2 * K; ++t) {
        const int gz = z0 - K + t;
        w[t] = (in && gz >= 0 && gz < n1) ? __ldg(x + (gz * pz + gy * px + gx)) : T(0);
      }
#pragma unroll
      for (int q = 0; q < K; ++q) {
        T am = T(0), ak = T(0);
        VPS_BAND_LOOP(q, j) {
          am = fma(coefM<T, false>(q * n + j), w[q + j], am);
          ak = fma(coefK<T, false>(q * n + j), w[q + j], ak);
        }
        zb[(2 * q * BX + yy) * RB + xx] = am;
        zb[((2 * q + 1) * BX + yy) * RB + xx] = ak;
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int q = 0; q < K; ++q) {
      const T* mZ = zb + 2 * q * BX * RB;
      const T* kZ = mZ + BX * RB;
      T* MM = mw + (q & 1) * 2 * TX * RB;
      T* WW = MM + TX * RB;
      // y contraction: units (x over the halo, cell segment in y)
      for (int u = threadIdx.x; u < BX * CX; u += NT) {
        const int xx = u % BX, cy = u / BX;
        T vm[2 * K + 1], vk[2 * K + 1];
#pragma unroll
        for (int i = 0; i <= 2 * K; ++i) {
          vm[i] = mZ[(cy * K + i) * RB + xx];
          vk[i] = kZ[(cy * K + i) * RB + xx];
        }
#pragma unroll
        for (int qy = 0; qy < K; ++qy) {
          T a = T(0), bb = T(0);
          VPS_BAND_LOOP(qy, j) {
            a = fma(coefM<T, false>(qy * n + j), vm[qy + j], a);
            bb = fma(coefK<T, false>(qy * n + j), vm[qy + j], bb);
            bb = fma(coefM<T, false>(qy * n + j), vk[qy + j], bb);
          }
          MM[(cy * K + qy) * RB + xx] = a;
          WW[(cy * K + qy) * RB + xx] = bb;
        }
      }
      __syncthreads();
      // x contraction and store: units (y fastest, cell segment in x)
      const int z = z0 + q;
      const bool inner_z = z >= 1 && z <= n1 - 2;
      for (int u = threadIdx.x; u < TX * CX; u += NT) {
        const int Y = u % TX, cx = u / TX;
        const int gy = y0 + Y;
        if (gy >= n1) continue;
        T vm[2 * K + 1], vw[2 * K + 1];
#pragma unroll
        for (int i = 0; i <= 2 * K; ++i) {
          vm[i] = MM[Y * RB + cx * K + i];
          vw[i] = WW[Y * RB + cx * K + i];
        }
        const bool inner_yz = inner_z && gy >= 1 && gy <= n1 - 2;
        const int rowi = z * pz + gy * px;
#pragma unroll
        for (int qx = 0; qx < K; ++qx) {
          const int gx = x0 + cx * K + qx;
          if (gx >= n1) continue;
          T acc = T(0);
          VPS_BAND_LOOP(qx, j) {
            acc = fma(coefK<T, false>(qx * n + j), vm[qx + j], acc);
            acc = fma(coefM<T, false>(qx * n + j), vw[qx + j], acc);
          }
          T out = T(0);
          if (inner_yz && gx >= 1 && gx <= n1 - 2)
            out = bvec ? bvec[rowi + gx] - scale * acc : scale * acc;
          y[rowi + gx] = out;
        }
      }
      // no barrier: the next y stage writes the other buffer; the one after
      // it follows the barrier that ends this x stage's reads
    }
    // no barrier: the next cell's z stage writes zb, which the y stages have
    // finished reading (the barrier after the last of them)
  }
}

// ------------------------------------------------- double-float operator
// y = A x in FP64-like accuracy with FP32 arithmetic, for the outer CG of the
// mixed-precision solver: FP64 runs at 1/64 of the FP32 rate on this GPU,
// while this operator is a short sum of products per output.  A value is a
// pair (hi, lo) of floats; a product c x of a coefficient (c_hi + c_lo) and
// a value is formed exactly up to its cross terms with one FMA for the
// rounding error of c_hi x_hi; sums use Knuth's TwoSum on the high words
// and accumulate the low words.  Relative accuracy about 2^-48 of the sum of
// the magnitudes of the terms.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ void df_madd(DF& s, float ch, float cl, const DF& x) {
  const float p = ch * x.hi;
  const float pe = fmaf(ch, x.hi, -p);                       // exact error of ch * x.hi
  const float pl = fmaf(ch, x.lo, fmaf(cl, x.hi, pe));
  const float t = s.hi + p;                                  // TwoSum(s.hi, p)
  const float bb = t - s.hi;
  const float e = (s.hi - (t - bb)) + (p - bb);
  s.hi = t;
  s.lo = s.lo + (e + pl);
}

__device__ __forceinline__ DF df_norm(const DF& s) {
  const float h = s.hi + s.lo;
  return DF{h, s.lo - (h - s.hi)};
}

#define VPS_DF_MADD(acc, TAB, q, j, v) \
  df_madd(acc, c_tab<float>.TAB[(q) * n + (j)], c_tab<float>.TAB##_lo[(q) * n + (j)], v)

// z contraction of plane z = z0 + Q (Q: the plane's position in its cell,
// which selects the band) over the halo'd tile, double-float.
template <int Q>
__device__ __forceinline__ void df_zstage(const float* __restrict__ xh,
                                          const float* __restrict__ xl, DF* mZ, DF* kZ, int x0,
                                          int y0, int z, int n1, int px, int pz) {
  using C = Apply3Cfg;
  constexpr int BX = C::BX, RB = C::RB, NT = C::NT;
  for (int u = threadIdx.x; u < BX * BX; u += NT) {
    const int xx = u % BX, yy = u / BX;
    const int gx = x0 - K + xx, gy = y0 - K + yy;
    DF am{0.f, 0.f}, ak{0.f, 0.f};
    if (gx >= 0 && gx < n1 && gy >= 0 && gy < n1) {
      const int col = gy * px + gx;
      VPS_BAND_LOOP(Q, j) {
        const int gz = z - K + j;
        DF v{0.f, 0.f};
        if (gz >= 0 && gz < n1) v = DF{__ldg(xh + col + gz * pz), __ldg(xl + col + gz * pz)};
        VPS_DF_MADD(am, Mb, Q, j, v);
        VPS_DF_MADD(ak, Kb, Q, j, v);
      }
    }
    mZ[yy * RB + xx] = df_norm(am);
    kZ[yy * RB + xx] = df_norm(ak);
  }
}

// df_zstage<q> for a run-time q < K: the plane loop of apply3_df_kernel
// stays rolled, so its large y and x stages are compiled once (unrolled over
// the K planes, the kernel's code stalled on instruction fetch).
template <int Qc>
__device__ __forceinline__ void df_zstage_at(int q, const float* __restrict__ xh,
                                             const float* __restrict__ xl, DF* mZ, DF* kZ,
                                             int x0, int y0, int z, int n1, int px, int pz) {
  if constexpr (Qc < K) {
    if (q == Qc) df_zstage<Qc>(xh, xl, mZ, kZ, x0, y0, z, n1, px, pz);
    else df_zstage_at<Qc + 1>(q, xh, xl, mZ, kZ, x0, y0, z, n1, px, pz);
  }
}

template <int DUMMY>
__global__ void __launch_bounds__(Apply3Cfg::NT, Apply3Cfg::MINB)
apply3_df_kernel(const float* __restrict__ xh, const float* __restrict__ xl,
                 double* __restrict__ y, int n1, int px, int pz, float scale, int zpb) {
  using C = Apply3Cfg;
  constexpr int TX = C::TX, BX = C::BX, RB = C::RB, CX = C::CX, NT = C::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DF* zbuf = reinterpret_cast<DF*>(smem_raw);  // [2][2][BX][RB]
  DF* MM = zbuf + 4 * BX * RB;
  DF* WW = MM + TX * RB;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TX;
  block_zero_faces<double>(y, n1, px, pz);
  // planes zpb * blockIdx.z .. (as in apply3_kernel)
  const int zb = blockIdx.z * zpb;
  const int ze = min(zb + zpb, n1 - 1);
  int buf = 0;
  {
#pragma unroll 1
    for (int z = zb; z < ze; ++z) {
      DF* mZ = zbuf + (2 * buf) * BX * RB;
      DF* kZ = mZ + BX * RB;
      df_zstage_at<0>(z % K, xh, xl, mZ, kZ, x0, y0, z, n1, px, pz);
      __syncthreads();
      for (int u = threadIdx.x; u < BX * CX; u += NT) {
        const int xx = u % BX, cy = u / BX;
        DF vm[2 * K + 1], vk[2 * K + 1];
#pragma unroll
        for (int i = 0; i <= 2 * K; ++i) {
          vm[i] = mZ[(cy * K + i) * RB + xx];
          vk[i] = kZ[(cy * K + i) * RB + xx];
        }
#pragma unroll
        for (int qy = 0; qy < K; ++qy) {
          DF a{0.f, 0.f}, bb{0.f, 0.f};
          VPS_BAND_LOOP(qy, j) {
            VPS_DF_MADD(a, Mb, qy, j, vm[qy + j]);
            VPS_DF_MADD(bb, Kb, qy, j, vm[qy + j]);
            VPS_DF_MADD(bb, Mb, qy, j, vk[qy + j]);
          }
          MM[(cy * K + qy) * RB + xx] = df_norm(a);
          WW[(cy * K + qy) * RB + xx] = df_norm(bb);
        }
      }
      __syncthreads();
      const bool inner_z = z >= 1 && z <= n1 - 2;
      for (int u = threadIdx.x; u < TX * CX; u += NT) {
        const int Y = u % TX, cx = u / TX;
        const int gy = y0 + Y;
        if (gy >= n1) continue;
        DF vm[2 * K + 1], vw[2 * K + 1];
#pragma unroll
        for (int i = 0; i <= 2 * K; ++i) {
          vm[i] = MM[Y * RB + cx * K + i];
          vw[i] = WW[Y * RB + cx * K + i];
        }
        const bool inner_yz = inner_z && gy >= 1 && gy <= n1 - 2;
        const int rowi = z * pz + gy * px;
#pragma unroll
        for (int qx = 0; qx < K; ++qx) {
          const int gx = x0 + cx * K + qx;
          if (gx >= n1) continue;
          DF acc{0.f, 0.f};
          VPS_BAND_LOOP(qx, j) {
            VPS_DF_MADD(acc, Kb, qx, j, vm[qx + j]);
            VPS_DF_MADD(acc, Mb, qx, j, vw[qx + j]);
          }
          // scale = h, a power of two: exact on both words; the words are
          // widened by integer operations and added with one FP64 addition
          double out = 0.0;
          if (inner_yz && gx >= 1 && gx <= n1 - 2) out = f2d(acc.hi * scale) + f2d(acc.lo * scale);
          y[rowi + gx] = out;
        }
      }
      buf ^= 1;
    }
  }
}

// 2D: tiles of TN x TN outputs, y first from global, then x.
template <int DUMMY>
__global__ void __launch_bounds__(ApplyCfg::NT)
apply2_df_kernel(const float* __restrict__ xh, const float* __restrict__ xl, double* __restrict__ y,
                 int n1, int px) {
  using C = ApplyCfg;
  constexpr int TN = C::TN, BN = C::BN, RB = C::RB, CT = C::CT, NT = C::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DF* tm = reinterpret_cast<DF*>(smem_raw);
  DF* tk = tm + C::a_sz;
  const int x0 = blockIdx.x * TN, y0 = blockIdx.y * TN;
  block_zero_faces<double>(y, n1, px, 0);
  for (int u = threadIdx.x; u < BN * CT; u += NT) {
    const int xx = u % BN, cy = u / BN;
    const int gx = x0 - K + xx, gy0 = y0 + cy * K - K;
    DF v[2 * K + 1];
#pragma unroll
    for (int i = 0; i <= 2 * K; ++i) {
      const int gy = gy0 + i;
      v[i] = (gx >= 0 && gx < n1 && gy >= 0 && gy < n1)
                 ? DF{__ldg(xh + gy * px + gx), __ldg(xl + gy * px + gx)}
                 : DF{0.f, 0.f};
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
      DF am{0.f, 0.f}, ak{0.f, 0.f};
      VPS_BAND_LOOP(q, j) {
        VPS_DF_MADD(am, Mb, q, j, v[q + j]);
        VPS_DF_MADD(ak, Kb, q, j, v[q + j]);
      }
      tm[(cy * K + q) * RB + xx] = df_norm(am);
      tk[(cy * K + q) * RB + xx] = df_norm(ak);
    }
  }
  __syncthreads();
  for (int u = threadIdx.x; u < TN * CT; u += NT) {
    const int Y = u % TN, cx = u / TN;
    const int gy = y0 + Y;
    if (gy >= n1) continue;
    DF vm[2 * K + 1], vk[2 * K + 1];
#pragma unroll
    for (int i = 0; i <= 2 * K; ++i) {
      vm[i] = tm[Y * RB + cx * K + i];
      vk[i] = tk[Y * RB + cx * K + i];
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int gx = x0 + cx * K + q;
      if (gx >= n1) continue;
      DF acc{0.f, 0.f};
      VPS_BAND_LOOP(q, j) {
        VPS_DF_MADD(acc, Kb, q, j, vm[q + j]);
        VPS_DF_MADD(acc, Mb, q, j, vk[q + j]);
      }
      double out = 0.0;
      if (gx >= 1 && gx <= n1 - 2 && gy >= 1 && gy <= n1 - 2) out = f2d(acc.hi) + f2d(acc.lo);
      y[gy * px + gx] = out;
    }
  }
}

// ------------------------------------------------------------ transfers
// Tiles of CC coarse cells per direction; the first contraction (slowest
// direction) reads from global memory.
struct TransferCfg {
  static constexpr int CC = DIM == 3 ? (K <= 1 ? 8 : K <= 2 ? 4 : K <= 4 ? 2 : 1)
                                     : (K <= 2 ? 16 : 8);
  static constexpr int CB = K * CC + 1;   // coarse nodes of the tile (prolongation input)
  static constexpr int CBp = CB | 1;
  static constexpr int FB = 2 * K * CC;   // owned fine nodes (prolongation output)
  static constexpr int RFB = 2 * K * CC + 2 * K + 1;  // fine nodes read (restriction)
  static constexpr int RFBp = RFB | 1;
  static constexpr int CN = K * CC;       // owned coarse nodes (restriction output)
  static constexpr int NT = 256;
  template <typename T>
  static constexpr size_t smem_prolong() {
    return sizeof(T) * (size_t)(DIM == 3 ? FB * CB * CBp + FB * FB * CBp : FB * CBp);
  }
  template <typename T>
  static constexpr size_t smem_restrict() {
    return sizeof(T) * (size_t)(DIM == 3 ? CN * RFB * RFBp + CN * CN * RFBp : CN * RFBp);
  }
};

// x_fine += P x_coarse.  Fine node 2K*C + s (s < 2K) of coarse cell C is
// sum_i P1[s][i] x_c[K*C + i] per direction; each block owns the fine nodes
// of its coarse cells (half-open), so no two blocks write the same node.
// The body processes the tile (bx, by, bz) of coarse cells; sP1 holds the 1D
// weights (filled by the caller, followed by a barrier).
template <typename T>
__device__ __forceinline__ void prolong_add_body(const T* __restrict__ xc, T* __restrict__ xf,
                                                 int n1c, int64_t pxc, int64_t pzc, int n1f,
                                                 int64_t pxf, int64_t pzf, int bx, int by, int bz,
                                                 const T* sP1) {
  using C = TransferCfg;
  constexpr int CB = C::CB, CBp = C::CBp, FB = C::FB, CC = C::CC, NT = C::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* t1 = reinterpret_cast<T*>(smem_raw);
  const int cx0 = bx * CC, cy0 = by * CC;
  if constexpr (DIM == 3) {
    const int cz0 = bz * CC;
    T* t2 = t1 + FB * CB * CBp;
    // along z from global: units (coarse y, coarse x) x coarse cell z
    for (int u = threadIdx.x; u < CB * CB * CC; u += NT) {
      const int xx = u % CB, yy = (u / CB) % CB, cz = u / (CB * CB);
      const int gx = K * cx0 + xx, gy = K * cy0 + yy;
      T v[K + 1];
#pragma unroll
      for (int i = 0; i <= K; ++i) {
        const int gz = K * (cz0 + cz) + i;
        v[i] = (gx < n1c && gy < n1c && gz < n1c) ? xc[(int64_t)gz * pzc + (int64_t)gy * pxc + gx]
                                                  : T(0);
      }
#pragma unroll
      for (int s = 0; s < 2 * K; ++s) {
        T acc = T(0);
#pragma unroll
        for (int i = 0; i <= K; ++i) acc = fma(c_tab<T>.P1[s * nl + i], v[i], acc);
        t1[((2 * K * cz + s) * CB + yy) * CBp + xx] = acc;
      }
    }
    __syncthreads();
    // along y: units (fine z, coarse cell y, coarse x)
    for (int u = threadIdx.x; u < FB * CC * CB; u += NT) {
      const int xx = u % CB, cy = (u / CB) % CC, Z = u / (CB * CC);
      T v[K + 1];
#pragma unroll
      for (int i = 0; i <= K; ++i) v[i] = t1[(Z * CB + K * cy + i) * CBp + xx];
#pragma unroll
      for (int s = 0; s < 2 * K; ++s) {
        T acc = T(0);
#pragma unroll
        for (int i = 0; i <= K; ++i) acc = fma(c_tab<T>.P1[s * nl + i], v[i], acc);
        t2[(Z * FB + 2 * K * cy + s) * CBp + xx] = acc;
      }
    }
    __syncthreads();
    // along x: one fine node per thread, x fastest, so that the update of the
    // fine vector is coalesced; the 1D weights come from shared memory (the
    // lanes of a warp need different rows of P1)
    for (int u = threadIdx.x; u < FB * FB * FB; u += NT) {
      const int X = u % FB, Y = (u / FB) % FB, Z = u / (FB * FB);
      const int gx = 2 * K * cx0 + X, gy = 2 * K * cy0 + Y, gz = 2 * K * cz0 + Z;
      if (gx < 1 || gx > n1f - 2 || gy < 1 || gy > n1f - 2 || gz < 1 || gz > n1f - 2) continue;
      const int cx = X / (2 * K), sx = X % (2 * K);
      const T* src = t2 + (Z * FB + Y) * CBp + K * cx;
      const T* w = sP1 + sx * nl;
      T acc = T(0);
#pragma unroll
      for (int i = 0; i <= K; ++i) acc = fma(w[i], src[i], acc);
      xf[(int64_t)gz * pzf + (int64_t)gy * pxf + gx] += acc;
    }
  } else {
    // along y from global: units (coarse x) x coarse cell y
    for (int u = threadIdx.x; u < CB * CC; u += NT) {
      const int xx = u % CB, cy = u / CB;
      const int gx = K * cx0 + xx;
      T v[K + 1];
#pragma unroll
      for (int i = 0; i <= K; ++i) {
        const int gy = K * (cy0 + cy) + i;
        v[i] = (gx < n1c && gy < n1c) ? xc[(int64_t)gy * pxc + gx] : T(0);
      }
#pragma unroll
      for (int s = 0; s < 2 * K; ++s) {
        T acc = T(0);
#pragma unroll
        for (int i = 0; i <= K; ++i) acc = fma(c_tab<T>.P1[s * nl + i], v[i], acc);
        t1[(2 * K * cy + s) * CBp + xx] = acc;
      }
    }
    __syncthreads();
    for (int u = threadIdx.x; u < FB * FB; u += NT) {  // one fine node per thread, x fastest
      const int X = u % FB, Y = u / FB;
      const int gx = 2 * K * cx0 + X, gy = 2 * K * cy0 + Y;
      if (gx < 1 || gx > n1f - 2 || gy < 1 || gy > n1f - 2) continue;
      const int cx = X / (2 * K), sx = X % (2 * K);
      const T* src = t1 + Y * CBp + K * cx;
      const T* w = sP1 + sx * nl;
      T acc = T(0);
#pragma unroll
      for (int i = 0; i <= K; ++i) acc = fma(w[i], src[i], acc);
      xf[(int64_t)gy * pxf + gx] += acc;
    }
  }
  (void)pzc;
  (void)pzf;
  (void)bz;
}

template <typename T>
__global__ void __launch_bounds__(TransferCfg::NT)
prolong_add_kernel(const T* __restrict__ xc, T* __restrict__ xf, int n1c, int64_t pxc,
                   int64_t pzc, int n1f, int64_t pxf, int64_t pzf) {
  __shared__ T sP1[2 * K * nl];
  for (int e = threadIdx.x; e < 2 * K * nl; e += TransferCfg::NT) sP1[e] = c_tab<T>.P1[e];
  __syncthreads();
  prolong_add_body<T>(xc, xf, n1c, pxc, pzc, n1f, pxf, pzf, blockIdx.x, blockIdx.y, blockIdx.z,
                      sP1);
}

// Tile r of a transfer item -> (bx, by, bz) on a t^DIM grid of tiles.
__device__ __forceinline__ void transfer_tile(int64_t r, int t, int* bx, int* by, int* bz) {
  *bx = (int)(r % t);
  *by = (int)((r / t) % t);
  *bz = DIM == 3 ? (int)(r / ((int64_t)t * t)) : 0;
}

// Persistent prolongations x_fine += P x_coarse of several levels (queue
// items: in = x_coarse, out = x_fine; a: coarse layout, b: fine layout).
template <typename T>
__global__ void __launch_bounds__(TransferCfg::NT)
prolong_add_batch_kernel(BatchQueue* __restrict__ q) {
  __shared__ T sP1[2 * K * nl];
  for (int e = threadIdx.x; e < 2 * K * nl; e += TransferCfg::NT) sP1[e] = c_tab<T>.P1[e];
  __syncthreads();
  int64_t t;
  int it;
  while (next_batch_tile(q, &t, &it)) {
    const BatchItem& I = q->items[it];
    int bx, by, bz;
    transfer_tile(t - I.tile0, I.tiles_per_dim, &bx, &by, &bz);
    prolong_add_body<T>(static_cast<const T*>(I.in), static_cast<T*>(I.out), I.n1a, I.pxa, I.pza,
                        I.n1b, I.pxb, I.pzb, bx, by, bz, sP1);
    __syncthreads();
  }
}

// Restriction r_c = P^T r_f per direction: coarse node K*C + i gathers the
// fine nodes of coarse cell C with weights P1[s][i]; a coarse vertex (i = 0)
// also gathers cell C-1 with weights P1[s][K] (the shared fine node once).
// v holds the 4K+1 fine values of cells C-1 and C.
template <typename T>
__device__ __forceinline__ void restrict_1d(const T (&v)[4 * K + 1], T (&out)[K]) {
#pragma unroll
  for (int i = 0; i < K; ++i) {
    T acc = T(0);
#pragma unroll
    for (int s = 0; s <= 2 * K; ++s) acc = fma(c_tab<T>.P1[s * nl + i], v[2 * K + s], acc);
    if (i == 0) {
#pragma unroll
      for (int s = 0; s < 2 * K; ++s) acc = fma(c_tab<T>.P1[s * nl + K], v[s], acc);
    }
    out[i] = acc;
  }
}

template <typename T>
__device__ __forceinline__ void restrict_body(const T* __restrict__ rf, T* __restrict__ rc,
                                              int n1c, int64_t pxc, int64_t pzc, int n1f,
                                              int64_t pxf, int64_t pzf, int bx, int by, int bz) {
  using C = TransferCfg;
  constexpr int RFB = C::RFB, RFBp = C::RFBp, CN = C::CN, CC = C::CC, NT = C::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* t1 = reinterpret_cast<T*>(smem_raw);
  const int C0x = bx * CC, C0y = by * CC;
  const int fx0 = 2 * K * (C0x - 1), fy0 = 2 * K * (C0y - 1);
  if constexpr (DIM == 3) {
    const int C0z = bz * CC;
    T* t2 = t1 + CN * RFB * RFBp;
    // along z from global: units (fine y, fine x) x coarse cell z
    for (int u = threadIdx.x; u < RFB * RFB * CC; u += NT) {
      const int xx = u % RFB, yy = (u / RFB) % RFB, cz = u / (RFB * RFB);
      const int gx = fx0 + xx, gy = fy0 + yy, gz0 = 2 * K * (C0z + cz - 1);
      const bool inxy = gx >= 0 && gx < n1f && gy >= 0 && gy < n1f;
      T v[4 * K + 1], o[K];
#pragma unroll
      for (int i = 0; i <= 4 * K; ++i) {
        const int gz = gz0 + i;
        v[i] = (inxy && gz >= 0 && gz < n1f) ? rf[(int64_t)gz * pzf + (int64_t)gy * pxf + gx] : T(0);
      }
      restrict_1d<T>(v, o);
#pragma unroll
      for (int i = 0; i < K; ++i) t1[((K * cz + i) * RFB + yy) * RFBp + xx] = o[i];
    }
    __syncthreads();
    // along y: units (coarse z, coarse cell y, fine x)
    for (int u = threadIdx.x; u < CN * CC * RFB; u += NT) {
      const int xx = u % RFB, cy = (u / RFB) % CC, Z = u / (RFB * CC);
      T v[4 * K + 1], o[K];
#pragma unroll
      for (int i = 0; i <= 4 * K; ++i) v[i] = t1[(Z * RFB + 2 * K * cy + i) * RFBp + xx];
      restrict_1d<T>(v, o);
#pragma unroll
      for (int i = 0; i < K; ++i) t2[(Z * CN + K * cy + i) * RFBp + xx] = o[i];
    }
    __syncthreads();
    // along x: units (coarse y fastest, coarse z, coarse cell x); write
    for (int u = threadIdx.x; u < CN * CN * CC; u += NT) {
      const int Y = u % CN, Z = (u / CN) % CN, cx = u / (CN * CN);
      const int gy = K * C0y + Y, gz = K * C0z + Z;
      if (gy >= n1c || gz >= n1c) continue;
      T v[4 * K + 1], o[K];
#pragma unroll
      for (int i = 0; i <= 4 * K; ++i) v[i] = t2[(Z * CN + Y) * RFBp + 2 * K * cx + i];
      restrict_1d<T>(v, o);
      const bool inner_yz = gy >= 1 && gy <= n1c - 2 && gz >= 1 && gz <= n1c - 2;
      T* dst = rc + (int64_t)gz * pzc + (int64_t)gy * pxc;
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int gx = K * (C0x + cx) + i;
        if (gx >= n1c) continue;
        dst[gx] = (inner_yz && gx >= 1 && gx <= n1c - 2) ? o[i] : T(0);
      }
    }
  } else {
    for (int u = threadIdx.x; u < RFB * CC; u += NT) {
      const int xx = u % RFB, cy = u / RFB;
      const int gx = fx0 + xx, gy0 = 2 * K * (C0y + cy - 1);
      T v[4 * K + 1], o[K];
#pragma unroll
      for (int i = 0; i <= 4 * K; ++i) {
        const int gy = gy0 + i;
        v[i] = (gx >= 0 && gx < n1f && gy >= 0 && gy < n1f) ? rf[(int64_t)gy * pxf + gx] : T(0);
      }
      restrict_1d<T>(v, o);
#pragma unroll
      for (int i = 0; i < K; ++i) t1[(K * cy + i) * RFBp + xx] = o[i];
    }
    __syncthreads();
    for (int u = threadIdx.x; u < CN * CC; u += NT) {
      const int Y = u % CN, cx = u / CN;
      const int gy = K * C0y + Y;
      if (gy >= n1c) continue;
      T v[4 * K + 1], o[K];
#pragma unroll
      for (int i = 0; i <= 4 * K; ++i) v[i] = t1[Y * RFBp + 2 * K * cx + i];
      restrict_1d<T>(v, o);
      T* dst = rc + (int64_t)gy * pxc;
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int gx = K * (C0x + cx) + i;
        if (gx >= n1c) continue;
        dst[gx] = (gy >= 1 && gy <= n1c - 2 && gx >= 1 && gx <= n1c - 2) ? o[i] : T(0);
      }
    }
  }
  (void)pzc;
  (void)bz;
}

template <typename T>
__global__ void __launch_bounds__(TransferCfg::NT)
restrict_kernel(const T* __restrict__ rf, T* __restrict__ rc, int n1c, int64_t pxc, int64_t pzc,
                int n1f, int64_t pxf, int64_t pzf) {
  block_zero_faces<T>(rc, n1c, pxc, pzc);
  restrict_body<T>(rf, rc, n1c, pxc, pzc, n1f, pxf, pzf, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Persistent restrictions r_coarse = P^T r_fine of several levels (queue
// items: in = r_fine, out = r_coarse; a: coarse layout, b: fine layout).
template <typename T>
__global__ void __launch_bounds__(TransferCfg::NT)
restrict_batch_kernel(BatchQueue* __restrict__ q) {
  int64_t t;
  int it;
  while (next_batch_tile(q, &t, &it)) {
    const BatchItem& I = q->items[it];
    int bx, by, bz;
    transfer_tile(t - I.tile0, I.tiles_per_dim, &bx, &by, &bz);
    restrict_body<T>(static_cast<const T*>(I.in), static_cast<T*>(I.out), I.n1a, I.pxa, I.pza,
                     I.n1b, I.pxb, I.pzb, bx, by, bz);
    __syncthreads();
  }
}


// The upper faces of the `out` vectors (layout a) of every item of a queue:
// blockIdx.y selects the item.
template <typename T>
__global__ void zero_upper_faces_batch_kernel(const BatchQueue* __restrict__ q) {
  if ((int)blockIdx.y >= q->nitems) return;
  const BatchItem& I = q->items[blockIdx.y];
  zero_upper_faces_body<T>(static_cast<T*>(I.out), I.n1a, I.pxa, I.pza,
                           blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                           (int64_t)gridDim.x * blockDim.x);
}

// ------------------------------------------------------------ launchers
template <typename T, int PP, bool BND, int W>
cudaError_t smooth_mult_launch(const LevelGeom& g, const ColourGeom& cg, const T* b, T* x,
                               const T* inv_lam, cudaStream_t s) {
  using C = SmoothCfg<T, PP, W>;  // PP: block shape, W: warps (0: automatic)
  if (cg.npatch == 0) return cudaSuccess;
  const int64_t grid = (cg.npatch + C::P - 1) / C::P;
  const T bscale = DIM == 3 ? T(1.0 / g.h) : T(1);
  VPS_COUNT_LAUNCH();
  return launch_pdl(smooth_mult_kernel<T, PP, BND, W, false>, dim3((unsigned)grid), dim3(C::NT),
                    BND ? C::smem_bnd : C::smem_mult, s, b, x, inv_lam, (int)g.px, (int)g.pz,
                    cg, bscale, static_cast<T*>(nullptr));
}

// Multiprocessor count of the current device (first call).
int sm_count() {
  static int n = 0;
  if (n == 0) {
    int d = 0, v = 0;
    if (cudaGetDevice(&d) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) == cudaSuccess && v > 0)
      n = v;
    else
      return 1;
  }
  return n;
}

// Grid of a persistent batched launch: every resident block slot of the GPU
// (occupancy of the kernel at its block size and shared memory), at most
// one block per tile.
template <typename KernT>
cudaError_t persistent_grid(KernT kern, int nt, size_t smem, int64_t ntiles, int* per_sm,
                            unsigned* grid) {
  if (*per_sm <= 0) {
    int nb = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, nt, smem);
    if (e != cudaSuccess) return e;
    *per_sm = nb > 0 ? nb : 1;
  }
  const int64_t cap = (int64_t)(*per_sm) * sm_count();
  *grid = (unsigned)(ntiles < cap ? ntiles : cap);
  return cudaSuccess;
}

template <typename T, int PP, bool BND, int W>
cudaError_t smooth_mult_batch_launch(BatchQueue* q, int64_t ntiles, const T* inv_lam,
                                     cudaStream_t s) {
  using C = SmoothCfg<T, PP, W>;
  if (ntiles <= 0) return cudaSuccess;
  static int per_sm = 0;
  const size_t smem = BND ? C::smem_bnd : C::smem_mult;
  unsigned grid = 0;
  cudaError_t e = persistent_grid(smooth_mult_batch_kernel<T, PP, BND, W>, C::NT, smem, ntiles,
                                  &per_sm, &grid);
  if (e != cudaSuccess) return e;
  VPS_COUNT_LAUNCH();
  smooth_mult_batch_kernel<T, PP, BND, W><<<grid, C::NT, smem, s>>>(q, inv_lam);
  return cudaGetLastError();
}

// A smoothing step as one dataflow sweep (smooth_sweep_kernel, one block per
// tile of every colour), launched as a programmatic dependent launch (the
// kernel waits for the previous one before it reads the counters or x).
template <typename T, int PP, bool BND, int W = 0>
cudaError_t smooth_sweep_launch(const LevelGeom& g, const SweepGeom& sg, const T* b, T* x,
                                const T* inv_lam, cudaStream_t s) {
  using C = SmoothCfg<T, PP, W>;
  const int64_t ntiles = sg.ncol > 0 ? sg.tile_end[sg.ncol - 1] : 0;
  if (ntiles <= 0) return cudaSuccess;
  if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  const size_t smem = BND ? C::smem_bnd : C::smem_mult;
  const T bscale = DIM == 3 ? T(1.0 / g.h) : T(1);
  VPS_COUNT_LAUNCH();
  return launch_pdl(smooth_sweep_kernel<T, PP, BND, W>, dim3((unsigned)ntiles), dim3(C::NT), smem, s,
                    b, x, inv_lam, (int)g.px, (int)g.pz, sg, bscale);
}

template <typename T>
cudaError_t restrict_batch_launch(BatchQueue* q, int64_t ntiles, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  static int per_sm = 0;
  const size_t smem = TransferCfg::smem_restrict<T>();
  unsigned grid = 0;
  cudaError_t e = persistent_grid(restrict_batch_kernel<T>, TransferCfg::NT, smem, ntiles, &per_sm,
                                  &grid);
  if (e != cudaSuccess) return e;
  VPS_COUNT_LAUNCH();
  restrict_batch_kernel<T><<<grid, TransferCfg::NT, smem, s>>>(q);
  return cudaGetLastError();
}

template <typename T>
cudaError_t prolong_batch_launch(BatchQueue* q, int64_t ntiles, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  static int per_sm = 0;
  const size_t smem = TransferCfg::smem_prolong<T>();
  unsigned grid = 0;
  cudaError_t e = persistent_grid(prolong_add_batch_kernel<T>, TransferCfg::NT, smem, ntiles,
                                  &per_sm, &grid);
  if (e != cudaSuccess) return e;
  VPS_COUNT_LAUNCH();
  prolong_add_batch_kernel<T><<<grid, TransferCfg::NT, smem, s>>>(q);
  return cudaGetLastError();
}

template <typename T>
cudaError_t zero_faces_batch_launch(const BatchQueue* q, int nitems, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  VPS_COUNT_LAUNCH();
  zero_upper_faces_batch_kernel<T><<<dim3(64, (unsigned)nitems), 256, 0, s>>>(q);
  return cudaGetLastError();
}

// The colour pass as an ordinary launch (no programmatic dependent launch;
// griddepcontrol.wait is then a no-op).
template <typename T, int PP, bool BND, int W>
cudaError_t smooth_mult_plain_launch(const LevelGeom& g, const ColourGeom& cg, const T* b, T* x,
                                     const T* inv_lam, cudaStream_t s) {
  using C = SmoothCfg<T, PP, W>;
  if (cg.npatch == 0) return cudaSuccess;
  const int64_t grid = (cg.npatch + C::P - 1) / C::P;
  const T bscale = DIM == 3 ? T(1.0 / g.h) : T(1);
  VPS_COUNT_LAUNCH();
  smooth_mult_kernel<T, PP, BND, W, false><<<(unsigned)grid, C::NT, BND ? C::smem_bnd : C::smem_mult,
                                             s>>>(b, x, inv_lam, (int)g.px, (int)g.pz, cg, bscale,
                                                  static_cast<T*>(nullptr));
  return cudaGetLastError();
}

// The colour pass with one thread per patch (kind 5): smooth_q1_kernel for
// k = 1, smooth_patch2d_kernel for 2D k = 2, 3.
template <typename T>
constexpr auto patch_thread_kernel() {
  if constexpr (K == 1) return smooth_q1_kernel<T>;
  else return smooth_patch2d_kernel<T>;
}

template <typename T>
cudaError_t smooth_q1_launch(const LevelGeom& g, const ColourGeom& cg, const T* b, T* x,
                             const T* inv_lam, cudaStream_t s) {
  if (cg.npatch == 0) return cudaSuccess;
  const int64_t grid = (cg.npatch + kQ1Threads - 1) / kQ1Threads;
  const T bscale = DIM == 3 ? T(1.0 / g.h) : T(1);
  VPS_COUNT_LAUNCH();
  return launch_pdl(patch_thread_kernel<T>(), dim3((unsigned)grid), dim3(kQ1Threads), 0, s, b, x,
                    inv_lam, (int)g.px, (int)g.pz, cg, bscale);
}

template <typename T>
cudaError_t smooth_q1_plain_launch(const LevelGeom& g, const ColourGeom& cg, const T* b, T* x,
                                   const T* inv_lam, cudaStream_t s) {
  if (cg.npatch == 0) return cudaSuccess;
  const int64_t grid = (cg.npatch + kQ1Threads - 1) / kQ1Threads;
  const T bscale = DIM == 3 ? T(1.0 / g.h) : T(1);
  VPS_COUNT_LAUNCH();
  patch_thread_kernel<T>()<<<(unsigned)grid, kQ1Threads, 0, s>>>(b, x, inv_lam, (int)g.px,
                                                                 (int)g.pz, cg, bscale);
  return cudaGetLastError();
}

template <typename T, int PP>
cudaError_t resid_launch(const LevelGeom& g, const ColourGeom& cg, const T* b, const T* x, T* r,
                         cudaStream_t s) {
  using C = SmoothCfg<T, PP, 0>;
  if (cg.npatch == 0) return cudaSuccess;
  const int64_t grid = (cg.npatch + C::P - 1) / C::P;
  const T bscale = DIM == 3 ? T(1.0 / g.h) : T(1);
  VPS_COUNT_LAUNCH();
  smooth_mult_kernel<T, PP, false, 0, true><<<(unsigned)grid, C::NT, C::smem_mult, s>>>(
      b, const_cast<T*>(x), nullptr, (int)g.px, (int)g.pz, cg, bscale, r);
  return cudaGetLastError();
}

template <typename T>
cudaError_t inverse_launch(const LevelGeom& g, const ColourGeom& cg, const T* r, T* x,
                           const T* AinvT, cudaStream_t s) {
  if constexpr (!kInvFits) {
    return cudaErrorInvalidValue;
  } else {
    if (cg.npatch == 0) return cudaSuccess;
    const T scale = DIM == 3 ? T(1.0 / g.h) : T(1);
    VPS_COUNT_LAUNCH();
    inverse_solve_kernel<T><<<(unsigned)cg.npatch, kInvThreads, 0, s>>>(r, x, AinvT, (int)g.px,
                                                                          (int)g.pz, cg, scale);
    return cudaGetLastError();
  }
}

template <typename T, int PP>
cudaError_t smooth_add_launch(const LevelGeom& g, const ColourGeom& cg, const T* r, T* x,
                              const T* inv_lam, T scale, cudaStream_t s) {
  using C = SmoothCfg<T, PP>;  // PP: block shape
  if (cg.npatch == 0) return cudaSuccess;
  const int64_t grid = (cg.npatch + C::P - 1) / C::P;
  const T sc = DIM == 3 ? T(scale / g.h) : scale;
  VPS_COUNT_LAUNCH();
  smooth_add_kernel<T, PP><<<(unsigned)grid, C::NT, C::smem_add, s>>>(r, x, inv_lam, (int)g.px,
                                                                       (int)g.pz, cg, sc);
  return cudaGetLastError();
}

// Planes per block of the per-plane 3D operators (apply3_kernel,
// apply3_df_kernel) for `planes` planes and tiles_xy tiles per plane: a
// launch takes about (rounds of resident blocks) x (planes per block), so
// the zpb that minimises ceil(tiles_xy ceil(planes / zpb) / slots) zpb,
// slots = the kernel's resident blocks per SM x SMs; on ties the most
// planes per block (fewest blocks).  A fixed cell of planes per block left
// the last round two-thirds full on 2^5 cells at k = 4 (512 blocks for 304
// slots); 7 planes per block fill one round.
template <typename KernT>
int planes_per_block(KernT kern, size_t smem, int planes, int64_t tiles_xy, int* per_sm) {
  if (*per_sm <= 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, Apply3Cfg::NT, smem) !=
            cudaSuccess ||
        nb <= 0)
      nb = 1;
    *per_sm = nb;
  }
  const int64_t slots = (int64_t)(*per_sm) * sm_count();
  int best = planes;
  int64_t best_cost = INT64_MAX;
  for (int zp = planes; zp >= 1; --zp) {
    const int64_t blocks = tiles_xy * ((planes + zp - 1) / zp);
    const int64_t cost = ((blocks + slots - 1) / slots) * zp;
    if (cost < best_cost) {
      best_cost = cost;
      best = zp;
    }
  }
  return best;
}

// Launch of apply3_kernel<T, ABS> over a level (tiles of TX x TX nodes in x
// and y, runs of planes in z).
template <typename T, bool ABS>
cudaError_t apply3_launch(const LevelGeom& g, const T* x, const T* b, T* y, T scale,
                          cudaStream_t s) {
  using C3 = Apply3Cfg;
  static int per_sm = 0;
  const int span = g.n1 - 1;
  const unsigned t = (unsigned)((span + C3::TX - 1) / C3::TX);
  const int zpb = planes_per_block(apply3_kernel<T, ABS>, C3::smem<T>(), span, (int64_t)t * t,
                                   &per_sm);
  const unsigned tz = (unsigned)((span + zpb - 1) / zpb);
  VPS_COUNT_LAUNCH();
  apply3_kernel<T, ABS><<<dim3(t, t, tz), C3::NT, C3::smem<T>(), s>>>(x, b, y, g.n1, (int)g.px,
                                                                      (int)g.pz, scale, zpb);
  return cudaGetLastError();
}

// Tiles cover the nodes 0 .. n1-2 of every direction; the upper boundary
// layer (index n1-1) is zeroed by the kernel's blocks (block_zero_faces).
// The per-plane 3D operator where the default is the cell-batched one.
template <typename T>
cudaError_t apply_alt_launch(const LevelGeom& g, const T* x, const T* b, T* y, cudaStream_t s) {
  if constexpr (DIM == 3 && kApply3C<T>) {
    return apply3_launch<T, false>(g, x, b, y, T(g.h), s);
  } else {
    (void)g; (void)x; (void)b; (void)y; (void)s;
    return cudaErrorNotSupported;
  }
}

template <typename T>
cudaError_t apply_launch(const LevelGeom& g, const T* x, const T* b, T* y, cudaStream_t s) {
  const int span = g.n1 - 1;
  if constexpr (DIM == 3) {
    if constexpr (kApply3C<T>) {
      using C3 = Apply3Cfg;
      const unsigned t = (unsigned)((span + C3::TX - 1) / C3::TX);
      const unsigned tz = (unsigned)((span + kApply3CZ * K - 1) / (kApply3CZ * K));
      VPS_COUNT_LAUNCH();
      apply3c_kernel<T><<<dim3(t, t, tz), C3::NT, C3::smem_c<T>(), s>>>(x, b, y, g.n1, (int)g.px,
                                                                        (int)g.pz, T(g.h));
    } else {
      return apply3_launch<T, false>(g, x, b, y, T(g.h), s);
    }
  } else {
    using C = ApplyCfg;
    const unsigned t = (unsigned)((span + C::TN - 1) / C::TN);
    VPS_COUNT_LAUNCH();
    apply_kernel<T><<<dim3(t, t, 1), C::NT, C::smem<T>(), s>>>(x, b, y, g.n1, g.px, g.pz, T(1));
  }
  return cudaGetLastError();
}

// y = |A| |x| with the band coefficients replaced by their absolute values
// (an upper bound of sum_j |A_ij| |x_j| for every row): the scale of the
// rounding error of any FP64 evaluation of A x.
cudaError_t apply_abs_launch(const LevelGeom& g, const double* x, double* y, cudaStream_t s) {
  const int span = g.n1 - 1;
  if constexpr (DIM == 3) {
    return apply3_launch<double, true>(g, x, static_cast<const double*>(nullptr), y, g.h, s);
  } else {
    using C = ApplyCfg;
    const unsigned t = (unsigned)((span + C::TN - 1) / C::TN);
    VPS_COUNT_LAUNCH();
    apply_kernel<double, true><<<dim3(t, t, 1), C::NT, C::smem<double>(), s>>>(
        x, nullptr, y, g.n1, g.px, g.pz, 1.0);
  }
  return cudaGetLastError();
}

cudaError_t apply_df_launch(const LevelGeom& g, const float* xh, const float* xl, double* y,
                            cudaStream_t s) {
  const int span = g.n1 - 1;
  if constexpr (DIM == 3) {
    using C3 = Apply3Cfg;
    static int per_sm = 0;
    const unsigned t = (unsigned)((span + C3::TX - 1) / C3::TX);
    const int zpb = planes_per_block(apply3_df_kernel<0>, C3::smem<double>(), span,
                                     (int64_t)t * t, &per_sm);
    const unsigned tz = (unsigned)((span + zpb - 1) / zpb);
    VPS_COUNT_LAUNCH();
    // g.h = 1 / 2^level: exact as a float
    apply3_df_kernel<0><<<dim3(t, t, tz), C3::NT, C3::smem<double>(), s>>>(xh, xl, y, g.n1,
                                                                          (int)g.px, (int)g.pz,
                                                                          (float)g.h, zpb);
  } else {
    using C = ApplyCfg;
    const unsigned t = (unsigned)((span + C::TN - 1) / C::TN);
    VPS_COUNT_LAUNCH();
    apply2_df_kernel<0><<<dim3(t, t, 1), C::NT, C::smem<double>(), s>>>(xh, xl, y, g.n1,
                                                                       (int)g.px);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t prolong_launch(const LevelGeom& f, const LevelGeom& c, const T* xc, T* xf,
                           cudaStream_t s) {
  using C = TransferCfg;
  const unsigned t = (unsigned)((c.ncell + C::CC - 1) / C::CC);
  dim3 grid(t, t, DIM == 3 ? t : 1);
  VPS_COUNT_LAUNCH();
  prolong_add_kernel<T><<<grid, C::NT, C::smem_prolong<T>(), s>>>(xc, xf, c.n1, c.px, c.pz, f.n1,
                                                                   f.px, f.pz);
  return cudaGetLastError();
}

template <typename T>
cudaError_t restrict_launch(const LevelGeom& f, const LevelGeom& c, const T* rf, T* rc,
                            cudaStream_t s) {
  using C = TransferCfg;
  const unsigned t = (unsigned)((c.ncell + C::CC - 1) / C::CC);
  dim3 grid(t, t, DIM == 3 ? t : 1);
  VPS_COUNT_LAUNCH();
  restrict_kernel<T><<<grid, C::NT, C::smem_restrict<T>(), s>>>(rf, rc, c.n1, c.px, c.pz, f.n1,
                                                                 f.px, f.pz);
  return cudaGetLastError();
}

// Dynamic shared memory of a smoother kernel, and the largest shared-memory
// carveout of the SM's unified L1/shared storage: the number of patches in
// flight per SM is bounded by shared memory (registers allow more), and the
// default carveout leaves part of the 228 KB unused.
template <typename KernT>
cudaError_t smoother_smem(KernT kern, size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared);
}

// The fewer-warps kinds 3 and 4 exist for a block shape where they launch
// fewer threads than the automatic block of kinds 0 and 1.
template <typename T, int PP>
constexpr bool kFewWarps = 32 * warps_min(PP) < SmoothCfg<T, PP>::NT;

template <typename T, int PP>
cudaError_t smooth_few_warps_limits() {
  if constexpr (kFewWarps<T, PP>) {
    constexpr int Wm = warps_min(PP);
    using CW = SmoothCfg<T, PP, Wm>;
    cudaError_t e = cudaSuccess;
    if constexpr (CW::fits_bnd) {
      if ((e = smoother_smem(smooth_mult_kernel<T, PP, true, Wm>, CW::smem_bnd)) ||
          (e = smoother_smem(smooth_mult_batch_kernel<T, PP, true, Wm>, CW::smem_bnd)) ||
          (e = smoother_smem(smooth_sweep_kernel<T, PP, true, Wm>, CW::smem_bnd)))
        return e;
    }
    if constexpr (CW::fits) {
      if ((e = smoother_smem(smooth_mult_kernel<T, PP, false, Wm>, CW::smem_mult)) ||
          (e = smoother_smem(smooth_mult_batch_kernel<T, PP, false, Wm>, CW::smem_mult)) ||
          (e = smoother_smem(smooth_sweep_kernel<T, PP, false, Wm>, CW::smem_mult)))
        return e;
    }
  }
  return cudaSuccess;
}

template <typename T, int PP>
cudaError_t smooth_limits() {
  using C = SmoothCfg<T, PP>;
  if (cudaError_t e = smooth_few_warps_limits<T, PP>(); e != cudaSuccess) return e;
  if constexpr (C::fits_bnd) {
    cudaError_t e = smoother_smem(smooth_mult_kernel<T, PP, true, 0>, C::smem_bnd);
    if (e != cudaSuccess) return e;
    if constexpr (kOneWarpVariants) {
      // the one-warp blocks run their stages in several rounds: no buffer
      // overlay, so their own (larger) shared-memory size
      using C1 = SmoothCfg<T, PP, 1>;
      e = smoother_smem(smooth_mult_kernel<T, PP, true, 1>, C1::smem_bnd);
      if (e != cudaSuccess) return e;
      e = smoother_smem(smooth_mult_batch_kernel<T, PP, true, 1>, C1::smem_bnd);
      if (e != cudaSuccess) return e;
    }
    e = smoother_smem(smooth_mult_batch_kernel<T, PP, true, 0>, C::smem_bnd);
    if (e != cudaSuccess) return e;
    e = smoother_smem(smooth_sweep_kernel<T, PP, true>, C::smem_bnd);
    if (e != cudaSuccess) return e;
  }
  if constexpr (!C::fits) {
    return cudaSuccess;
  } else {
    cudaError_t e = smoother_smem(smooth_mult_kernel<T, PP, false, 0>, C::smem_mult);
    if (e != cudaSuccess) return e;
    e = smoother_smem(smooth_mult_kernel<T, PP, false, 0, true>, C::smem_mult);
    if (e != cudaSuccess) return e;
    e = smoother_smem(smooth_mult_batch_kernel<T, PP, false, 0>, C::smem_mult);
    if (e != cudaSuccess) return e;
    e = smoother_smem(smooth_sweep_kernel<T, PP, false>, C::smem_mult);
    if (e != cudaSuccess) return e;
    return smoother_smem(smooth_add_kernel<T, PP>, C::smem_add);
  }
}

// Kinds 3 (fused) and 4 (Boundary) of block shape PP: the blocks of
// warps_min(PP) warps; multiplicative smoother only.
template <typename T, int PP>
void register_few_warps(KernelFns<T>* f, int v) {
  constexpr int vf = v0_kind(3), vb = v0_kind(4);
  f->variant_p[vf + v] = f->variant_p[vb + v] = SmoothCfg<T, PP>::P;
  f->smooth_add_v[vf + v] = f->smooth_add_v[vb + v] = nullptr;
  f->smooth_mult_v[vf + v] = f->smooth_mult_plain_v[vf + v] = nullptr;
  f->smooth_mult_batch_v[vf + v] = nullptr;
  f->smooth_sweep_v[vf + v] = nullptr;
  f->smooth_mult_v[vb + v] = f->smooth_mult_plain_v[vb + v] = nullptr;
  f->smooth_mult_batch_v[vb + v] = nullptr;
  f->smooth_sweep_v[vb + v] = nullptr;
  if constexpr (kFewWarps<T, PP>) {
    constexpr int Wm = warps_min(PP);
    using CW = SmoothCfg<T, PP, Wm>;
    if constexpr (CW::fits) {
      f->smooth_mult_v[vf + v] = smooth_mult_launch<T, PP, false, Wm>;
      f->smooth_mult_plain_v[vf + v] = smooth_mult_plain_launch<T, PP, false, Wm>;
      f->smooth_mult_batch_v[vf + v] = smooth_mult_batch_launch<T, PP, false, Wm>;
      f->smooth_sweep_v[vf + v] = smooth_sweep_launch<T, PP, false, Wm>;
    }
    if constexpr (CW::fits_bnd) {
      f->smooth_mult_v[vb + v] = smooth_mult_launch<T, PP, true, Wm>;
      f->smooth_mult_plain_v[vb + v] = smooth_mult_plain_launch<T, PP, true, Wm>;
      f->smooth_mult_batch_v[vb + v] = smooth_mult_batch_launch<T, PP, true, Wm>;
      f->smooth_sweep_v[vb + v] = smooth_sweep_launch<T, PP, true, Wm>;
    }
  }
}

// Kind 5 (variant 15): the colour pass with one thread per patch -- the
// point Gauss-Seidel form for k = 1, the patch in registers for 2D k = 2, 3
// (FP32 only at k = 3, whose FP64 patch would not fit the registers);
// multiplicative smoother only.
template <typename T>
constexpr bool kPatchThread = K == 1 || (DIM == 2 && (K == 2 || (K == 3 && sizeof(T) == 4)));

template <typename T>
void register_q1(KernelFns<T>* f, int v) {
  const int vq = v0_kind(5) + v;
  f->variant_p[vq] = 0;
  f->smooth_add_v[vq] = nullptr;
  f->smooth_mult_v[vq] = f->smooth_mult_plain_v[vq] = nullptr;
  f->smooth_mult_batch_v[vq] = nullptr;
  f->smooth_sweep_v[vq] = nullptr;
  if constexpr (kPatchThread<T>) {
    if (v == 0) {
      f->variant_p[vq] = kQ1Threads;
      f->smooth_mult_v[vq] = smooth_q1_launch<T>;
      f->smooth_mult_plain_v[vq] = smooth_q1_plain_launch<T>;
    }
  }
}

template <typename T, int PP>
void register_variant(KernelFns<T>* f, int v) {
  using C = SmoothCfg<T, PP>;
  register_few_warps<T, PP>(f, v);
  register_q1<T>(f, v);
  f->variant_p[v] = C::P;
  f->variant_p[v + kQVariants] = C::P;
  f->variant_p[v + 2 * kQVariants] = C::P;
  f->smooth_add_v[v + kQVariants] = nullptr;
  f->smooth_add_v[v + 2 * kQVariants] = nullptr;
  f->smooth_sweep_v[v + 2 * kQVariants] = nullptr;
  if constexpr (C::fits_bnd) {
    f->smooth_sweep_v[v + kQVariants] = smooth_sweep_launch<T, PP, true>;
    f->smooth_mult_v[v + kQVariants] = smooth_mult_launch<T, PP, true, 0>;
    f->smooth_mult_plain_v[v + kQVariants] = smooth_mult_plain_launch<T, PP, true, 0>;
    f->smooth_mult_batch_v[v + kQVariants] = smooth_mult_batch_launch<T, PP, true, 0>;
    if constexpr (kOneWarpVariants) {
      f->smooth_mult_v[v + 2 * kQVariants] = smooth_mult_launch<T, PP, true, 1>;
      f->smooth_mult_plain_v[v + 2 * kQVariants] = smooth_mult_plain_launch<T, PP, true, 1>;
      f->smooth_mult_batch_v[v + 2 * kQVariants] = smooth_mult_batch_launch<T, PP, true, 1>;
    } else {
      f->smooth_mult_v[v + 2 * kQVariants] = nullptr;
      f->smooth_mult_plain_v[v + 2 * kQVariants] = nullptr;
      f->smooth_mult_batch_v[v + 2 * kQVariants] = nullptr;
    }
  } else {
    f->smooth_sweep_v[v + kQVariants] = nullptr;
    f->smooth_mult_v[v + kQVariants] = nullptr;
    f->smooth_mult_v[v + 2 * kQVariants] = nullptr;
    f->smooth_mult_plain_v[v + kQVariants] = nullptr;
    f->smooth_mult_plain_v[v + 2 * kQVariants] = nullptr;
    f->smooth_mult_batch_v[v + kQVariants] = nullptr;
    f->smooth_mult_batch_v[v + 2 * kQVariants] = nullptr;
  }
  if constexpr (C::fits) f->resid_v[v] = resid_launch<T, PP>;
  else f->resid_v[v] = nullptr;
  if constexpr (C::fits) {
    f->smooth_sweep_v[v] = smooth_sweep_launch<T, PP, false>;
    f->smooth_mult_v[v] = smooth_mult_launch<T, PP, false, 0>;
    f->smooth_mult_plain_v[v] = smooth_mult_plain_launch<T, PP, false, 0>;
    f->smooth_mult_batch_v[v] = smooth_mult_batch_launch<T, PP, false, 0>;
    f->smooth_add_v[v] = smooth_add_launch<T, PP>;
  } else {
    f->smooth_sweep_v[v] = nullptr;
    f->smooth_mult_v[v] = nullptr;
    f->smooth_mult_plain_v[v] = nullptr;
    f->smooth_mult_batch_v[v] = nullptr;
    f->smooth_add_v[v] = nullptr;
  }
}

template <typename T>
void register_fns(KernelFns<T>* f) {
  register_variant<T, 0>(f, 0);
  register_variant<T, 1>(f, 1);
  register_variant<T, 2>(f, 2);
  // default additive variant (the allocation-free entry point): shape 0
  f->smooth_add = f->smooth_add_v[0] ? f->smooth_add_v[0] : f->smooth_add_v[1];
  f->apply = apply_launch<T>;
  if constexpr (DIM == 3 && kApply3C<T>) f->apply_alt = apply_alt_launch<T>;
  else f->apply_alt = nullptr;
  f->prolong_add = prolong_launch<T>;
  f->restrict_ = restrict_launch<T>;
  f->prolong_batch = prolong_batch_launch<T>;
  f->restrict_batch = restrict_batch_launch<T>;
  f->zero_faces_batch = zero_faces_batch_launch<T>;
  f->transfer_cells = TransferCfg::CC;
  f->inverse_solve = kInvFits ? inverse_launch<T> : nullptr;
}

template <typename T>
cudaError_t set_smem_limits() {
  cudaError_t e;
  e = smooth_limits<T, 0>();
  if (e != cudaSuccess) return e;
  e = smooth_limits<T, 1>();
  if (e != cudaSuccess) return e;
  e = smooth_limits<T, 2>();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(apply_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ApplyCfg::smem<T>());
  if (e != cudaSuccess) return e;
  if constexpr (DIM == 3) {
    e = cudaFuncSetAttribute(apply3_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Apply3Cfg::smem<T>());
    if (e != cudaSuccess) return e;
    if constexpr (kApply3C<T>) {
      e = cudaFuncSetAttribute(apply3c_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)Apply3Cfg::smem_c<T>());
      if (e != cudaSuccess) return e;
    }
  }
  e = cudaFuncSetAttribute(prolong_add_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)TransferCfg::smem_prolong<T>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(prolong_add_batch_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)TransferCfg::smem_prolong<T>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(restrict_batch_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)TransferCfg::smem_restrict<T>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(restrict_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)TransferCfg::smem_restrict<T>());
}

template <typename T>
void fill_tab(const HostTables& h, DevTab<T>* d) {
  for (int i = 0; i < m * n; ++i) {
    d->Ap[i] = (T)h.Ap[i];
    d->Mp[i] = (T)h.Mp[i];
  }
  for (int i = 0; i < m * m; ++i) d->S[i] = (T)h.S[i];
  for (int o = 0; o <= H; ++o)
    for (int c = 0; c <= K; ++c) {
      const double mr = c < K ? h.Mp[o * n + n - 1 - c] : h.Mp[o * n + c];
      const double ar = c < K ? h.Ap[o * n + n - 1 - c] : h.Ap[o * n + c];
      d->MpE[o * KE + c] = (T)(c < K ? 0.5 * (h.Mp[o * n + c] + mr) : h.Mp[o * n + c]);
      d->ApE[o * KE + c] = (T)(c < K ? 0.5 * (h.Ap[o * n + c] + ar) : h.Ap[o * n + c]);
      if (o < H && c < K) {
        d->MpO[o * K + c] = (T)(0.5 * (h.Mp[o * n + c] - mr));
        d->ApO[o * K + c] = (T)(0.5 * (h.Ap[o * n + c] - ar));
      }
    }
  for (int c = 0; c <= H; ++c)
    for (int a = 0; a <= H; ++a) d->SE[c * HE + a] = (T)h.S[c * m + a];
  for (int c = 0; c < H; ++c)
    for (int a = 0; a < H; ++a) d->SO[c * HO + a] = (T)h.S[c * m + HE + a];
  for (int i = 0; i < K * n; ++i) {
    d->Kb[i] = (T)h.Kb[i];
    d->Mb[i] = (T)h.Mb[i];
  }
  for (int i = 0; i < n * nl; ++i) d->P1[i] = (T)h.P1[i];
  for (int i = 0; i < K * n; ++i) {
    d->Kb_lo[i] = (T)(h.Kb[i] - (double)(T)h.Kb[i]);
    d->Mb_lo[i] = (T)(h.Mb[i] - (double)(T)h.Mb[i]);
  }
}

cudaError_t df_limits() {
  if constexpr (DIM == 3)
    return cudaFuncSetAttribute(apply3_df_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Apply3Cfg::smem<double>());
  else
    return cudaFuncSetAttribute(apply2_df_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ApplyCfg::smem<double>());
}

cudaError_t upload(const HostTables& h) {
  if (h.k != K) return cudaErrorInvalidValue;
  DevTab<float> tf;
  DevTab<double> td;
  fill_tab(h, &tf);
  fill_tab(h, &td);
  AbsTab ta;
  for (int i = 0; i < K * n; ++i) {
    ta.Kb[i] = std::fabs(h.Kb[i]);
    ta.Mb[i] = std::fabs(h.Mb[i]);
  }
  cudaError_t e = cudaMemcpyToSymbol(c_tab<float>, &tf, sizeof(tf));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_tab<double>, &td, sizeof(td));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_abs, &ta, sizeof(ta));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(apply_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ApplyCfg::smem<double>());
  if (e != cudaSuccess) return e;
  if constexpr (DIM == 3) {
    e = cudaFuncSetAttribute(apply3_kernel<double, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Apply3Cfg::smem<double>());
    if (e != cudaSuccess) return e;
  }
  e = set_smem_limits<float>();
  if (e != cudaSuccess) return e;
  e = df_limits();
  if (e != cudaSuccess) return e;
  return set_smem_limits<double>();
}

}  // namespace

#define VPS_CAT2(a, b, c) a##b##_k##c
#define VPS_CAT(a, b, c) VPS_CAT2(a, b, c)
void VPS_CAT(register_kernels_d, VPS_DIM, VPS_K)(KernelSet* ks) {
  ks->present = true;
  ks->upload = upload;
  register_fns<float>(&ks->f);
  register_fns<double>(&ks->d);
  ks->apply_df = apply_df_launch;
  ks->apply_abs = apply_abs_launch;
}

}  // namespace vps
