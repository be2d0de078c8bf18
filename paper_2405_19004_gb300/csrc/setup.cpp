// Host set-up of the 1D finite element tables (FP64, once per degree).
//
// Section 2: Q_k Lagrange basis on k+1 Gauss-Lobatto support points per
// direction.  Section 2.4: the patch operator is a Kronecker sum of 1D
// stiffness and mass matrices of the two-cell patch (Eq. 2.11/2.12), and the
// local inverse is applied by fast diagonalisation with the generalised
// eigenpairs A^d S^d = M^d S^d Lambda^d (Eq. 2.13-2.15), here normalised by
// S^T M S = I.  The eigenproblem is reduced to a symmetric one by a Cholesky
// factor of M and solved with cyclic Jacobi rotations (m <= 13).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "vps_internal.h"

namespace vps {

namespace {

// Legendre P_n(x) and P_n'(x) by the three-term recurrences.
void legendre(int n, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int j = 1; j < n; ++j) {
    double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
    double d2 = d0 + (2.0 * j + 1.0) * p1;  // P'_{j+1} = P'_{j-1} + (2j+1) P_j
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *p = p1; *dp = d1;
}

// Gauss-Lobatto points on [0,1]: 0, 1 and the roots of P_k' (Newton; the
// second derivative from Legendre's equation).
void gll_points(int k, double* z) {
  z[0] = 0.0; z[k] = 1.0;
  for (int j = 1; j < k; ++j) {
    double x = -std::cos(M_PI * j / k);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(k, x, &p, &dp);
      double d2 = (2.0 * x * dp - k * (k + 1.0) * p) / (1.0 - x * x);
      double dx = dp / d2;
      x -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    z[j] = 0.5 * (x + 1.0);
  }
}

void lagrange_deriv(int k, const double* z, double x, double* der) {
  for (int i = 0; i <= k; ++i) {
    double s = 0.0;
    for (int mm = 0; mm <= k; ++mm) {
      if (mm == i) continue;
      double t = 1.0 / (z[i] - z[mm]);
      for (int j = 0; j <= k; ++j)
        if (j != i && j != mm) t *= (x - z[j]) / (z[i] - z[j]);
      s += t;
    }
    der[i] = s;
  }
}

// Cholesky factor L (lower) of an SPD m x m matrix, in place in a copy.
bool cholesky(int m, const double* A, double* L) {
  std::memset(L, 0, sizeof(double) * m * m);
  for (int j = 0; j < m; ++j) {
    double s = A[j * m + j];
    for (int p = 0; p < j; ++p) s -= L[j * m + p] * L[j * m + p];
    if (!(s > 0.0)) return false;
    L[j * m + j] = std::sqrt(s);
    for (int i = j + 1; i < m; ++i) {
      double t = A[i * m + j];
      for (int p = 0; p < j; ++p) t -= L[i * m + p] * L[j * m + p];
      L[i * m + j] = t / L[j * m + j];
    }
  }
  return true;
}

// Cyclic Jacobi eigen-decomposition of a symmetric matrix C (destroyed):
// C = Q diag(w) Q^T, Q row-major with eigenvectors in columns.
void jacobi_eigen(int m, double* C, double* Q, double* w) {
  for (int i = 0; i < m * m; ++i) Q[i] = 0.0;
  for (int i = 0; i < m; ++i) Q[i * m + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) (i == j ? diag : off) += C[i * m + j] * C[i * m + j];
    if (off <= 1e-32 * diag) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        double apq = C[p * m + q];
        if (std::fabs(apq) < 1e-300) continue;
        double theta = (C[q * m + q] - C[p * m + p]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < m; ++r) {  // columns p, q of C
          double crp = C[r * m + p], crq = C[r * m + q];
          C[r * m + p] = c * crp - s * crq;
          C[r * m + q] = s * crp + c * crq;
        }
        for (int r = 0; r < m; ++r) {  // rows p, q of C
          double cpr = C[p * m + r], cqr = C[q * m + r];
          C[p * m + r] = c * cpr - s * cqr;
          C[q * m + r] = s * cpr + c * cqr;
        }
        for (int r = 0; r < m; ++r) {
          double qrp = Q[r * m + p], qrq = Q[r * m + q];
          Q[r * m + p] = c * qrp - s * qrq;
          Q[r * m + q] = s * qrp + c * qrq;
        }
      }
  }
  for (int i = 0; i < m; ++i) w[i] = C[i * m + i];
}

// Generalised symmetric eigenproblem A S = M S diag(w), S^T M S = I
// (M SPD; m <= 13): Cholesky M = L L^T, C = L^-1 A L^-T, Jacobi on C,
// S = L^-T Q.  Returns false if M is not positive definite.
bool generalised_eigen(int m, const double* A, const double* M, double* S, double* w) {
  double L[13 * 13], C[13 * 13], Q[13 * 13], tmp[13 * 13];
  if (!cholesky(m, M, L)) return false;
  // tmp = L^-1 A  (forward substitution per column), C = tmp L^-T
  for (int col = 0; col < m; ++col)
    for (int i = 0; i < m; ++i) {
      double s = A[i * m + col];
      for (int p = 0; p < i; ++p) s -= L[i * m + p] * tmp[p * m + col];
      tmp[i * m + col] = s / L[i * m + i];
    }
  for (int row = 0; row < m; ++row)
    for (int i = 0; i < m; ++i) {
      double s = tmp[row * m + i];
      for (int p = 0; p < i; ++p) s -= L[i * m + p] * C[row * m + p];
      C[row * m + i] = s / L[i * m + i];
    }
  for (int i = 0; i < m; ++i)  // symmetrise against rounding
    for (int j = i + 1; j < m; ++j) C[i * m + j] = C[j * m + i] = 0.5 * (C[i * m + j] + C[j * m + i]);
  jacobi_eigen(m, C, Q, w);
  // S = L^-T Q: back substitution L^T S = Q per column
  for (int col = 0; col < m; ++col)
    for (int i = m - 1; i >= 0; --i) {
      double s = Q[i * m + col];
      for (int p = i + 1; p < m; ++p) s -= L[p * m + i] * S[p * m + col];
      S[i * m + col] = s / L[i * m + i];
    }
  return true;
}

}  // namespace

void gauss_rule(int q, double* x, double* w) {
  for (int i = 0; i < q; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (q + 0.5));
    double p = 0.0, dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      legendre(q, t, &p, &dp);
      double dt = p / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    legendre(q, t, &p, &dp);
    x[q - 1 - i] = 0.5 * (t + 1.0);
    w[q - 1 - i] = 1.0 / ((1.0 - t * t) * dp * dp);  // 2/((1-t^2) P'^2) halved for [0,1]
  }
}

void lagrange_eval(int k, const double* z, double x, double* val) {
  for (int i = 0; i <= k; ++i) {
    double t = 1.0;
    for (int j = 0; j <= k; ++j)
      if (j != i) t *= (x - z[j]) / (z[i] - z[j]);
    val[i] = t;
  }
}

bool build_tables(int k, HostTables* T, char* err, size_t errlen) {
  if (k < 1 || k > kMaxK) {
    std::snprintf(err, errlen, "degree %d outside 1..%d", k, kMaxK);
    return false;
  }
  std::memset(T, 0, sizeof(*T));
  const int n = 2 * k + 1, m = 2 * k - 1, nl = k + 1;
  T->k = k; T->n = n; T->m = m;
  gll_points(k, T->z);

  // Reference element matrices on [0,1], (k+1)-point Gauss rule (exact).
  double xq[16], wq[16], val[kMaxK + 1], der[kMaxK + 1];
  gauss_rule(k + 1, xq, wq);
  for (int q = 0; q <= k; ++q) {
    lagrange_eval(k, T->z, xq[q], val);
    lagrange_deriv(k, T->z, xq[q], der);
    for (int i = 0; i < nl; ++i)
      for (int j = 0; j < nl; ++j) {
        T->Khat[i * nl + j] += wq[q] * der[i] * der[j];
        T->Mhat[i * nl + j] += wq[q] * val[i] * val[j];
      }
  }

  // Two-cell patch closure matrices (nodes 0..2k), interior rows 1..2k-1.
  double Af[(2 * kMaxK + 1) * (2 * kMaxK + 1)] = {0}, Mf[(2 * kMaxK + 1) * (2 * kMaxK + 1)] = {0};
  for (int c = 0; c < 2; ++c)
    for (int i = 0; i < nl; ++i)
      for (int j = 0; j < nl; ++j) {
        Af[(c * k + i) * n + c * k + j] += T->Khat[i * nl + j];
        Mf[(c * k + i) * n + c * k + j] += T->Mhat[i * nl + j];
      }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) {
      T->Ap[i * n + j] = Af[(i + 1) * n + j];
      T->Mp[i * n + j] = Mf[(i + 1) * n + j];
    }

  // Generalised eigenproblem of the interior blocks.  The two-cell patch is
  // symmetric about its centre node k, so A_I and M_I commute with the
  // reversal J of the m interior nodes: every eigenvector can be taken even
  // (J s = s) or odd (J s = -s).  The problem is solved separately on the
  // even subspace (basis (e_i + e_{m-1-i})/sqrt2, i < h, and e_h; h = k-1)
  // and the odd one ((e_i - e_{m-1-i})/sqrt2), so that the columns of S have
  // exact parity: the h+1 even eigenvectors first, then the h odd ones.  The
  // kernels use this to apply S and S^T with half the multiply-adds.
  double AI[13 * 13], MI[13 * 13];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      AI[i * m + j] = T->Ap[i * n + j + 1];
      MI[i * m + j] = T->Mp[i * n + j + 1];
    }
  const int h = k - 1, ne = h + 1, no = h;
  const double r2 = std::sqrt(0.5);
  // basis vectors of the even (j < ne) and odd (j >= ne) subspaces, columns of B
  double B[13 * 13] = {0};
  for (int j = 0; j < ne; ++j) {
    if (j < h) {
      B[j * m + j] = r2;
      B[(m - 1 - j) * m + j] = r2;
    } else {
      B[h * m + j] = 1.0;
    }
  }
  for (int j = 0; j < no; ++j) {
    B[j * m + ne + j] = r2;
    B[(m - 1 - j) * m + ne + j] = -r2;
  }
  for (int part = 0; part < 2; ++part) {
    const int off = part == 0 ? 0 : ne, sz = part == 0 ? ne : no;
    if (sz == 0) continue;
    double Ab[13 * 13], Mb[13 * 13], Sb[13 * 13], lb[13];
    for (int a = 0; a < sz; ++a)
      for (int b = 0; b < sz; ++b) {
        double sa = 0.0, sm = 0.0;
        for (int p = 0; p < m; ++p)
          for (int q = 0; q < m; ++q) {
            const double w = B[p * m + off + a] * B[q * m + off + b];
            sa += w * AI[p * m + q];
            sm += w * MI[p * m + q];
          }
        Ab[a * sz + b] = sa;
        Mb[a * sz + b] = sm;
      }
    if (!generalised_eigen(sz, Ab, Mb, Sb, lb)) {
      std::snprintf(err, errlen, "mass matrix not positive definite (k=%d)", k);
      return false;
    }
    for (int a = 0; a < sz; ++a) T->lam[off + a] = lb[a];
    // S column off+a = B_part Sb column a
    for (int i = 0; i < m; ++i)
      for (int a = 0; a < sz; ++a) {
        double v = 0.0;
        for (int b = 0; b < sz; ++b) v += B[i * m + off + b] * Sb[b * sz + a];
        T->S[i * m + off + a] = v;
      }
  }
  // exact parity (the products above give it up to rounding only)
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < h; ++i) T->S[(m - 1 - i) * m + j] = (j < ne ? 1.0 : -1.0) * T->S[i * m + j];
  for (int j = ne; j < m; ++j) T->S[h * m + j] = 0.0;
  // self-check: S^T M S = I and S^T A S = diag(lam)
  double worst = 0.0, scale = 0.0;
  for (int i = 0; i < m; ++i) scale = std::fmax(scale, std::fabs(T->lam[i]));
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      double sm = 0.0, sa = 0.0;
      for (int p = 0; p < m; ++p)
        for (int q2 = 0; q2 < m; ++q2) {
          sm += T->S[p * m + i] * MI[p * m + q2] * T->S[q2 * m + j];
          sa += T->S[p * m + i] * AI[p * m + q2] * T->S[q2 * m + j];
        }
      worst = std::fmax(worst, std::fabs(sm - (i == j)));
      worst = std::fmax(worst, std::fabs(sa - (i == j ? T->lam[i] : 0.0)) / scale);
    }
  double lmin = T->lam[0];
  for (int i = 1; i < m; ++i) lmin = std::fmin(lmin, T->lam[i]);
  if (!(worst < 1e-10) || !(lmin > 0)) {
    std::snprintf(err, errlen, "fast-diagonalisation self-check failed (k=%d, err %.3g)", k, worst);
    return false;
  }

  // Bands of the global 1D matrices (reference cell size 1).
  const int bw = 2 * k + 1;
  for (int q = 0; q < k; ++q) {
    if (q == 0) {
      for (int j = 0; j <= k; ++j) {
        T->Kb[j] += T->Khat[k * nl + j];
        T->Mb[j] += T->Mhat[k * nl + j];
        T->Kb[k + j] += T->Khat[0 * nl + j];
        T->Mb[k + j] += T->Mhat[0 * nl + j];
      }
    } else {
      for (int j = k - q; j <= 2 * k - q; ++j) {
        T->Kb[q * bw + j] = T->Khat[q * nl + j - (k - q)];
        T->Mb[q * bw + j] = T->Mhat[q * nl + j - (k - q)];
      }
    }
  }

  // 1D prolongation on one coarse cell: fine node s = fc*k + j at (fc + z_j)/2.
  for (int s = 0; s <= 2 * k; ++s) {
    int fc = s < k ? 0 : 1;
    if (s == 2 * k) fc = 1;
    int j = s - fc * k;
    double xi = 0.5 * (fc + T->z[j]);
    lagrange_eval(k, T->z, xi, val);
    for (int i = 0; i <= k; ++i) T->P1[s * nl + i] = val[i];
  }
  return true;
}

bool build_global_fd(int k, int level, std::vector<double>* S, std::vector<double>* lam, char* err,
                     size_t errlen) {
  const int ncell = 1 << level, n1 = k * ncell + 1, ni = n1 - 2, nl = k + 1;
  if (ni < 1 || ni > kMaxGlobalFd) {
    std::snprintf(err, errlen, "global fast diagonalisation needs 1..%d interior nodes (got %d)",
                  kMaxGlobalFd, ni);
    return false;
  }
  HostTables t;
  if (!build_tables(k, &t, err, errlen)) return false;
  // global 1D matrices of the level in reference units (cell size 1), interior block
  std::vector<double> Kg((size_t)n1 * n1, 0.0), Mg((size_t)n1 * n1, 0.0);
  for (int c = 0; c < ncell; ++c)
    for (int i = 0; i < nl; ++i)
      for (int j = 0; j < nl; ++j) {
        Kg[(size_t)(c * k + i) * n1 + c * k + j] += t.Khat[i * nl + j];
        Mg[(size_t)(c * k + i) * n1 + c * k + j] += t.Mhat[i * nl + j];
      }
  std::vector<double> A((size_t)ni * ni), M((size_t)ni * ni), L((size_t)ni * ni),
      tmp((size_t)ni * ni), C((size_t)ni * ni), Q((size_t)ni * ni);
  for (int i = 0; i < ni; ++i)
    for (int j = 0; j < ni; ++j) {
      A[(size_t)i * ni + j] = Kg[(size_t)(i + 1) * n1 + j + 1];
      M[(size_t)i * ni + j] = Mg[(size_t)(i + 1) * n1 + j + 1];
    }
  if (!cholesky(ni, M.data(), L.data())) {
    std::snprintf(err, errlen, "global mass matrix not positive definite");
    return false;
  }
  for (int col = 0; col < ni; ++col)
    for (int i = 0; i < ni; ++i) {
      double sacc = A[(size_t)i * ni + col];
      for (int q = 0; q < i; ++q) sacc -= L[(size_t)i * ni + q] * tmp[(size_t)q * ni + col];
      tmp[(size_t)i * ni + col] = sacc / L[(size_t)i * ni + i];
    }
  for (int row = 0; row < ni; ++row)
    for (int i = 0; i < ni; ++i) {
      double sacc = tmp[(size_t)row * ni + i];
      for (int q = 0; q < i; ++q) sacc -= L[(size_t)i * ni + q] * C[(size_t)row * ni + q];
      C[(size_t)row * ni + i] = sacc / L[(size_t)i * ni + i];
    }
  for (int i = 0; i < ni; ++i)
    for (int j = i + 1; j < ni; ++j)
      C[(size_t)i * ni + j] = C[(size_t)j * ni + i] =
          0.5 * (C[(size_t)i * ni + j] + C[(size_t)j * ni + i]);
  lam->assign(ni, 0.0);
  S->assign((size_t)ni * ni, 0.0);
  jacobi_eigen(ni, C.data(), Q.data(), lam->data());
  for (int col = 0; col < ni; ++col)
    for (int i = ni - 1; i >= 0; --i) {
      double sacc = Q[(size_t)i * ni + col];
      for (int q = i + 1; q < ni; ++q) sacc -= L[(size_t)q * ni + i] * (*S)[(size_t)q * ni + col];
      (*S)[(size_t)i * ni + col] = sacc / L[(size_t)i * ni + i];
    }
  // self-check S^T M S = I
  double worst = 0.0;
  for (int i = 0; i < ni; ++i)
    for (int j = 0; j < ni; ++j) {
      double v = 0.0;
      for (int a = 0; a < ni; ++a) {
        double ma = 0.0;
        for (int b2 = 0; b2 < ni; ++b2) ma += M[(size_t)a * ni + b2] * (*S)[(size_t)b2 * ni + j];
        v += (*S)[(size_t)a * ni + i] * ma;
      }
      worst = std::fmax(worst, std::fabs(v - (i == j)));
    }
  if (!(worst < 1e-9) || !((*lam)[0] > 0.0)) {
    std::snprintf(err, errlen, "global eigen-decomposition self-check failed (%.3g)", worst);
    return false;
  }
  return true;
}

double level_elements(int dim, int k, int level) {
  if (level < 0 || level > 30 || k < 1 || k > kMaxK || (dim != 2 && dim != 3)) return HUGE_VAL;
  const double n1 = (double)k * std::ldexp(1.0, level) + 1.0;
  const double px = std::ceil(n1 / 8.0) * 8.0;
  return dim == 2 ? px * n1 : px * n1 * n1;
}

LevelGeom make_geom(int dim, int k, int level) {
  LevelGeom g;
  g.dim = dim; g.k = k; g.level = level;
  // every caller checks level_elements (or the saturated total below)
  // before it uses a level: no product here may overflow
  if (!(level_elements(dim, k, level) <= kMaxLevelElements)) {
    g.total = INT64_MAX;
    return g;
  }
  g.ncell = 1 << level;
  g.n1 = k * g.ncell + 1;
  g.px = (g.n1 + 7) / 8 * 8;
  g.pz = g.px * g.n1;
  g.total = dim == 2 ? g.pz : g.pz * g.n1;
  g.h = 1.0 / g.ncell;
  return g;
}

ColourGeom make_colour(const LevelGeom& g, int colour) {
  ColourGeom c;
  c.npatch = 1;
  for (int t = 0; t < 3; ++t) {
    if (t >= g.dim) { c.cnt[t] = 1; c.par[t] = 0; continue; }
    c.par[t] = (colour >> t) & 1;
    int half = g.ncell / 2;  // vertices 1..ncell-1: odd ones (parity 0) and even ones (parity 1)
    c.cnt[t] = c.par[t] == 0 ? half : half - 1;
    c.npatch *= c.cnt[t];
  }
  return c;
}

int64_t& launch_counter() {
  static thread_local int64_t count = 0;
  return count;
}

static KernelSet g_registry[2][kMaxK];

KernelSet* kernel_registry(int dim, int k) {
  if (dim < 2 || dim > 3 || k < 1 || k > kMaxK) return nullptr;
  return &g_registry[dim - 2][k - 1];
}

}  // namespace vps
