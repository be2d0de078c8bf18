"""Vertex-patch Schwarz smoothers (oracle; test infrastructure only).

Section 2.2.  Every interior vertex p_j of the mesh defines a vertex patch:
the 2^d cells sharing p_j.  V_j is spanned by the basis functions whose
support points lie strictly inside the patch, (2k-1)^d of them; R_j selects
their coefficients and A_j = R_j A R_j^T (the definition of Eq. 2.4
restricted to V_j).  One subspace correction is

    r <- b - A x,   y <- x + R_j^T A_j^{-1} R_j r          (Eq. 2.5, 2.6)

and the multiplicative smoother applies s_J o ... o s_1 (Eq. 2.7).

Colouring (Section 2.2, Figure "patch coloring"; Algorithm 3): patches whose
vertices are shifted by one cell in a coordinate direction get a different
colour; the reading used here is colour(v) = sum_t ((v_t - 1) mod 2) 2^t for
vertex indices v_t in 1..2^l-1, giving 2^d colours, visited in increasing
order.  Same-colour patches do not overlap, so the parallel update of
Algorithm 3 equals the sequential one (pinned in the tests).

The additive smoother x <- x + omega sum_j R_j^T A_j^{-1} R_j (b - A x) has no
counterpart in the paper; it is the additive Schwarz form of the same
subspace corrections.

Local solves use dense LU of A_j (scipy), the "obviously correct" solver;
the fast-diagonalisation inverse of Eq. 2.13/2.14 is not used here.
"""

import numpy as np
import scipy.linalg as sla

from . import fe


def vertices(level):
    """Interior vertices v (values 1..2^l-1 per direction), lexicographic."""
    nv = level.ncell - 1
    return fe.multi_indices(nv, level.d) + 1


def colour_of(v):
    """Colour of a vertex (array (..., d)) -> int in 0..2^d-1."""
    v = np.asarray(v)
    d = v.shape[-1]
    return sum(((v[..., t] - 1) % 2) * (1 << t) for t in range(d))


def patch_interior(level, v):
    """Compact indices of the (2k-1)^d interior DoFs of the patch at vertex v.

    Along direction t the interior nodes are k(v_t-1)+1 .. k(v_t+1)-1 (full
    grid numbering); ordered lexicographically with dimension 0 fastest.
    """
    k, d = level.k, level.d
    m = 2 * k - 1
    L = fe.multi_indices(m, d)
    idx = np.zeros(len(L), dtype=np.int64)
    for t in range(d):
        g = k * (v[t] - 1) + 1 + L[:, t]
        idx += (g - 1) * level.ni ** t
    return idx


def patch_closure_full(level, v):
    """Full-grid indices of the (2k+1)^d closure nodes of the patch at v."""
    k, d = level.k, level.d
    n = 2 * k + 1
    L = fe.multi_indices(n, d)
    idx = np.zeros(len(L), dtype=np.int64)
    for t in range(d):
        idx += (k * (v[t] - 1) + L[:, t]) * level.n1 ** t
    return idx


class PatchSolver:
    """Dense LU of the patch matrix A_j = A[I_j, I_j].

    Constant coefficients on a uniform mesh make every A_j the same matrix;
    the constructor asserts that for every patch and factors one copy.
    """

    def __init__(self, level, A):
        self.level = level
        self.V = vertices(level)
        self.I = np.stack([patch_interior(level, v) for v in self.V])
        self.colour = colour_of(self.V)
        Aj0 = A[self.I[0]][:, self.I[0]].toarray()
        for I in self.I[1:]:
            Aj = A[I][:, I].toarray()
            if not np.allclose(Aj, Aj0, rtol=1e-12, atol=1e-12 * abs(Aj0).max()):
                raise AssertionError("patch matrices differ")
        self.Aj = Aj0
        self.lu = sla.lu_factor(Aj0)

    def solve(self, R):
        """A_j^{-1} R for R of shape (m^d,) or (m^d, nrhs)."""
        return sla.lu_solve(self.lu, R)


def multiplicative_sequential(A, ps, x, b, colours=None):
    """One multiplicative smoothing step, strictly sequential (Eq. 2.7).

    Colours in the given order (default 0..2^d-1); inside a colour, patches
    in lexicographic vertex order.  Every correction recomputes the residual
    rows R_j (b - A x) from the current x.
    """
    x = np.array(x, dtype=np.float64, copy=True)
    d = ps.level.d
    if colours is None:
        colours = range(2 ** d)
    for c in colours:
        for j in np.nonzero(ps.colour == c)[0]:
            I = ps.I[j]
            r = b[I] - A[I] @ x
            x[I] += ps.solve(r)
    return x


def multiplicative(A, ps, x, b, colours=None):
    """One colourised multiplicative step (Algorithm 3).

    For each colour: one residual r = b - A x for the whole colour, then all
    patches of the colour are corrected from that residual.
    """
    x = np.array(x, dtype=np.float64, copy=True)
    d = ps.level.d
    if colours is None:
        colours = range(2 ** d)
    for c in colours:
        js = np.nonzero(ps.colour == c)[0]
        r = b - A @ x
        Ic = ps.I[js]                                     # (npatch_c, m^d)
        U = ps.solve(r[Ic].T).T
        x[Ic] += U
    return x


def additive(A, ps, x, b, omega):
    """One additive step x <- x + omega sum_j R_j^T A_j^{-1} R_j (b - A x)."""
    x = np.array(x, dtype=np.float64, copy=True)
    r = b - A @ x
    U = ps.solve(r[ps.I].T).T
    delta = np.zeros_like(x)
    np.add.at(delta, ps.I, U)
    return x + omega * delta


def colour_counts(level):
    """Number of patches of each colour."""
    c = colour_of(vertices(level))
    return np.bincount(c, minlength=2 ** level.d)
