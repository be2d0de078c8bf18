"""Q_k finite elements on Cartesian cells (oracle; test infrastructure only).

Section 2 of the paper: the Q_k space uses k+1 Gauss-Lobatto support points
on the reference interval, tensorised to (k+1)^d points per cell, with the
Lagrange basis on them.  The stiffness entries are a_ij = int grad phi_j .
grad phi_i (Eq. 2.4, the matrix definition); on a Cartesian cell the
Jacobian is diagonal and constant (Section 2.3, Eq. 2.9), so an element
integral is a reference integral times powers of the cell size h.

All quantities are FP64.  Quadrature: Gauss-Legendre with k+1 points per
direction for stiffness and mass (exact: integrands have degree <= 2k), k+2
points for load vectors and L2 errors (the paper names no rule; this reading
is listed in the design notes).
"""

import numpy as np
from numpy.polynomial import legendre as npleg


def gll_nodes(k):
    """k+1 Gauss-Lobatto-Legendre points on [0, 1], ascending.

    The interior points are the roots of P_k' (derivative of the Legendre
    polynomial of degree k); the end points are 0 and 1.
    """
    if k < 1:
        raise ValueError("degree must be >= 1")
    if k == 1:
        return np.array([0.0, 1.0])
    c = np.zeros(k + 1)
    c[k] = 1.0
    dc = npleg.legder(c)
    r = np.sort(npleg.legroots(dc).real)
    ddc = npleg.legder(dc)
    for _ in range(4):  # Newton polish of the companion-matrix roots
        r = r - npleg.legval(r, dc) / npleg.legval(r, ddc)
    x = np.concatenate([[-1.0], r, [1.0]])
    return 0.5 * (x + 1.0)


def gauss_points(q):
    """q-point Gauss-Legendre rule on [0, 1]: (points, weights)."""
    x, w = npleg.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange_values(nodes, x):
    """V[i, q] = l_i(x_q) for the Lagrange basis on ``nodes``."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    V = np.ones((n, len(x)))
    for i in range(n):
        for j in range(n):
            if j != i:
                V[i] *= (x - nodes[j]) / (nodes[i] - nodes[j])
    return V


def lagrange_derivatives(nodes, x):
    """D[i, q] = l_i'(x_q): product rule over the factors of l_i."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    D = np.zeros((n, len(x)))
    for i in range(n):
        for m in range(n):
            if m == i:
                continue
            term = np.full(len(x), 1.0 / (nodes[i] - nodes[m]))
            for j in range(n):
                if j != i and j != m:
                    term = term * (x - nodes[j]) / (nodes[i] - nodes[j])
            D[i] += term
    return D


def reference_matrices_1d(k):
    """Stiffness K^ and mass M^ of Q_k on the unit interval [0, 1].

    K^_ij = int_0^1 l_i' l_j' dx,  M^_ij = int_0^1 l_i l_j dx, evaluated with
    the (k+1)-point Gauss rule (exact for these polynomial integrands).
    """
    z = gll_nodes(k)
    xq, wq = gauss_points(k + 1)
    V = lagrange_values(z, xq)
    D = lagrange_derivatives(z, xq)
    K = (D * wq) @ D.T
    M = (V * wq) @ V.T
    return K, M


def multi_indices(n, d):
    """Lexicographic multi-indices of an n^d tensor grid, dimension 0 fastest.

    Row a of the result is (i_0, ..., i_{d-1}) with a = sum_t i_t n^t.
    """
    a = np.arange(n ** d)
    return np.stack([(a // n ** t) % n for t in range(d)], axis=1)


def tensor_basis_at(mats, d, n, nq):
    """E[a, q] = prod_t mats[t][a_t, q_t] for local basis a and point q.

    This is the definition of the tensor-product basis evaluated at tensor
    points: each d-variate basis function is a product of 1D functions.
    """
    A = multi_indices(n, d)
    Q = multi_indices(nq, d)
    E = np.ones((n ** d, nq ** d))
    for t in range(d):
        E *= mats[t][A[:, t][:, None], Q[:, t][None, :]]
    return E


def cell_stiffness(d, k, h):
    """Element stiffness matrix of Q_k on a Cartesian cell of edge h.

    A^K_ab = sum_q grad phi_a(x_q) . grad phi_b(x_q) w_q  (Eq. 2.4 on one
    cell, in the quadrature form of Eq. 2.9).  Physical gradients are reference
    gradients / h and the volume element is h^d, giving the factor h^(d-2).
    """
    z = gll_nodes(k)
    xq, wq = gauss_points(k + 1)
    V = lagrange_values(z, xq)
    D = lagrange_derivatives(z, xq)
    n, nq = k + 1, k + 1
    W = np.ones(nq ** d)
    Q = multi_indices(nq, d)
    for t in range(d):
        W *= wq[Q[:, t]]
    AK = np.zeros((n ** d, n ** d))
    for t in range(d):
        mats = [D if s == t else V for s in range(d)]
        G = tensor_basis_at(mats, d, n, nq)  # d/dx_t phi_a at points
        AK += (G * W) @ G.T
    return AK * h ** (d - 2)


def cell_mass(d, k, h):
    """Element mass matrix of Q_k on a Cartesian cell of edge h (used by pins)."""
    z = gll_nodes(k)
    xq, wq = gauss_points(k + 1)
    V = lagrange_values(z, xq)
    n, nq = k + 1, k + 1
    W = np.ones(nq ** d)
    Q = multi_indices(nq, d)
    for t in range(d):
        W *= wq[Q[:, t]]
    E = tensor_basis_at([V] * d, d, n, nq)
    return (E * W) @ E.T * h ** d


class Level:
    """Uniform mesh of (0,1)^d with 2^l cells per direction and Q_k nodes.

    Section 2: mesh M_l is obtained from the single cell M_0 by l uniform
    refinements.  Nodes are numbered lexicographically over the whole grid
    with dimension 0 fastest (Section 3.1.2, the paper's DoF layout); there
    are n1 = k 2^l + 1 nodes per direction including the boundary.  The
    "compact" numbering lists interior nodes only, also lexicographically
    with dimension 0 fastest.
    """

    def __init__(self, d, k, l):
        if d not in (2, 3) or k < 1 or l < 1:
            raise ValueError("need d in {2,3}, k >= 1, l >= 1")
        self.d, self.k, self.l = d, k, l
        self.ncell = 2 ** l
        self.h = 1.0 / self.ncell
        self.n1 = k * self.ncell + 1
        self.ni = self.n1 - 2
        self.N = self.ni ** d
        self.z = gll_nodes(k)

    def node_coords_1d(self):
        """Coordinate of every node along one direction (n1 values)."""
        g = np.arange(self.n1)
        c = np.minimum(g // self.k, self.ncell - 1)
        i = g - self.k * c
        return (c + self.z[i]) * self.h

    def global_to_compact(self):
        """Map full-grid node index -> compact interior index (-1: boundary)."""
        G = multi_indices(self.n1, self.d)
        inside = np.all((G >= 1) & (G <= self.n1 - 2), axis=1)
        out = np.full(self.n1 ** self.d, -1, dtype=np.int64)
        idx = np.zeros(len(G), dtype=np.int64)
        for t in range(self.d):
            idx += (G[:, t] - 1) * self.ni ** t
        out[inside] = idx[inside]
        return out

    def cell_node_indices(self):
        """Full-grid indices of the (k+1)^d nodes of every cell.

        Returns (ncell^d, (k+1)^d); cells lexicographic (dim 0 fastest).
        """
        C = multi_indices(self.ncell, self.d)
        Lc = multi_indices(self.k + 1, self.d)
        idx = np.zeros((len(C), len(Lc)), dtype=np.int64)
        for t in range(self.d):
            idx += (self.k * C[:, t][:, None] + Lc[:, t][None, :]) * self.n1 ** t
        return idx
