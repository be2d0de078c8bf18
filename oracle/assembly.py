"""Global matrices and vectors by explicit assembly (oracle; test infrastructure only).

* ``stiffness``    -- A_l of Eq. 2.3/2.4 by a loop over all cells, scattering
                      each element matrix, then eliminating boundary rows and
                      columns (Dirichlet condition, Section 2).
* ``load_vector``  -- b_i = int f phi_i (Eq. 2.4), cell loop, (k+2)^d Gauss
                      points per cell.
* ``prolongation`` -- I^up of Section 2.1: the embedding V_{l-1} -> V_l written
                      as interpolation of every coarse basis function at the
                      fine support points.  Restriction is its transpose.
* ``interpolate``  -- nodal interpolant of a function (used by pins).

All vectors use the compact interior numbering of ``fe.Level``.
"""

import numpy as np
import scipy.sparse as sp

from . import fe


def stiffness(level):
    """Assembled stiffness matrix on interior nodes (CSR, FP64)."""
    d, k, h = level.d, level.k, level.h
    AK = fe.cell_stiffness(d, k, h)
    cells = level.cell_node_indices()  # (ncells, nloc) full-grid indices
    g2c = level.global_to_compact()
    nloc = cells.shape[1]
    rows = np.repeat(cells, nloc, axis=1).ravel()
    cols = np.tile(cells, (1, nloc)).ravel()
    vals = np.tile(AK.ravel(), cells.shape[0])
    r, c = g2c[rows], g2c[cols]
    keep = (r >= 0) & (c >= 0)
    A = sp.coo_matrix((vals[keep], (r[keep], c[keep])), shape=(level.N, level.N))
    return A.tocsr()


def _cell_quadrature(level, q):
    """Physical points, weights and basis values for every cell.

    Returns (X, W, E, cells): X (ncells, q^d, d) points, W (q^d,) weights
    including the volume element h^d, E (nloc, q^d) basis values on the
    reference cell, cells (ncells, nloc) full-grid node indices.
    """
    d, k, h = level.d, level.k, level.h
    xq, wq = fe.gauss_points(q)
    V = fe.lagrange_values(level.z, xq)
    E = fe.tensor_basis_at([V] * d, d, k + 1, q)
    Q = fe.multi_indices(q, d)
    W = np.ones(q ** d)
    for t in range(d):
        W *= wq[Q[:, t]]
    W = W * h ** d
    C = fe.multi_indices(level.ncell, d)
    X = (C[:, None, :] + xq[Q][None, :, :]) * h
    return X, W, E, level.cell_node_indices()


def load_vector(level, f):
    """b_i = int_Omega f phi_i dx on interior nodes (Eq. 2.4).

    ``f`` maps an (npts, d) array of points to npts values.
    """
    X, W, E, cells = _cell_quadrature(level, level.k + 2)
    nc, nq, d = X.shape
    fv = np.asarray(f(X.reshape(-1, d)), dtype=np.float64).reshape(nc, nq)
    contrib = (fv * W) @ E.T  # (ncells, nloc)
    g2c = level.global_to_compact()
    r = g2c[cells.ravel()]
    keep = r >= 0
    b = np.zeros(level.N)
    np.add.at(b, r[keep], contrib.ravel()[keep])
    return b


def interpolate(level, u):
    """Nodal values of ``u`` at the interior support points (compact order)."""
    x1 = level.node_coords_1d()[1:-1]
    Q = fe.multi_indices(level.ni, level.d)
    return np.asarray(u(x1[Q]), dtype=np.float64)


def prolongation(fine):
    """I^up: compact coarse interior vector -> compact fine interior vector.

    Entry (i, j) is the coarse basis function of coarse node j evaluated at
    fine support point i (Section 2.1: the spaces are nested and the
    embedding is polynomial interpolation).  A fine point on a coarse cell
    face is evaluated in one adjacent coarse cell; the coarse basis is
    continuous, so the choice does not change the value.
    """
    if fine.l < 2:
        raise ValueError("prolongation needs a fine level >= 2")
    d, k = fine.d, fine.k
    coarse = fe.Level(d, k, fine.l - 1)
    H = coarse.h
    xf = fine.node_coords_1d()[1:-1]                      # fine interior coords
    cc = np.minimum(np.floor(xf / H).astype(np.int64), coarse.ncell - 1)
    xr = (xf - cc * H) / H                                # reference coordinate
    V = fe.lagrange_values(coarse.z, xr)                  # (k+1, ni_f)
    g2c = coarse.global_to_compact()
    Qf = fe.multi_indices(fine.ni, d)                     # fine interior multi-index
    Lc = fe.multi_indices(k + 1, d)                       # coarse local nodes
    rows, cols, vals = [], [], []
    for a in range(len(Lc)):
        val = np.ones(len(Qf))
        gidx = np.zeros(len(Qf), dtype=np.int64)
        for t in range(d):
            pos = Qf[:, t]
            val *= V[Lc[a, t], pos]
            gidx += (k * cc[pos] + Lc[a, t]) * coarse.n1 ** t
        cj = g2c[gidx]
        keep = (cj >= 0) & (val != 0.0)
        rows.append(np.nonzero(keep)[0])
        cols.append(cj[keep])
        vals.append(val[keep])
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(fine.N, coarse.N))
    return P.tocsr()
