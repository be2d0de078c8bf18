"""Single-patch and single-row evaluations of the same definitions (oracle; test infrastructure only).

At the sizes the benchmarks run (millions of DoFs) the global matrix of
``assembly.stiffness`` does not fit in host memory.  The rows of A at a node
only involve the cells that contain the node, so they are obtained here by
the same element loop restricted to those cells (Eq. 2.4 summed over the
cells of the support).  This gives

* ``patch_update``   -- R_j^T A_j^{-1} R_j (b - A x) for one vertex patch
                        (Eq. 2.5/2.6, equivalently the localised form of
                        Section 2.2 that only reads the patch closure);
* ``patch_boundary_solve`` -- the new interior values A_j^{-1}(b^I - A^{IB} x^B)
                        of the reduced local residual of Section 3.2
                        ("Boundary"), from the partition of Abar_j into
                        interior and boundary columns;
* ``apply_rows``     -- (A x)_i for chosen nodes i;
* ``prolongate_rows``-- (I^up x_c)_i for chosen fine nodes i;
* ``restrict_rows``  -- ((I^up)^T r_f)_j for chosen coarse nodes j.

Inputs are full-grid vectors of a level (n1^d values, boundary entries 0).
The tests pin each function against the globally assembled oracle at small
sizes.
"""

import numpy as np
import scipy.linalg as sla

from . import fe


def _cell_matrix(level):
    return fe.cell_stiffness(level.d, level.k, level.h)


def _cells_containing(level, g):
    """Cells (multi-index) whose closure contains full-grid node multi-index g."""
    k, d = level.k, level.d
    options = []
    for t in range(d):
        c = []
        if g[t] % k == 0:
            if g[t] // k - 1 >= 0:
                c.append(g[t] // k - 1)
            if g[t] // k < level.ncell:
                c.append(g[t] // k)
        else:
            c.append(g[t] // k)
        options.append(c)
    out = [[]]
    for t in range(d):
        out = [o + [c] for o in out for c in options[t]]
    return [np.array(o) for o in out]


def apply_rows(level, xfull, nodes):
    """(A x)_g for each full-grid node multi-index g in ``nodes`` (interior).

    Sum over the cells containing g of the element matrix row of g times
    the cell's nodal values (Eq. 2.4).
    """
    d, k, n1 = level.d, level.k, level.n1
    AK = _cell_matrix(level)
    Lc = fe.multi_indices(k + 1, d)
    out = np.zeros(len(nodes))
    for r, g in enumerate(nodes):
        g = np.asarray(g)
        acc = 0.0
        for c in _cells_containing(level, g):
            loc = g - k * c
            a = int(sum(loc[t] * (k + 1) ** t for t in range(d)))
            gi = np.zeros(len(Lc), dtype=np.int64)
            for t in range(d):
                gi += (k * c[t] + Lc[:, t]) * n1 ** t
            acc += AK[a] @ xfull[gi]
        out[r] = acc
    return out


def patch_matrices(level):
    """(Abar, Aj): rows of A at the patch interior over the closure, and A_j.

    Assembled from the 2^d element matrices of one patch.  Closure nodes are
    numbered lexicographically over the (2k+1)^d closure grid; interior
    rows are the closure nodes with all local coordinates in 1..2k-1.
    """
    d, k = level.d, level.k
    n = 2 * k + 1
    AK = _cell_matrix(level)
    Lc = fe.multi_indices(k + 1, d)
    Abar_full = np.zeros((n ** d, n ** d))
    for cell in fe.multi_indices(2, d):
        li = np.zeros(len(Lc), dtype=np.int64)
        for t in range(d):
            li += (k * cell[t] + Lc[:, t]) * n ** t
        Abar_full[np.ix_(li, li)] += AK
    Ln = fe.multi_indices(n, d)
    interior = np.all((Ln >= 1) & (Ln <= n - 2), axis=1)
    rows = np.nonzero(interior)[0]
    Abar = Abar_full[rows]
    Aj = Abar[:, rows]
    return Abar, Aj, rows


def patch_update(level, xfull, bfull, v, mats=None):
    """Correction A_j^{-1} (R_j b - Abar_j Rbar_j x) of the patch at vertex v.

    Returns (interior full-grid indices, correction values).
    """
    d, k, n1 = level.d, level.k, level.n1
    n = 2 * k + 1
    Abar, Aj, rows = patch_matrices(level) if mats is None else mats
    Ln = fe.multi_indices(n, d)
    gi = np.zeros(len(Ln), dtype=np.int64)
    for t in range(d):
        gi += (k * (v[t] - 1) + Ln[:, t]) * n1 ** t
    r = bfull[gi[rows]] - Abar @ xfull[gi]
    return gi[rows], sla.solve(Aj, r, assume_a="sym")


def patch_boundary_solve(level, xfull, bfull, v, mats=None):
    """x^I <- A_j^{-1} (b^I - A^{IB} x^B) for the patch at vertex v (Section 3.2).

    Abar_j = [A^{II} A^{IB}] over the closure columns split into the patch
    interior I and its boundary B; A_j = A^{II}.  Returns (interior
    full-grid indices, new interior values).
    """
    d, k, n1 = level.d, level.k, level.n1
    n = 2 * k + 1
    Abar, Aj, rows = patch_matrices(level) if mats is None else mats
    Ln = fe.multi_indices(n, d)
    gi = np.zeros(len(Ln), dtype=np.int64)
    for t in range(d):
        gi += (k * (v[t] - 1) + Ln[:, t]) * n1 ** t
    bcols = np.setdiff1d(np.arange(len(Ln)), rows)
    AIB = Abar[:, bcols]
    r = bfull[gi[rows]] - AIB @ xfull[gi[bcols]]
    return gi[rows], sla.solve(Aj, r, assume_a="sym")


def prolongate_rows(fine, xc_full, nodes):
    """(I^up x_c)_g at fine full-grid nodes g: coarse basis at the point."""
    d, k = fine.d, fine.k
    coarse = fe.Level(d, k, fine.l - 1)
    H = coarse.h
    xf1 = fine.node_coords_1d()
    Lc = fe.multi_indices(k + 1, d)
    out = np.zeros(len(nodes))
    for r, g in enumerate(nodes):
        val = np.ones(len(Lc))
        gi = np.zeros(len(Lc), dtype=np.int64)
        for t in range(d):
            x = xf1[g[t]]
            c = min(int(np.floor(x / H)), coarse.ncell - 1)
            V = fe.lagrange_values(coarse.z, [(x - c * H) / H])[:, 0]
            val *= V[Lc[:, t]]
            gi += (k * c + Lc[:, t]) * coarse.n1 ** t
        out[r] = val @ xc_full[gi]
    return out


def restrict_rows(fine, rf_full, coarse_nodes):
    """((I^up)^T r_f)_j at coarse full-grid nodes j: sum over the fine support
    points i inside the support of coarse basis function j of phi_j(x_i) r_i."""
    d, k = fine.d, fine.k
    coarse = fe.Level(d, k, fine.l - 1)
    H = coarse.h
    xf1 = fine.node_coords_1d()
    out = np.zeros(len(coarse_nodes))
    for r, j in enumerate(coarse_nodes):
        # per direction: fine nodes in the coarse cells touching node j, and phi_j there
        idx, wts = [], []
        for t in range(d):
            cells = []
            if j[t] % k == 0:
                if j[t] // k - 1 >= 0:
                    cells.append(j[t] // k - 1)
                if j[t] // k < coarse.ncell:
                    cells.append(j[t] // k)
            else:
                cells.append(j[t] // k)
            g = sorted(set(f for c in cells for f in range(2 * k * c, 2 * k * (c + 1) + 1)))
            w = []
            for f in g:
                x = xf1[f]
                c = min(int(np.floor(x / H)), coarse.ncell - 1)
                if c not in cells:  # a shared endpoint evaluated in the other cell
                    c = cells[-1] if x >= cells[-1] * H else cells[0]
                loc = j[t] - k * c
                w.append(fe.lagrange_values(coarse.z, [(x - c * H) / H])[loc, 0] if 0 <= loc <= k else 0.0)
            idx.append(np.array(g))
            wts.append(np.array(w))
        acc = 0.0
        grids = np.meshgrid(*[np.arange(len(i)) for i in idx], indexing="ij")
        for combo in zip(*[gg.ravel() for gg in grids]):
            w = np.prod([wts[t][combo[t]] for t in range(d)])
            if w == 0.0:
                continue
            f = sum(idx[t][combo[t]] * fine.n1 ** t for t in range(d))
            acc += w * rf_full[f]
        out[r] = acc
    return out
