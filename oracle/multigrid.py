"""Multigrid V-cycle, full multigrid and preconditioned CG (oracle; test infrastructure only).

* V-cycle: Algorithm 1 (pre-smooth, residual, restrict with the transpose of
  the prolongation, recurse from a zero initial guess, prolongate-add,
  post-smooth).  The coarse problem is solved exactly (dense LU) on a
  chosen coarsest level (default 1).  The paper closes the
  recursion "on level 0" with one smoother step; the mesh M_0 has no interior
  vertex, so the reading used here is that the coarsest level is level 1,
  whose single vertex patch covers every interior DoF -- one patch solve is
  the exact coarse solve.  It is computed here by dense LU of A_1.
* Symmetric variant (``symmetric=True``): post-smoothing visits the colours in
  reverse order, which makes the cycle a symmetric preconditioner for CG
  (the paper uses the same smoother on both sides with GMRES).
* Full multigrid: Algorithm 2, counting the V-cycles of its while loop.
* PCG: conjugate gradients on level L preconditioned by one V-cycle, x0 = 0,
  stopping at ||b - A x|| <= rtol ||b||; beta in the flexible
  (Polak-Ribiere) form r_{i+1}^T (z_{i+1} - z_i) / r_i^T z_i.
* FGMRES: GMRES (the paper's outer solver, Section 4) with right
  preconditioning by one V-cycle, in the flexible form that stores the
  preconditioned vectors (the V-cycle may be inexact, e.g. in FP32); Arnoldi
  by modified Gram-Schmidt, Givens rotations, restarts.
* L2 error: ||u_h - u||_{L2} with (k+2)^d Gauss points per cell.
"""

import numpy as np
import scipy.linalg as sla

from . import fe, assembly, smoothers


class Hierarchy:
    """Levels 1..L of one problem (d, k): A_l, I^up_l, patch solvers."""

    def __init__(self, d, k, L, smoother="multiplicative", omega=1.0,
                 n_pre=1, n_post=1, symmetric=True, coarse_level=1):
        """coarse_level: the level solved exactly (Algorithm 1's coarse grid
        solver); 1 recurses as deep as the mesh allows."""
        if L < 1 or not 1 <= coarse_level <= L:
            raise ValueError("need 1 <= coarse_level <= L")
        self.d, self.k, self.L = d, k, L
        self.coarse = coarse_level
        self.smoother, self.omega = smoother, omega
        self.n_pre, self.n_post, self.symmetric = n_pre, n_post, symmetric
        lo = coarse_level
        self.levels = {l: fe.Level(d, k, l) for l in range(lo, L + 1)}
        self.A = {l: assembly.stiffness(self.levels[l]) for l in range(lo, L + 1)}
        self.P = {l: assembly.prolongation(self.levels[l]) for l in range(lo + 1, L + 1)}
        self.ps = {l: smoothers.PatchSolver(self.levels[l], self.A[l])
                   for l in range(max(2, lo + 1), L + 1)}
        self.coarse_lu = sla.lu_factor(self.A[lo].toarray())

    def smooth(self, l, x, b, forward=True):
        if self.smoother == "additive":
            return smoothers.additive(self.A[l], self.ps[l], x, b, self.omega)
        nc = 2 ** self.d
        order = range(nc) if forward else range(nc - 1, -1, -1)
        return smoothers.multiplicative(self.A[l], self.ps[l], x, b, order)

    def vcycle(self, l, b, x=None):
        """x_l = Vcycle_l(A_l, x, b) (Algorithm 1); x defaults to 0."""
        if l == self.coarse:
            return sla.lu_solve(self.coarse_lu, b)
        x = np.zeros_like(b) if x is None else np.array(x, dtype=np.float64)
        for _ in range(self.n_pre):
            x = self.smooth(l, x, b, forward=True)
        r = b - self.A[l] @ x
        rc = self.P[l].T @ r
        x = x + self.P[l] @ self.vcycle(l - 1, rc)
        for _ in range(self.n_post):
            x = self.smooth(l, x, b, forward=not self.symmetric)
        return x

    def precondition(self, r):
        return self.vcycle(self.L, r)


def pcg(A, b, precond, rtol=1e-10, max_it=200):
    """Preconditioned CG with flexible beta; returns (x, iterations, rel_res).

    The iteration count is the number of products A p taken.
    """
    x = np.zeros_like(b)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, 0.0
    r = b.copy()
    z = precond(r)
    p = z.copy()
    rz = r @ z
    rel = 1.0
    for it in range(1, max_it + 1):
        Ap = A @ p
        pAp = p @ Ap
        if not np.isfinite(pAp) or pAp <= 0.0:
            raise FloatingPointError("CG breakdown: p^T A p <= 0")
        alpha = rz / pAp
        x = x + alpha * p
        r_new = r - alpha * Ap
        rel = np.linalg.norm(r_new) / nb
        if rel <= rtol:
            return x, it, rel
        z_new = precond(r_new)
        beta = (r_new @ (z_new - z)) / rz
        rz = r_new @ z_new
        p = z_new + beta * p
        r, z = r_new, z_new
    return x, max_it, rel


def fmg_iterations(d, k, L, f, tol=1e-9, max_it=100):
    """Full multigrid (Algorithm 2) with the paper's V-cycle; V-cycle count.

    The same forward colour order is used before and after the coarse
    correction (Algorithm 1 applies S_l on both sides).  Right-hand sides are
    assembled on every level from f.  Returns the number of while-loop
    repetitions until ||b_L - A_L x_L|| <= tol ||b_L||.
    """
    H = Hierarchy(d, k, L, symmetric=False)
    b = {l: assembly.load_vector(H.levels[l], f) for l in range(1, L + 1)}
    x = sla.lu_solve(H.coarse_lu, b[1])
    for l in range(2, L + 1):
        x = H.P[l] @ x
        x = H.vcycle(l, b[l], x)
    d0 = np.linalg.norm(b[L])
    delta = d0
    it = 0
    while delta > tol * d0 and it < max_it:
        x = H.vcycle(L, b[L], x)
        delta = np.linalg.norm(b[L] - H.A[L] @ x)
        it += 1
    return it


def fgmres(A, b, precond, rtol=1e-9, restart=30, max_it=300):
    """Flexible GMRES, x0 = 0; returns (x, iterations, rel_res, history).

    Each cycle builds an orthonormal basis v_1 = r / ||r||, ..., with
    z_j = precond(v_j) and A z_j orthogonalised against v_1..v_j (modified
    Gram-Schmidt); x = x0 + Z y with y minimising ||beta e_1 - H y|| (Givens
    rotations).  The loop stops when the least-squares residual |g_{j+1}|
    is <= rtol ||b|| or after max_it products A z; a cycle ends after
    `restart` of them and the next one starts from r = b - A x.  history:
    the least-squares residual after every product.
    """
    n = len(b)
    x = np.zeros(n)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, 0.0, []
    it, hist = 0, []
    r = b.copy()
    beta = np.linalg.norm(r)
    while True:
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        j = 0
        while j < restart and it < max_it:
            z = precond(V[j])
            Z.append(z)
            w = A @ z
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j] if H[j + 1, j] > 0 else w)
            for i in range(j):  # previous rotations on the new column
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            j += 1
            it += 1
            hist.append(abs(g[j]) / nb)
            if abs(g[j]) <= rtol * nb:
                break
        y = sla.solve_triangular(H[:j, :j], g[:j])
        x = x + np.array(Z).T @ y
        r = b - A @ x
        beta = np.linalg.norm(r)
        if beta <= rtol * nb or it >= max_it:
            return x, it, beta / nb, hist


def l2_error(level, x, u):
    """||u_h - u||_{L2(Omega)} for the compact interior vector x.

    u_h = sum_i x_i phi_i (boundary coefficients 0); (k+2)^d Gauss points per
    cell.
    """
    d, k, h = level.d, level.k, level.h
    q = k + 2
    xq, wq = fe.gauss_points(q)
    V = fe.lagrange_values(level.z, xq)
    E = fe.tensor_basis_at([V] * d, d, k + 1, q)            # (nloc, q^d)
    Q = fe.multi_indices(q, d)
    W = np.ones(q ** d)
    for t in range(d):
        W *= wq[Q[:, t]]
    W = W * h ** d
    C = fe.multi_indices(level.ncell, d)
    X = (C[:, None, :] + xq[Q][None, :, :]) * h
    cells = level.cell_node_indices()
    g2c = level.global_to_compact()
    full = np.zeros(level.n1 ** d)
    inside = g2c >= 0
    full[inside] = x[g2c[inside]]
    uh = full[cells] @ E                                      # (ncells, q^d)
    ue = np.asarray(u(X.reshape(-1, d))).reshape(uh.shape)
    return float(np.sqrt(np.sum((uh - ue) ** 2 * W)))
