"""The algorithmic work behind the smoother's roofline figures.

bench.py and the studies divide smoother_flops_per_patch by measured times.
Here the sum-factorised patch update is executed step by step in numpy with
every contraction's multiply-adds counted (FMA = 2 flops) and checked two
ways: its result against the dense patch operator and its dense inverse
(Eq. 2.13/2.14, Sections 3.1.1 and 3.2), its count against the closed form.

Schedule counted (n = 2k+1 closure, m = 2k-1 interior nodes per direction):
  residual r = s b_I - (sum_t M x..x A_t x..x M) x on the interior rows, by
  contractions along z, then y, then x, reusing the inner mass contraction;
  the Boundary variant reads only the closure boundary x_B, so in its first
  contraction the lines through the interior have just two nonzero nodes;
  then u = (S x S x S) diag(1 / sum lambda) (S x S x S)^T r and x_I += u
  (Boundary: x_I = u).  Pointwise: 2 flops for the residual's fma, 1 for the
  scaling, 1 for the update.
"""
import numpy as np
import pytest
import scipy.linalg

from paper_2405_19004_gb300.studies import smoother_flops_per_patch


class Counter:
    def __init__(self):
        self.flops = 0

    def contract(self, mat, t, axis, cols=None):
        """mat (m x n) applied along `axis` of t; cols: the nonzero input
        positions along that axis (all when None)."""
        t = np.moveaxis(t, axis, 0)
        lines = t[0].size
        used = mat.shape[1] if cols is None else len(cols)
        self.flops += 2 * lines * mat.shape[0] * used
        if cols is not None:
            out = np.tensordot(mat[:, cols], t[cols], axes=(1, 0))
        else:
            out = np.tensordot(mat, t, axes=(1, 0))
        return np.moveaxis(out, 0, axis)


def _patch_matrices(k, rng):
    n = 2 * k + 1
    B = rng.standard_normal((n, n))
    M = B @ B.T + n * np.eye(n)  # SPD mass-like
    C = rng.standard_normal((n, n))
    A = C @ C.T + np.eye(n)      # SPD stiffness-like
    return A, M


def _dense_patch(A, M, d):
    terms = []
    for t in range(d):
        f = [M] * d
        f[t] = A
        K = f[0]
        for g in f[1:]:
            K = np.kron(K, g)
        terms.append(K)
    return sum(terms)


def _residual_3d(c, A, M, x, b, s, boundary):
    """Interior rows of s b - Abar x (3D, axes z, y, x), counted.  With
    `boundary` the first contraction skips the zero interior of x."""
    n = A.shape[0]
    I = slice(1, n - 1)
    AI, MI = A[I, :], M[I, :]
    if boundary:
        # z-lines (y, x): on a face (y or x on the boundary) all n nodes,
        # through the interior only z = 0 and z = n-1
        face = np.zeros((n, n), dtype=bool)
        face[[0, -1], :] = True
        face[:, [0, -1]] = True
        mz = np.zeros((n - 2, n, n))
        az = np.zeros((n - 2, n, n))
        for yy in range(n):
            for xx in range(n):
                col = x[:, yy, xx]
                cols = None if face[yy, xx] else [0, n - 1]
                mz[:, yy, xx] = c.contract(MI, col, 0, cols)
                az[:, yy, xx] = c.contract(AI, col, 0, cols)
    else:
        mz = c.contract(MI, x, 0)
        az = c.contract(AI, x, 0)
    mm = c.contract(MI, mz, 1)                              # M_y M_z x
    w = c.contract(AI, mz, 1) + c.contract(MI, az, 1)       # A_y M_z x + M_y A_z x (one accumulator)
    out = c.contract(AI, mm, 2) + c.contract(MI, w, 2)      # A_x (..) + M_x (..)
    c.flops += 2 * b.size                                    # s b - (..) as one fma
    return s * b - out


def _residual_2d(c, A, M, x, b, s, boundary):
    n = A.shape[0]
    I = slice(1, n - 1)
    AI, MI = A[I, :], M[I, :]
    if boundary:
        my = np.zeros((n - 2, n))
        ay = np.zeros((n - 2, n))
        for xx in range(n):
            cols = None if xx in (0, n - 1) else [0, n - 1]
            my[:, xx] = c.contract(MI, x[:, xx], 0, cols)
            ay[:, xx] = c.contract(AI, x[:, xx], 0, cols)
    else:
        my = c.contract(MI, x, 0)
        ay = c.contract(AI, x, 0)
    out = c.contract(AI, my, 1) + c.contract(MI, ay, 1)
    c.flops += 2 * b.size
    return s * b - out


def _fd_solve(c, S, lam, r, d):
    for ax in range(d):
        r = c.contract(S.T, r, ax)
    L = lam
    for _ in range(d - 1):
        L = np.add.outer(L, lam)
    r = r / L
    c.flops += r.size
    for ax in range(d):
        r = c.contract(S, r, ax)
    return r


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("boundary", [False, True])
def test_counted_patch_update_matches_dense_and_closed_form(d, k, boundary):
    rng = np.random.default_rng(100 * d + 10 * k + boundary)
    n, m = 2 * k + 1, 2 * k - 1
    A, M = _patch_matrices(k, rng)
    x = rng.standard_normal((n,) * d)
    b = rng.standard_normal((m,) * d)
    s = 0.75
    if boundary:
        x[(slice(1, n - 1),) * d] = 0.0  # the Boundary kernel never reads x_I
    c = Counter()
    r = (_residual_3d if d == 3 else _residual_2d)(c, A, M, x, b, s, boundary)

    # dense check of the residual
    Abar = _dense_patch(A, M, d)
    inner = np.zeros((n,) * d, dtype=bool)
    inner[(slice(1, n - 1),) * d] = True
    rd = s * b.ravel() - (Abar @ x.ravel())[inner.ravel()]
    assert np.allclose(r.ravel(), rd, rtol=1e-12, atol=1e-10 * np.abs(rd).max())

    # fast diagonalisation of the interior blocks: S^T M_I S = I, S^T A_I S = Lambda
    AI = A[1:-1, 1:-1]
    MI = M[1:-1, 1:-1]
    lam, S = scipy.linalg.eigh(AI, MI)
    u = _fd_solve(c, S, lam, r, d)
    AbarI = _dense_patch(AI, MI, d)
    ud = np.linalg.solve(AbarI, rd)
    assert np.allclose(u.ravel(), ud, rtol=1e-9, atol=1e-9 * np.abs(ud).max())
    if not boundary:
        c.flops += u.size  # x_I += u
    assert c.flops == smoother_flops_per_patch(d, k, boundary)


def test_closed_form_values_quoted_for_q4():
    # the per-patch counts quoted with the 3D Q4 measurements
    assert smoother_flops_per_patch(3, 4, False) == 86758
    assert smoother_flops_per_patch(3, 4, True) == 76811
