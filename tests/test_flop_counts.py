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


# ------------------------------------------------------------ even/odd halves
# The kernels apply every 1D matrix through its even/odd halves: the two-cell
# patch is symmetric about its centre, so the patch matrices are
# centrosymmetric (W[m-1-o][n-1-c] = W[o][c]) and the eigenvectors of the
# interior blocks have even or odd parity.  The same update is executed here
# in that form, every operation counted (FMA = 2, add/multiply = 1), and
# checked against the dense patch operator and inverse and against
# smoother_flops_executed_per_patch.

from paper_2405_19004_gb300.studies import smoother_flops_executed_per_patch  # noqa: E402


def _centrosymmetric(k, rng):
    A, M = _patch_matrices(k, rng)
    J = np.eye(A.shape[0])[::-1]
    return 0.5 * (A + J @ A @ J), 0.5 * (M + J @ M @ J)


def _parity_eigen(AI, MI):
    """Generalised eigenvectors on the even and odd subspaces: S (even
    columns first) with exact parity, and the eigenvalues."""
    m = AI.shape[0]
    h = (m - 1) // 2
    B = np.zeros((m, m))
    r2 = np.sqrt(0.5)
    for j in range(h):
        B[j, j] = B[m - 1 - j, j] = r2
        B[j, h + 1 + j], B[m - 1 - j, h + 1 + j] = r2, -r2
    B[h, h] = 1.0
    S = np.zeros((m, m))
    lam = np.zeros(m)
    for cols in (slice(0, h + 1), slice(h + 1, m)):
        Bp = B[:, cols]
        if Bp.shape[1] == 0:
            continue
        w, V = scipy.linalg.eigh(Bp.T @ AI @ Bp, Bp.T @ MI @ Bp)
        lam[cols] = w
        S[:, cols] = Bp @ V
    return S, lam


class EO:
    """Even/odd contractions along an axis, counted."""

    def __init__(self):
        self.flops = 0

    def split(self, t, axis):
        t = np.moveaxis(t, axis, 0)
        hk = (t.shape[0] - 1) // 2
        e = t[:hk] + t[::-1][:hk]
        d = t[:hk] - t[::-1][:hk]
        self.flops += 2 * hk * t[0].size
        return np.concatenate([e, t[hk:hk + 1]]), d

    def halves(self, W):
        m, n = W.shape
        k, h = (n - 1) // 2, (m - 1) // 2
        WE = np.concatenate([0.5 * (W[:h + 1, :k] + W[:h + 1, ::-1][:, :k]), W[:h + 1, k:k + 1]], 1)
        WO = 0.5 * (W[:h, :k] - W[:h, ::-1][:, :k])
        return WE, WO

    def apply(self, W, e, d):
        """Even and odd sums of the interior rows of W (m x n) on split lines."""
        WE, WO = self.halves(W)
        lines = e[0].size
        self.flops += 2 * lines * (WE.size + WO.size)
        return np.tensordot(WE, e, axes=(1, 0)), np.tensordot(WO, d, axes=(1, 0))

    def combine(self, E, O, axis):
        h = O.shape[0]
        self.flops += 2 * h * E[0].size
        out = np.concatenate([E[:h] + O, E[h:h + 1], (E[:h] - O)[::-1]])
        return np.moveaxis(out, 0, axis)

    def st(self, S, t, axis):
        """S^T along axis: even components from the even parts, odd from odd."""
        t = np.moveaxis(t, axis, 0)
        m = t.shape[0]
        h = (m - 1) // 2
        e = np.concatenate([t[:h] + t[::-1][:h], t[h:h + 1]])
        d = t[:h] - t[::-1][:h]
        SE, SO = S[:h + 1, :h + 1], S[:h, h + 1:]
        self.flops += 2 * h * t[0].size + 2 * t[0].size * (SE.size + SO.size)
        out = np.concatenate([np.tensordot(SE.T, e, axes=(1, 0)), np.tensordot(SO.T, d, axes=(1, 0))])
        return np.moveaxis(out, 0, axis)

    def s(self, S, t, axis):
        t = np.moveaxis(t, axis, 0)
        m = t.shape[0]
        h = (m - 1) // 2
        SE, SO = S[:h + 1, :h + 1], S[:h, h + 1:]
        self.flops += 2 * t[0].size * (SE.size + SO.size)
        E = np.tensordot(SE, t[:h + 1], axes=(1, 0))
        O = np.tensordot(SO, t[h + 1:], axes=(1, 0))
        return self.combine(E, O, axis)


def _eo_update(c, A, M, S, lam, x, b, s, d, boundary):
    """The kernels' schedule: residual contractions z -> y -> x (2D: y -> x),
    then S^T per direction, the scaling, S per direction; x_I += u or, with
    `boundary`, x_I = u.  Returns the new interior."""
    n = A.shape[0]
    m = n - 2
    AI, MI = A[1:-1, :], M[1:-1, :]
    if boundary:
        # lines of the first contraction through the interior: the two end
        # nodes only, one multiply and one multiply-add per output and matrix
        lines = (m * m) if d == 3 else m
        inner = np.zeros((n,) * (d - 1), dtype=bool)
        inner[(slice(1, n - 1),) * (d - 1)] = True
        faces = (~inner).sum()
        xb = np.moveaxis(x, 0, -1)
        mz = np.zeros(xb.shape[:-1] + (m,))
        az = np.zeros_like(mz)
        e, dd = c.split(np.moveaxis(xb[~inner], -1, 0), 0)
        E, O = c.apply(MI, e, dd)
        mz[~inner] = np.moveaxis(c.combine(E, O, 0), 0, -1)
        E, O = c.apply(AI, e, dd)
        az[~inner] = np.moveaxis(c.combine(E, O, 0), 0, -1)
        ends = xb[inner][:, [0, -1]]
        mz[inner] = ends @ MI[:, [0, -1]].T
        az[inner] = ends @ AI[:, [0, -1]].T
        c.flops += lines * 2 * 3 * m
        assert faces == (8 * ((n - 1) // 2) if d == 3 else 2)
        mz, az = np.moveaxis(mz, -1, 0), np.moveaxis(az, -1, 0)
    else:
        e, dd = c.split(x, 0)
        mz = c.combine(*c.apply(MI, e, dd), 0)
        az = c.combine(*c.apply(AI, e, dd), 0)
    if d == 3:
        em, dm = c.split(mz, 1)
        ea, da = c.split(az, 1)
        U = c.combine(*c.apply(MI, em, dm), 1)
        E1, O1 = c.apply(AI, em, dm)
        E2, O2 = c.apply(MI, ea, da)
        W = c.combine(E1 + E2, O1 + O2, 1)  # one accumulator for both products
        eu, du = c.split(U, 2)
        ew, dw = c.split(W, 2)
        E1, O1 = c.apply(AI, eu, du)
        E2, O2 = c.apply(MI, ew, dw)
        r = s * b - c.combine(E1 + E2, O1 + O2, 2)
    else:
        em, dm = c.split(mz, 1)
        ea, da = c.split(az, 1)
        E1, O1 = c.apply(AI, em, dm)
        E2, O2 = c.apply(MI, ea, da)
        r = s * b - c.combine(E1 + E2, O1 + O2, 1)
    c.flops += 2 * r.size  # s b - (..) as one fma
    L = lam
    for _ in range(d - 1):
        L = np.add.outer(L, lam)
    for ax in range(d):
        r = c.st(S, r, ax)
    r = r / L
    c.flops += r.size
    for ax in range(d):
        r = c.s(S, r, ax)
    xi = x[(slice(1, n - 1),) * d]
    c.flops += r.size * (1 if boundary else 2)  # x_I = 1 * u, or x_I += 1 * u as one fma
    return r if boundary else xi + r


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 6])
@pytest.mark.parametrize("boundary", [False, True])
def test_even_odd_update_matches_dense_and_executed_count(d, k, boundary):
    rng = np.random.default_rng(300 * d + 10 * k + boundary)
    n, m = 2 * k + 1, 2 * k - 1
    A, M = _centrosymmetric(k, rng)
    S, lam = _parity_eigen(A[1:-1, 1:-1], M[1:-1, 1:-1])
    x = rng.standard_normal((n,) * d)
    if boundary:
        x[(slice(1, n - 1),) * d] = 0.0
    b = rng.standard_normal((m,) * d)
    c = EO()
    got = _eo_update(c, A, M, S, lam, x, b, 1.0, d, boundary)
    # dense: x_I + A_I^-1 (b - Abar x)
    Abar = _dense_patch(A, M, d)
    inner = np.zeros((n,) * d, dtype=bool)
    inner[(slice(1, n - 1),) * d] = True
    rd = b.ravel() - (Abar @ x.ravel())[inner.ravel()]
    AbarI = _dense_patch(A[1:-1, 1:-1], M[1:-1, 1:-1], d)
    ref = x[inner] + np.linalg.solve(AbarI, rd)
    assert np.allclose(got.ravel(), ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
    assert c.flops == smoother_flops_executed_per_patch(d, k, boundary)


def test_paper_count_per_dof_at_the_degree_sweep_sizes():
    """The plain sum-factorisation count per patch (the roofline's algorithmic
    work) per DoF at the sweep's sizes: 3D on 2^7 cells (2^8 for k = 2, 2^6 for
    k = 6, 7), 2D on 2^12, as tabulated for the degree sweep."""
    from paper_2405_19004_gb300.studies import paper_flops_per_patch
    want = {3: [513, 788, 1140, 1521, 1911, 2262, 2651], 2: [155, 261, 381, 505, 630, 756, 883]}
    lev3 = [7, 8, 7, 7, 7, 6, 6]
    for d in (2, 3):
        for k in range(1, 8):
            L = lev3[k - 1] if d == 3 else 12
            per_dof = paper_flops_per_patch(d, k) * (2 ** L - 1) ** d / (k * 2 ** L - 1) ** d
            assert round(per_dof) == want[d][k - 1], (d, k)
    # and it counts more than the kernels' dense count (the shared mass contraction)
    from paper_2405_19004_gb300.studies import smoother_flops_per_patch
    for d in (2, 3):
        for k in range(1, 8):
            assert paper_flops_per_patch(d, k) > smoother_flops_per_patch(d, k)
