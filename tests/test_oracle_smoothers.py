"""Pins of the oracle's vertex-patch smoothers (Section 2.2, Eq. 2.5-2.7, Algorithm 3)."""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import assembly, fe, smoothers


def _setup(d, k, l):
    lv = fe.Level(d, k, l)
    A = assembly.stiffness(lv)
    return lv, A, smoothers.PatchSolver(lv, A)


@pytest.mark.parametrize("d,k", [(2, 1), (2, 2), (2, 5), (3, 1), (3, 2), (3, 3)])
def test_level1_single_patch_step_is_exact_solve(d, k):
    """Level 1 has one interior vertex whose patch holds every DoF: one step from 0 solves."""
    lv, A, ps = _setup(d, k, 1)
    assert len(ps.I) == 1 and ps.I.shape[1] == lv.N
    b = np.random.default_rng(1).normal(size=lv.N)
    x = smoothers.multiplicative(A, ps, np.zeros(lv.N), b)
    np.testing.assert_allclose(x, spla.spsolve(A.tocsc(), b), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("d,l", [(2, 3), (3, 2)])
def test_q1_smoother_is_four_colour_point_gauss_seidel(d, l):
    """Q1: each patch holds one DoF, so one step is point Gauss-Seidel in colour order.

    Textbook point GS written as a plain loop: x_i += (b_i - sum_j a_ij x_j) / a_ii.
    """
    lv, A, ps = _setup(d, 1, l)
    rng = np.random.default_rng(2)
    x0, b = rng.normal(size=lv.N), rng.normal(size=lv.N)
    Ad = A.toarray()
    x = x0.copy()
    V = smoothers.vertices(lv)
    for c in range(2 ** d):
        for v in V:
            if smoothers.colour_of(v) != c:
                continue
            i = int(sum((v[t] - 1) * lv.ni ** t for t in range(d)))
            x[i] += (b[i] - Ad[i] @ x) / Ad[i, i]
    np.testing.assert_allclose(smoothers.multiplicative(A, ps, x0, b), x, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("d,k,l", [(2, 2, 3), (2, 3, 2), (3, 2, 2)])
def test_colour_parallel_equals_sequential(d, k, l):
    """Algorithm 3 (parallel inside a colour) equals Eq. 2.7 (strictly sequential)."""
    lv, A, ps = _setup(d, k, l)
    rng = np.random.default_rng(3)
    x0, b = rng.normal(size=lv.N), rng.normal(size=lv.N)
    xs = smoothers.multiplicative_sequential(A, ps, x0, b)
    xp = smoothers.multiplicative(A, ps, x0, b)
    assert np.abs(xs - xp).max() <= 1e-14 * np.abs(xs).max()
    rev = list(range(2 ** d))[::-1]
    xs = smoothers.multiplicative_sequential(A, ps, x0, b, rev)
    xp = smoothers.multiplicative(A, ps, x0, b, rev)
    assert np.abs(xs - xp).max() <= 1e-14 * np.abs(xs).max()


@pytest.mark.parametrize("d,k,l", [(2, 2, 3), (3, 3, 2)])
def test_same_colour_patches_do_not_overlap(d, k, l):
    """Interior of a patch is disjoint from the closure of every other same-colour patch."""
    lv = fe.Level(d, k, l)
    V = smoothers.vertices(lv)
    col = smoothers.colour_of(V)
    g2c = lv.global_to_compact()
    for c in range(2 ** d):
        js = np.nonzero(col == c)[0]
        for a in js:
            Ia = set(smoothers.patch_interior(lv, V[a]).tolist())
            for b in js:
                if a == b:
                    continue
                cl = g2c[smoothers.patch_closure_full(lv, V[b])]
                assert not (Ia & set(cl[cl >= 0].tolist()))
    counts = smoothers.colour_counts(lv)
    assert counts.sum() == (2 ** l - 1) ** d
    assert counts[0] == 2 ** ((l - 1) * d)


def test_patch_interior_is_2k_minus_1_cubed():
    lv = fe.Level(3, 3, 2)
    I = smoothers.patch_interior(lv, np.array([2, 1, 3]))
    assert len(I) == 5 ** 3 and len(set(I.tolist())) == 125
    assert I.min() >= 0 and I.max() < lv.N


@pytest.mark.parametrize("d,k,l", [(2, 2, 3), (3, 2, 2)])
def test_additive_smoother_is_symmetric_and_linear(d, k, l):
    """x -> additive(x) is affine with a symmetric linear part omega sum R^T A_j^-1 R."""
    lv, A, ps = _setup(d, k, l)
    N = lv.N
    rng = np.random.default_rng(4)
    cols = rng.choice(N, size=6, replace=False)
    Bcols = []
    for i in cols:
        e = np.zeros(N)
        e[i] = 1.0
        Bcols.append(smoothers.additive(A, ps, np.zeros(N), e, 0.7))
    B = np.stack(Bcols, axis=1)
    np.testing.assert_allclose(B[cols], B[cols].T, atol=1e-13)
    x0, b = rng.normal(size=N), rng.normal(size=N)
    lin = smoothers.additive(A, ps, x0, b, 0.7) - x0
    np.testing.assert_allclose(lin, 0.7 * (smoothers.additive(A, ps, np.zeros(N), b - A @ x0, 1.0)),
                               atol=1e-12)


@pytest.mark.parametrize("d,k,l", [(2, 2, 3), (2, 3, 3), (3, 2, 2)])
def test_additive_operator_norm_is_two_to_the_d(d, k, l):
    """lambda_max(sum_j P_j) = 2^d for k >= 2: a cell bubble lies in 2^d patch interiors."""
    lv, A, ps = _setup(d, k, l)
    N = lv.N
    Ad = A.toarray()
    Bs = np.zeros((N, N))
    Ainv = np.linalg.inv(ps.Aj)
    for I in ps.I:
        Bs[np.ix_(I, I)] += Ainv
    lam = np.linalg.eigvals(Bs @ Ad).real
    assert abs(lam.max() - 2 ** d) < 1e-9
