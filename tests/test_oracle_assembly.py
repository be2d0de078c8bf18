"""Pins of the oracle's assembled operators (Section 2, Eq. 2.3/2.4; Section 2.1)."""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import assembly, fe


def _bubble(d):
    u = lambda X: np.prod(X * (1 - X), axis=1)

    def f(X):  # -Laplace of prod x_t (1 - x_t)
        s = np.zeros(len(X))
        for t in range(d):
            s += 2 * np.prod(np.delete(X * (1 - X), t, axis=1), axis=1)
        return s
    return u, f


def test_q1_2d_nine_point_stencil():
    """Textbook: bilinear Q1 Laplacian = 8/3 centre, -1/3 at all 8 neighbours."""
    lv = fe.Level(2, 1, 3)
    A = assembly.stiffness(lv).toarray()
    ni = lv.ni
    i = 3 + 3 * ni
    row = A[i].reshape(ni, ni)
    expect = np.full((3, 3), -1 / 3)
    expect[1, 1] = 8 / 3
    np.testing.assert_allclose(row[2:5, 2:5], expect, atol=1e-14)
    assert np.count_nonzero(np.abs(A[i]) > 1e-14) == 9


@pytest.mark.parametrize("d,k,l", [(2, 2, 2), (2, 3, 3), (2, 5, 2), (3, 2, 2), (3, 3, 1)])
def test_discrete_solution_is_exact_for_u_in_Vh(d, k, l):
    """u = prod x_t(1-x_t) lies in V_h for k >= 2, so A u_I = b exactly.

    This pins A (Eq. 2.4, all d gradient terms, the h-scaling) and the load
    vector quadrature jointly against the PDE -Laplace u = f.
    """
    lv = fe.Level(d, k, l)
    u, f = _bubble(d)
    A = assembly.stiffness(lv)
    b = assembly.load_vector(lv, f)
    x = assembly.interpolate(lv, u)
    assert np.abs(A @ x - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("d,k,l", [(2, 1, 3), (2, 4, 2), (3, 2, 2)])
def test_load_vector_integrates_exactly(d, k, l):
    """b^T u_I = int f u for u in V_h; f = 1 + x_0 gives prod(1/6)-type closed forms."""
    lv = fe.Level(d, k, l)
    if k == 1:  # u = hat-type function in V_h: use the discrete identity with Q1
        rng = np.random.default_rng(0)
        x = rng.normal(size=lv.N)
        # int 1 * u_h = sum_i x_i int phi_i = x . b(f=1); compare with mass lumping-free route
        b1 = assembly.load_vector(lv, lambda X: np.ones(len(X)))
        Mc = fe.cell_mass(d, k, lv.h)
        cells = lv.cell_node_indices()
        g2c = lv.global_to_compact()
        full = np.zeros(lv.n1 ** d)
        full[g2c >= 0] = x[g2c[g2c >= 0]]
        ones = np.ones((k + 1) ** d)
        exact = sum(full[c] @ Mc @ ones for c in cells)
        assert abs(x @ b1 - exact) < 1e-13 * np.abs(x).sum()
        return
    u = lambda X: np.prod(X * (1 - X), axis=1)
    b = assembly.load_vector(lv, lambda X: 1.0 + X[:, 0])
    uI = assembly.interpolate(lv, u)
    # int (1 + x0) prod x_t(1-x_t) = (1/6 + 1/12) (1/6)^(d-1)
    exact = (1 / 6 + 1 / 12) * (1 / 6) ** (d - 1)
    assert abs(b @ uI - exact) < 1e-14


@pytest.mark.parametrize("d,k,l", [(2, 1, 3), (2, 2, 3), (2, 3, 2), (3, 1, 2), (3, 2, 2)])
def test_galerkin_identity(d, k, l):
    """Nested spaces: (I^up)^T A_l I^up = A_{l-1} (Section 2.1)."""
    fine, coarse = fe.Level(d, k, l), fe.Level(d, k, l - 1)
    P = assembly.prolongation(fine)
    Af, Ac = assembly.stiffness(fine), assembly.stiffness(coarse)
    G = (P.T @ Af @ P).toarray()
    np.testing.assert_allclose(G, Ac.toarray(), atol=1e-12 * abs(Ac).max())


@pytest.mark.parametrize("d,k,l", [(2, 2, 3), (2, 4, 2), (3, 3, 2)])
def test_prolongation_reproduces_coarse_functions(d, k, l):
    """I^up maps the coarse interpolant of u in V_{l-1} to the fine interpolant."""
    fine, coarse = fe.Level(d, k, l), fe.Level(d, k, l - 1)
    u = lambda X: np.prod(X * (1 - X), axis=1) * (1 + 0.5 * X[:, 0] ** (k - 2))
    P = assembly.prolongation(fine)
    np.testing.assert_allclose(P @ assembly.interpolate(coarse, u), assembly.interpolate(fine, u),
                               atol=1e-14)


@pytest.mark.parametrize("d,k,l", [(2, 3, 3), (3, 2, 2)])
def test_stiffness_matches_kronecker_sum_of_1d_matrices(d, k, l):
    """Secondary cross-check: A = sum_t (x)_s (K or M) of global 1D matrices (Eq. 2.11/2.12)."""
    lv = fe.Level(d, k, l)
    K1, M1 = fe.reference_matrices_1d(k)
    n1, h = lv.n1, lv.h
    Kg, Mg = np.zeros((n1, n1)), np.zeros((n1, n1))
    for c in range(lv.ncell):
        s = slice(k * c, k * c + k + 1)
        Kg[s, s] += K1 / h
        Mg[s, s] += M1 * h
    Kg, Mg = Kg[1:-1, 1:-1], Mg[1:-1, 1:-1]
    A = np.zeros((lv.N, lv.N))
    for t in range(d):
        mats = [Kg if s == t else Mg for s in range(d)]
        T = mats[d - 1]
        for s in range(d - 2, -1, -1):
            T = np.kron(T, mats[s])
        A += T
    np.testing.assert_allclose(assembly.stiffness(lv).toarray(), A, atol=1e-12 * abs(A).max())
    assert sp.issparse(assembly.stiffness(lv))
