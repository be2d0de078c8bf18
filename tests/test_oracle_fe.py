"""Pins of the oracle's finite-element building blocks (Section 2).

Each quantity is checked against something other than the oracle itself:
closed forms derived by hand, exact polynomial integrals computed with
numpy's power-basis polynomials (a different route from the Lagrange basis +
Gauss quadrature of the oracle), and structural invariants.
"""

import numpy as np
import pytest
from numpy.polynomial import Polynomial as Poly

from oracle import fe


def test_gll_nodes_closed_forms():
    # Gauss-Lobatto points on [-1,1]: k=2: 0; k=3: +-1/sqrt5; k=4: 0, +-sqrt(3/7);
    # k=5: +-sqrt(1/3 -+ 2 sqrt7/21).  Mapped to [0,1].
    m = lambda t: (np.asarray(t) + 1.0) / 2.0
    np.testing.assert_allclose(fe.gll_nodes(1), [0, 1], atol=0)
    np.testing.assert_allclose(fe.gll_nodes(2), m([-1, 0, 1]), atol=1e-15)
    a = 1 / np.sqrt(5)
    np.testing.assert_allclose(fe.gll_nodes(3), m([-1, -a, a, 1]), atol=1e-15)
    b = np.sqrt(3 / 7)
    np.testing.assert_allclose(fe.gll_nodes(4), m([-1, -b, 0, b, 1]), atol=1e-15)
    c1 = np.sqrt(1 / 3 - 2 * np.sqrt(7) / 21)
    c2 = np.sqrt(1 / 3 + 2 * np.sqrt(7) / 21)
    np.testing.assert_allclose(fe.gll_nodes(5), m([-1, -c2, -c1, c1, c2, 1]), atol=1e-15)


def test_q1_q2_reference_matrices_closed_form():
    K, M = fe.reference_matrices_1d(1)
    np.testing.assert_allclose(K, [[1, -1], [-1, 1]], atol=1e-15)
    np.testing.assert_allclose(M, np.array([[2, 1], [1, 2]]) / 6, atol=1e-15)
    # Q2 on nodes 0, 1/2, 1: l0 = 2x^2-3x+1, l1 = 4x-4x^2, l2 = 2x^2-x.
    K, M = fe.reference_matrices_1d(2)
    np.testing.assert_allclose(K, np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / 3, atol=1e-14)
    np.testing.assert_allclose(M, np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) / 30, atol=1e-15)


@pytest.mark.parametrize("k", range(1, 9))
def test_reference_matrices_invariants(k):
    K, M = fe.reference_matrices_1d(k)
    np.testing.assert_allclose(K, K.T, atol=1e-13)
    np.testing.assert_allclose(M, M.T, atol=1e-15)
    np.testing.assert_allclose(K @ np.ones(k + 1), 0, atol=1e-11 * abs(K).max())
    assert abs(M.sum() - 1.0) < 1e-14          # int_0^1 (sum_i l_i)^2 = 1
    assert np.linalg.eigvalsh(M).min() > 0
    assert np.linalg.eigvalsh(K).min() > -1e-10 * abs(K).max()


@pytest.mark.parametrize("k", [1, 2, 3, 5, 7])
def test_reference_matrices_integrate_polynomials_exactly(k):
    rng = np.random.default_rng(k)
    z = fe.gll_nodes(k)
    K, M = fe.reference_matrices_1d(k)
    for _ in range(3):
        p, q = Poly(rng.normal(size=k + 1)), Poly(rng.normal(size=k + 1))
        mass = (p * q).integ()
        stiff = (p.deriv() * q.deriv()).integ()
        assert abs(p(z) @ M @ q(z) - (mass(1) - mass(0))) < 1e-12
        assert abs(p(z) @ K @ q(z) - (stiff(1) - stiff(0))) < 1e-10 * (1 + abs(stiff(1)))


@pytest.mark.parametrize("d,k", [(2, 1), (2, 3), (3, 1), (3, 2)])
def test_cell_stiffness_exact_on_tensor_polynomials(d, k):
    """u^T A^K v = int_cell grad u . grad v for u, v in Q_k on [0,h]^d."""
    rng = np.random.default_rng(10 * d + k)
    h = 0.37
    z = fe.gll_nodes(k) * h
    A = fe.cell_stiffness(d, k, h)
    Mc = fe.cell_mass(d, k, h)
    idx = fe.multi_indices(k + 1, d)
    integ = lambda poly: (lambda P: P(h) - P(0))(poly.integ())
    for _ in range(2):
        pu = [Poly(rng.normal(size=k + 1)) for _ in range(d)]
        pv = [Poly(rng.normal(size=k + 1)) for _ in range(d)]
        uI = np.prod([pu[t](z)[idx[:, t]] for t in range(d)], axis=0)
        vI = np.prod([pv[t](z)[idx[:, t]] for t in range(d)], axis=0)
        exact = 0.0
        for t in range(d):
            term = integ(pu[t].deriv() * pv[t].deriv())
            for s in range(d):
                if s != t:
                    term *= integ(pu[s] * pv[s])
            exact += term
        mass = np.prod([integ(pu[t] * pv[t]) for t in range(d)])
        assert abs(uI @ A @ vI - exact) < 1e-11 * (1 + abs(exact))
        assert abs(uI @ Mc @ vI - mass) < 1e-13 * (1 + abs(mass))


def test_level_sizes_and_numbering():
    lv = fe.Level(3, 4, 5)
    assert lv.n1 == 129 and lv.ni == 127 and lv.N == 127 ** 3
    lv = fe.Level(2, 2, 4)
    assert lv.n1 == 33 and lv.N == 961
    g2c = lv.global_to_compact()
    assert (g2c >= 0).sum() == lv.N
    assert g2c[0] == -1 and g2c[lv.n1 + 1] == 0 and g2c[lv.n1 + 2] == 1
    x = lv.node_coords_1d()
    assert x[0] == 0.0 and abs(x[-1] - 1.0) < 1e-15 and np.all(np.diff(x) > 0)
