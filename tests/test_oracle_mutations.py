"""Planted mistakes in the oracle must be caught by its pins.

Each test patches one plausible mistake into the oracle (on the CPU, inside
the test only) and checks that the corresponding pin fails.  This shows the
pins are sensitive to a dropped term, a wrong sign or index, and a
transposed operand.
"""

import numpy as np
import pytest

from oracle import assembly, fe, multigrid, smoothers


def _bubble_residual(d, k, l):
    lv = fe.Level(d, k, l)
    u = lambda X: np.prod(X * (1 - X), axis=1)

    def f(X):
        s = np.zeros(len(X))
        for t in range(d):
            s += 2 * np.prod(np.delete(X * (1 - X), t, axis=1), axis=1)
        return s
    A = assembly.stiffness(lv)
    b = assembly.load_vector(lv, f)
    return np.abs(A @ assembly.interpolate(lv, u) - b).max() / np.abs(b).max()


def test_dropped_gradient_term_is_caught(monkeypatch):
    """Forgetting the last direction's gradient term breaks A u_I = b for u in V_h."""
    orig = fe.cell_stiffness
    monkeypatch.setattr(fe, "cell_stiffness", lambda d, k, h: orig(d, k, h) - _last_term(d, k, h))
    assert _bubble_residual(2, 2, 2) > 1e-3
    assert _bubble_residual(3, 2, 1) > 1e-3


def _last_term(d, k, h):
    z = fe.gll_nodes(k)
    xq, wq = fe.gauss_points(k + 1)
    V, D = fe.lagrange_values(z, xq), fe.lagrange_derivatives(z, xq)
    mats = [V] * (d - 1) + [D]
    G = fe.tensor_basis_at(mats, d, k + 1, k + 1)
    Q = fe.multi_indices(k + 1, d)
    W = np.prod([wq[Q[:, t]] for t in range(d)], axis=0)
    return (G * W) @ G.T * h ** (d - 2)


def test_wrong_h_scaling_is_caught(monkeypatch):
    orig = fe.cell_stiffness
    monkeypatch.setattr(fe, "cell_stiffness", lambda d, k, h: orig(d, k, h) / h)
    assert _bubble_residual(2, 2, 2) > 1e-3


def test_wrong_correction_sign_is_caught(monkeypatch):
    """A sign error in the local correction moves the Q1 smoother away from point GS."""
    lv = fe.Level(2, 1, 3)
    A = assembly.stiffness(lv)
    ps = smoothers.PatchSolver(lv, A)
    rng = np.random.default_rng(0)
    x0, b = rng.normal(size=lv.N), rng.normal(size=lv.N)
    good = smoothers.multiplicative(A, ps, x0, b)
    orig = smoothers.PatchSolver.solve
    monkeypatch.setattr(smoothers.PatchSolver, "solve", lambda self, R: -orig(self, R))
    bad = smoothers.multiplicative(A, ps, x0, b)
    assert np.abs(good - bad).max() > 1e-2


def test_mirrored_interpolation_breaks_galerkin_pin(monkeypatch):
    """Coarse basis evaluated at the mirrored reference coordinate inside each coarse cell."""
    fine, coarse = fe.Level(2, 3, 3), fe.Level(2, 3, 2)
    Af, Ac = assembly.stiffness(fine), assembly.stiffness(coarse)
    orig = fe.lagrange_values
    monkeypatch.setattr(fe, "lagrange_values", lambda nodes, x: orig(nodes, 1.0 - np.asarray(x)))
    P = assembly.prolongation(fine)
    G = (P.T @ Af @ P).toarray()
    assert np.abs(G - Ac.toarray()).max() > 1e-3 * np.abs(Ac).max()


def test_same_order_post_smoothing_breaks_symmetry_pin():
    H = multigrid.Hierarchy(2, 2, 3, symmetric=True)
    H.symmetric = False
    N = H.levels[3].N
    B = np.stack([H.vcycle(3, np.eye(N)[i]) for i in range(N)], axis=1)
    assert np.abs(B - B.T).max() > 1e-6 * np.abs(B).max()


def test_extra_smoothing_step_breaks_the_operator_pin():
    """A V-cycle that smooths twice before the coarse correction no longer
    equals Algorithm 1's product of error propagators."""
    from test_oracle_multigrid import _patch_sets, _smoothing_propagator, _vcycle_matrix
    H = multigrid.Hierarchy(2, 2, 3, symmetric=True)
    H.n_pre = 2
    B = None
    for l in range(1, 4):
        A = H.A[l].toarray()
        if l == 1:
            B = np.linalg.inv(A)
            continue
        sets = _patch_sets(2, 2, l)
        S = _smoothing_propagator(A, sets, range(4))
        Sr = _smoothing_propagator(A, sets, range(3, -1, -1))
        P = H.P[l].toarray()
        E = Sr @ (np.eye(len(A)) - P @ B @ P.T @ A) @ S
        B = (np.eye(len(A)) - E) @ np.linalg.inv(A)
    assert np.abs(_vcycle_matrix(H) - B).max() > 1e-6 * np.abs(B).max()


def test_coarse_right_hand_side_on_too_few_levels_breaks_the_3d_count_pin(monkeypatch):
    """Full multigrid whose nested iteration gets no right-hand side below the
    finest level (its start is then zero) needs more V-cycles: the count the
    two-sided 3D pin compares with Table 2 is sensitive to that mistake."""
    f = lambda X: np.ones(len(X))
    good = multigrid.fmg_iterations(3, 2, 3, f)
    orig = assembly.load_vector

    def zero_below_finest(level, ff):
        b = orig(level, ff)
        return b if level.l == 3 else 0.0 * b
    monkeypatch.setattr(assembly, "load_vector", zero_below_finest)
    assert multigrid.fmg_iterations(3, 2, 3, f) > good
