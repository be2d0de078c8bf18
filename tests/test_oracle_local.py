"""Pins of the oracle's single-patch / single-row evaluations against the global oracle."""

import numpy as np
import pytest

from oracle import assembly, fe, local, smoothers


def _full(lv, x):
    g2c = lv.global_to_compact()
    out = np.zeros(lv.n1 ** lv.d)
    out[g2c >= 0] = x[g2c[g2c >= 0]]
    return out


@pytest.mark.parametrize("d,k,l", [(2, 2, 3), (3, 2, 2), (3, 3, 2)])
def test_apply_rows_equals_global_product(d, k, l):
    lv = fe.Level(d, k, l)
    A = assembly.stiffness(lv)
    rng = np.random.default_rng(7)
    x = rng.normal(size=lv.N)
    y = A @ x
    Q = fe.multi_indices(lv.ni, d)
    pick = rng.choice(lv.N, size=25, replace=False)
    got = local.apply_rows(lv, _full(lv, x), Q[pick] + 1)
    np.testing.assert_allclose(got, y[pick], rtol=1e-13, atol=1e-13 * np.abs(y).max())


@pytest.mark.parametrize("d,k,l", [(2, 3, 3), (3, 2, 2)])
def test_patch_update_equals_colour_zero_of_global_smoother(d, k, l):
    lv = fe.Level(d, k, l)
    A = assembly.stiffness(lv)
    ps = smoothers.PatchSolver(lv, A)
    rng = np.random.default_rng(8)
    x0, b = rng.normal(size=lv.N), rng.normal(size=lv.N)
    x1 = smoothers.multiplicative(A, ps, x0, b, colours=[0])
    xf, bf = _full(lv, x0), _full(lv, b)
    g2c = lv.global_to_compact()
    mats = local.patch_matrices(lv)
    np.testing.assert_allclose(mats[1], ps.Aj, atol=1e-13 * np.abs(ps.Aj).max())
    for v in smoothers.vertices(lv):
        if smoothers.colour_of(v) != 0:
            continue
        gi, u = local.patch_update(lv, xf, bf, v, mats)
        np.testing.assert_allclose(x0[g2c[gi]] + u, x1[g2c[gi]], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("d,k,l", [(2, 3, 3), (3, 2, 3)])
def test_prolongate_rows_equals_global_prolongation(d, k, l):
    fine, coarse = fe.Level(d, k, l), fe.Level(d, k, l - 1)
    P = assembly.prolongation(fine)
    rng = np.random.default_rng(9)
    xc = rng.normal(size=coarse.N)
    y = P @ xc
    Q = fe.multi_indices(fine.ni, d)
    pick = rng.choice(fine.N, size=30, replace=False)
    got = local.prolongate_rows(fine, _full(coarse, xc), Q[pick] + 1)
    np.testing.assert_allclose(got, y[pick], atol=1e-13)


@pytest.mark.parametrize("d,k,l", [(2, 3, 3), (3, 2, 3), (2, 1, 4)])
def test_restrict_rows_equals_global_restriction(d, k, l):
    fine, coarse = fe.Level(d, k, l), fe.Level(d, k, l - 1)
    P = assembly.prolongation(fine)
    rng = np.random.default_rng(10)
    rf = rng.normal(size=fine.N)
    y = P.T @ rf
    Q = fe.multi_indices(coarse.ni, d)
    pick = rng.choice(coarse.N, size=min(30, coarse.N), replace=False)
    got = local.restrict_rows(fine, _full(fine, rf), Q[pick] + 1)
    np.testing.assert_allclose(got, y[pick], atol=1e-13)


@pytest.mark.parametrize("d,k,l", [(2, 3, 3), (3, 2, 2), (2, 1, 3)])
def test_boundary_solve_equals_fused_update(d, k, l):
    """Section 3.2: with the exact local solver, x^I + A_j^{-1} R_j (b - Abar x)
    equals A_j^{-1} (b^I - A^{IB} x^B), and the result does not depend on x^I."""
    lv = fe.Level(d, k, l)
    mats = local.patch_matrices(lv)
    rng = np.random.default_rng(11)
    xf, bf = _full(lv, rng.normal(size=lv.N)), _full(lv, rng.normal(size=lv.N))
    for v in smoothers.vertices(lv)[:6]:
        gi, u = local.patch_update(lv, xf, bf, v, mats)
        gi2, xi = local.patch_boundary_solve(lv, xf, bf, v, mats)
        assert np.array_equal(gi, gi2)
        np.testing.assert_allclose(xi, xf[gi] + u, rtol=1e-11, atol=1e-11 * np.abs(xi).max())
        x2 = xf.copy()
        x2[gi] = rng.normal(size=len(gi))  # other interior values: same new interior
        _, xi2 = local.patch_boundary_solve(lv, x2, bf, v, mats)
        np.testing.assert_allclose(xi2, xi, rtol=1e-12, atol=1e-12 * np.abs(xi).max())
        gi3, u3 = local.patch_update(lv, x2, bf, v, mats)
        np.testing.assert_allclose(x2[gi3] + u3, xi, rtol=1e-11, atol=1e-11 * np.abs(xi).max())
