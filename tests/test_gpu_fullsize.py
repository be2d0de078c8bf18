"""Parity at the benchmark's full size (3D Q4 on 32^3 cells, 2,048,383 DoFs).

The global matrix cannot be assembled here, so every check uses outputs the
oracle computes one by one from the same definitions (oracle.local): sampled
patch corrections of every colour pass, sampled rows of A x, of the
prolongation and of the restriction; and properties of the full solve.  The
handles are autotuned first, as bench.py does, so the launches checked are
the ones it times.
"""

import numpy as np
import pytest

from oracle import fe, local, smoothers
from synthetic import normal_vector, uniform_vector

from gpu_helpers import as_prec

pytestmark = pytest.mark.gpu

import paper_2405_19004_gb300 as vps  # noqa: E402

D, K, L = 3, 4, 5
N_SAMPLE = 24


def _full(P, lev, level):
    """Level-layout tensor -> full-grid numpy vector (n1^d, padding dropped)."""
    n1, px, _ = P.layout(level)
    a = lev.double().cpu().numpy().reshape(n1, n1, px)[:, :, :n1]
    return a.reshape(-1)


@pytest.fixture(scope="module", params=[vps.VPS_FP32, vps.VPS_FP64], ids=["fp32", "fp64"])
def handle(request):
    P = vps.Poisson(D, K, L, precision=request.param)
    P.vps_autotune(None)
    return P


def test_every_colour_pass_on_sampled_patches(handle):
    import torch
    P = handle
    prec = 1 if P.precision == vps.VPS_FP32 else 0
    lv = fe.Level(D, K, L)
    mats = local.patch_matrices(lv)
    N = P.n_interior()
    x = P.to_level(torch.as_tensor(as_prec(normal_vector(N, 41), prec), device="cuda"))
    b = P.to_level(torch.as_tensor(as_prec(normal_vector(N, 42), prec), device="cuda"))
    bf = _full(P, b, L)
    rng = np.random.default_rng(43)
    V = smoothers.vertices(lv)
    col = smoothers.colour_of(V)
    for c in range(2 ** D):
        before = _full(P, x, L)
        P.vps_smooth_colour(L, c, b, x)
        after = _full(P, x, L)
        js = rng.choice(np.nonzero(col == c)[0], size=N_SAMPLE, replace=False)
        for j in js:
            gi, u = local.patch_update(lv, before, bf, V[j], mats)
            if prec == 0:
                err = np.linalg.norm(after[gi] - before[gi] - u) / np.linalg.norm(u)
                assert err <= 1e-12, (c, j, err)
            else:  # FP32: compare the updated values, relative to their size
                ref = before[gi] + u
                err = np.abs(after[gi] - ref).max() / np.abs(ref).max()
                assert err <= 1e-5, (c, j, err)
        # nothing outside the interiors of this colour's patches moved: those
        # interiors form a tensor product of 1D node sets
        masks = []
        for t in range(D):
            par = (c >> t) & 1
            m1 = np.zeros(lv.n1, dtype=bool)
            for v in range(1 + par, 2 ** L, 2):
                m1[K * (v - 1) + 1:K * (v + 1)] = True
            masks.append(m1)
        inside = masks[2][:, None, None] & masks[1][None, :, None] & masks[0][None, None, :]
        moved = after != before
        assert not np.any(moved & ~inside.reshape(-1))


def test_operator_on_sampled_rows(handle):
    import torch
    P = handle
    prec = 1 if P.precision == vps.VPS_FP32 else 0
    lv = fe.Level(D, K, L)
    N = P.n_interior()
    x = P.to_level(torch.as_tensor(as_prec(normal_vector(N, 44), prec), device="cuda"))
    y = P.empty_level(L)
    P.vps_apply(L, x, y)
    xf, yf = _full(P, x, L), _full(P, y, L)
    rng = np.random.default_rng(45)
    nodes = rng.integers(1, lv.n1 - 1, size=(4 * N_SAMPLE, D))
    ref = local.apply_rows(lv, xf, nodes)
    got = yf[sum(nodes[:, t] * lv.n1 ** t for t in range(D))]
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= (1e-12 if prec == 0 else 2e-6) * scale


def test_transfers_on_sampled_rows(handle):
    import torch
    P = handle
    prec = 1 if P.precision == vps.VPS_FP32 else 0
    fine, coarse = fe.Level(D, K, L), fe.Level(D, K, L - 1)
    xc = P.to_level(torch.as_tensor(as_prec(normal_vector(coarse.N, 46), prec), device="cuda"), L - 1)
    xf = P.empty_level(L)
    P.vps_prolongate_add(L, xc, xf)
    rng = np.random.default_rng(47)
    nodes = rng.integers(1, fine.n1 - 1, size=(4 * N_SAMPLE, D))
    ref = local.prolongate_rows(fine, _full(P, xc, L - 1), nodes)
    got = _full(P, xf, L)[sum(nodes[:, t] * fine.n1 ** t for t in range(D))]
    assert np.abs(got - ref).max() <= (1e-13 if prec == 0 else 2e-6) * np.abs(ref).max()
    rf = P.to_level(torch.as_tensor(as_prec(normal_vector(fine.N, 48), prec), device="cuda"))
    rc = P.empty_level(L - 1)
    P.vps_restrict(L, rf, rc)
    cn = rng.integers(1, coarse.n1 - 1, size=(N_SAMPLE, D))
    ref = local.restrict_rows(fine, _full(P, rf, L), cn)
    got = _full(P, rc, L - 1)[sum(cn[:, t] * coarse.n1 ** t for t in range(D))]
    assert np.abs(got - ref).max() <= (1e-12 if prec == 0 else 1e-5) * np.abs(ref).max()


def test_full_solve_reaches_the_tolerance(handle):
    import torch
    P = handle
    N = P.n_interior()
    b = torch.as_tensor(uniform_vector(N, 1), device="cuda")
    x = torch.zeros_like(b)
    it, rel = P.vps_solve(b, x, 1e-10, 100)
    assert rel <= 1e-10 and it <= 10
    # independent residual in FP64 through a separate FP64 handle's operator
    Q = vps.Poisson(D, K, L, precision=vps.VPS_FP64)
    xl, bl, yl = Q.to_level(x), Q.to_level(b), Q.empty_level(L)
    Q.vps_apply(L, xl, yl)
    r = torch.linalg.norm(Q.to_compact(yl) - b) / torch.linalg.norm(b)
    assert r.item() <= 1.05e-10
