"""The exact coarse solve (global fast diagonalisation, Algorithm 1's coarse
grid solver) in each of its forms -- one cooperative launch with grid
barriers between its passes or one launch per pass, tiles of 32 or 64
outputs -- against the passes launched one by one (bit for bit) and against
the oracle's direct solve."""

import pytest

from synthetic import normal_vector

from gpu_helpers import oracle_level, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

import paper_2405_19004_gb300 as vps  # noqa: E402


def _solve_exact(P, L, b, solver):
    P.vps_set_coarse_solver(solver)
    x = P.empty_level(L)
    x.fill_(5.0)  # boundary and padding must come back as 0
    P.vps_vcycle(to_dev(P, b, L), x)
    P.vps_check_waits()
    return x


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d,k,L", [(2, 3, 4), (3, 2, 3), (2, 7, 2), (3, 5, 2), (2, 4, 6), (3, 4, 4)])
def test_cooperative_coarse_solve_equals_passes_and_the_direct_solve(d, k, L, prec):
    import scipy.sparse.linalg as spla
    import torch
    P = vps.Poisson(d, k, L, precision=prec)
    P.vps_set_coarse_level(L)  # the V-cycle is then the exact solve
    n1 = P.layout(L)[0]
    b = normal_vector((n1 - 2) ** d, 61)
    ref = _solve_exact(P, L, b, vps.VPS_COARSE_PASSES)
    for solver in (vps.VPS_COARSE_COOPERATIVE, vps.VPS_COARSE_WIDE_TILES,
                   vps.VPS_COARSE_COOPERATIVE | vps.VPS_COARSE_WIDE_TILES):
        got = _solve_exact(P, L, b, solver)
        assert torch.equal(got, ref), solver
    if (n1 - 2) ** d <= (70000 if d == 2 else 8000):  # the oracle's sparse direct solve
        lv, A, _ = oracle_level(d, k, L)
        tol = 1e-11 if prec == 0 else 1e-5
        bb = b if prec == 0 else b.astype("float32").astype("float64")
        assert rel_err(to_host(P, got, L), spla.spsolve(A.tocsc(), bb)) <= tol


@pytest.mark.parametrize("d,k,L", [(3, 4, 5), (2, 2, 6)])
def test_solve_with_cooperative_coarse_solve_equals_passes(d, k, L):
    """Full CG solves through CUDA graphs (the cooperative launch captured in
    the V-cycle graph) with the default coarse level: the same bits."""
    import torch
    from synthetic import uniform_vector
    res = []
    for solver in (vps.VPS_COARSE_PASSES, vps.VPS_COARSE_COOPERATIVE | vps.VPS_COARSE_WIDE_TILES):
        P = vps.Poisson(d, k, L, precision=vps.VPS_FP32)
        P.vps_set_coarse_solver(solver)
        assert P.vps_get_coarse_solver() == solver
        b = torch.as_tensor(uniform_vector(P.n_interior(), 62), device="cuda")
        x = torch.zeros_like(b)
        it, rel = P.vps_solve(b, x, 1e-10, 100)
        assert rel <= 1e-10
        res.append((it, x))
    assert res[0][0] == res[1][0] and torch.equal(res[0][1], res[1][1])


def test_coarse_solver_argument_checked():
    P = vps.Poisson(2, 2, 3)
    with pytest.raises(vps.VpsError):
        P.vps_set_coarse_solver(4)
