"""Flexible GMRES with the V-cycle of Algorithm 1 (the paper's outer solver).

The oracle runs the same method (``multigrid.fgmres``: right
preconditioning by the non-symmetric V-cycle on the same hierarchy,
modified Gram-Schmidt); the GPU orthogonalises by classical Gram-Schmidt
applied twice, equal in exact arithmetic.  FP64 handles must take the
oracle's iteration count and reach its solution; FP32 handles (V-cycle in
FP32, double-float outer operator) within one iteration.
"""

import numpy as np
import pytest

from oracle import multigrid
from synthetic import uniform_vector

pytestmark = pytest.mark.gpu

import paper_2405_19004_gb300 as vps  # noqa: E402


def _run(d, k, L, prec, restart, rtol, smoother=vps.VPS_MULTIPLICATIVE, damping=1.0):
    import torch
    P = vps.Poisson(d, k, L, precision=prec, smoother=smoother, damping=damping)
    n = P.n_interior()
    b = uniform_vector(n, 91)
    bt = torch.as_tensor(b, device="cuda")
    xt = torch.zeros_like(bt)
    it, rel = P.vps_gmres(bt, xt, rtol, restart, 300)
    return P, b, xt.cpu().numpy(), it, rel


@pytest.mark.parametrize("restart", [30, 3])
@pytest.mark.parametrize("d,k,L", [(2, 2, 4), (2, 3, 3), (3, 2, 3), (3, 3, 3), (2, 1, 5)])
def test_gmres_matches_the_oracle(d, k, L, restart):
    P, b, x, it, rel = _run(d, k, L, vps.VPS_FP64, restart, 1e-9)
    H = multigrid.Hierarchy(d, k, L, symmetric=False, coarse_level=P.vps_get_coarse_level())
    xo, ito, relo, _ = multigrid.fgmres(H.A[L], b, H.precondition, rtol=1e-9, restart=restart)
    assert it == ito
    assert rel <= 1e-9
    assert np.linalg.norm(b - H.A[L] @ x) <= 1.01e-9 * np.linalg.norm(b)
    assert np.linalg.norm(x - xo) <= 1e-7 * np.linalg.norm(xo)


@pytest.mark.parametrize("d,k,L", [(2, 2, 4), (3, 2, 3), (3, 4, 2)])
def test_mixed_precision_gmres(d, k, L):
    P, b, x, it, rel = _run(d, k, L, vps.VPS_FP32, 30, 1e-9)
    assert P.vps_get_outer_operator() == vps.VPS_OUTER_DOUBLE_FLOAT
    H = multigrid.Hierarchy(d, k, L, symmetric=False, coarse_level=P.vps_get_coarse_level())
    _, ito, _, _ = multigrid.fgmres(H.A[L], b, H.precondition, rtol=1e-9)
    assert abs(it - ito) <= 1
    assert np.linalg.norm(b - H.A[L] @ x) <= 1.01e-9 * np.linalg.norm(b)


def test_gmres_with_the_additive_smoother():
    P, b, x, it, rel = _run(2, 3, 3, vps.VPS_FP64, 30, 1e-9, vps.VPS_ADDITIVE, 0.35)
    H = multigrid.Hierarchy(2, 3, 3, smoother="additive", omega=0.35, symmetric=False,
                            coarse_level=P.vps_get_coarse_level())
    _, ito, _, _ = multigrid.fgmres(H.A[3], b, H.precondition, rtol=1e-9)
    assert it == ito and rel <= 1e-9


def test_gmres_rejects_bad_arguments():
    import torch
    P = vps.Poisson(2, 2, 3, precision=vps.VPS_FP64)
    b = torch.ones(P.n_interior(), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    for rtol, restart, max_it in ((0.0, 30, 10), (1e-9, 0, 10), (1e-9, 30, 0), (1e-9, 600, 10)):
        with pytest.raises(vps.VpsError) as e:
            P.vps_gmres(b, x, rtol, restart, max_it)
        assert e.value.code == vps.VPS_EINVAL
