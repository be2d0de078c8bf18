"""Kernel structures of the multiplicative smoother (Section 3.1): Separate,
Global and Global with the dense inverse as local solver give the same
smoothing step as the fused kernel and as the oracle."""

import numpy as np
import pytest

from oracle import smoothers
from synthetic import normal_vector, uniform_vector

from gpu_helpers import TOL, as_prec, oracle_level, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

import paper_2405_19004_gb300 as vps  # noqa: E402

KINDS = [vps.VPS_KERNEL_SEPARATE, vps.VPS_KERNEL_GLOBAL, vps.VPS_KERNEL_GLOBAL_INVERSE]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d,k,l", [(2, 1, 4), (2, 3, 3), (2, 7, 2), (3, 1, 3), (3, 2, 3), (3, 4, 2),
                                   (3, 5, 2)])
def test_kernel_structures_match_the_oracle(d, k, l, prec, kind):
    lv, A, ps = oracle_level(d, k, l)
    x0 = as_prec(normal_vector(lv.N, 51), prec)
    b = as_prec(normal_vector(lv.N, 52), prec)
    ref = smoothers.multiplicative(A, ps, x0, b)
    P = vps.Poisson(d, k, l, precision=prec)
    P.vps_set_smoother_kernel(kind)
    assert P.vps_get_smoother_kernel() == kind
    for v in (0, 1, 3, 4):  # the block shape of the solve kernels follows the level's variant
        try:
            P.vps_set_smooth_variant(0, v)
        except vps.VpsError:
            continue
        xg = to_dev(P, x0, l)
        P.vps_smooth(l, to_dev(P, b, l), xg, 1)
        assert rel_err(to_host(P, xg, l), ref) <= TOL[prec], v
        xg = to_dev(P, x0, l)
        bg = to_dev(P, b, l)
        for c in range(2 ** d):
            P.vps_smooth_colour(l, c, bg, xg)
        assert rel_err(to_host(P, xg, l), ref) <= TOL[prec], v


def test_dense_inverse_limit_and_additive_handles():
    P = vps.Poisson(3, 6, 2, precision=vps.VPS_FP32)
    with pytest.raises(vps.VpsError) as e:
        P.vps_set_smoother_kernel(vps.VPS_KERNEL_GLOBAL_INVERSE)
    assert e.value.code == vps.VPS_EINVAL
    P.vps_set_smoother_kernel(vps.VPS_KERNEL_SEPARATE)  # other structures work at k = 6
    Q = vps.Poisson(2, 2, 3, precision=vps.VPS_FP64, smoother=vps.VPS_ADDITIVE, damping=0.35)
    with pytest.raises(vps.VpsError):
        Q.vps_set_smoother_kernel(vps.VPS_KERNEL_GLOBAL)
    with pytest.raises(vps.VpsError):
        P.vps_set_smoother_kernel(4)


@pytest.mark.parametrize("kind", KINDS)
def test_solve_with_each_structure_takes_the_fused_iterations(kind):
    import torch
    d, k, L = 3, 3, 3
    lv, A, _ = oracle_level(d, k, L)
    b = torch.as_tensor(uniform_vector(lv.N, 53), device="cuda")
    its = []
    for kd in (vps.VPS_KERNEL_FUSED, kind):
        P = vps.Poisson(d, k, L, precision=vps.VPS_FP64)
        P.vps_set_smoother_kernel(kd)
        x = torch.zeros_like(b)
        it, rel = P.vps_solve(b, x, 1e-10, 100)
        its.append(it)
        assert np.linalg.norm(b.cpu().numpy() - A @ x.cpu().numpy()) <= 1.01e-10 * np.linalg.norm(b.cpu().numpy())
    assert its[0] == its[1]
